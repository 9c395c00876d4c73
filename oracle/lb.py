"""Oracle for the discretised Landau-Brazovskii energy, its gradient and Hessian (paper §2).

Test infrastructure, not product code (see oracle/__init__.py).  Everything is FP64.

Readings of the paper used here (each is listed with its reason in the design notes):
  * Lambda_k = xi^2 (1 - |Bk|^2)^2.  The paper prints [1 - k^T k]^2 (§2, eq.
    `interaction_bulk_energy` and the Hessian formulas after it) where k must be the
    reciprocal vector Bk of the expansion; xi = 1 reproduces the paper exactly.
  * A = diag(L_1..L_d) (rectangular box), so B = 2 pi A^{-T} = diag(2 pi / L_a).
  * The F-term convolution sums over k1+...=0 are evaluated pseudo-spectrally, i.e.
    as (1/N) sum_x F(psi(x)) in physical space (the remark after eq.
    `interaction_bulk_energy`), with wavevector sums taken modulo M (aliasing kept).
  * Unknowns are zero-mean real fields; the paper's Euclidean metric on Fourier
    coefficients equals <u,v>_N = (1/N) sum_x u v by Parseval, so gradients and
    Hessian-vector products are returned as physical fields in that metric and
    projected onto zero mean (P = [0, I_{N-1}] of §3 removes the k = 0 coefficient).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import fft


@dataclass(frozen=True)
class Problem:
    """Grid shape (array order, last axis contiguous), box lengths per array axis,
    and the model parameters xi, tau, gamma of eq. `lb_energy`."""

    shape: tuple
    box: tuple
    xi: float
    tau: float
    gamma: float

    @property
    def n(self) -> int:
        return int(np.prod(self.shape))

    @staticmethod
    def from_workload(w) -> "Problem":
        return Problem(tuple(w.shape), tuple(float(b) for b in w.box),
                       float(w.xi), float(w.tau), float(w.gamma))


def bk_squared(p: Problem) -> np.ndarray:
    """|Bk|^2 on the full spectrum grid, B = diag(2 pi / L_a) (paper §2)."""
    out = np.zeros(p.shape, dtype=np.float64)
    for a, (m, length) in enumerate(zip(p.shape, p.box)):
        k = fft.wavenumbers(m).astype(np.float64) * (2.0 * np.pi / length)
        sh = [1] * len(p.shape)
        sh[a] = m
        out = out + (k * k).reshape(sh)
    return out


def lam(p: Problem) -> np.ndarray:
    """Diagonal of grad^2 G in reciprocal space: xi^2 (1 - |Bk|^2)^2 (paper §2)."""
    q = bk_squared(p)
    return p.xi ** 2 * (1.0 - q) ** 2


# Bulk density F(psi) = tau/2 psi^2 - gamma/6 psi^3 + psi^4/24 (eq. `lb_energy`)
def f0(p: Problem, u):
    return p.tau / 2.0 * u ** 2 - p.gamma / 6.0 * u ** 3 + u ** 4 / 24.0


def f1(p: Problem, u):
    """Gamma = F'(psi) = tau psi - gamma/2 psi^2 + psi^3/6 (paper §2, grad F)."""
    return p.tau * u - p.gamma / 2.0 * u ** 2 + u ** 3 / 6.0


def f2(p: Problem, u):
    """Gamma' = F''(psi) = tau - gamma psi + psi^2/2 (paper §2, grad^2 F)."""
    return p.tau - p.gamma * u + u ** 2 / 2.0


def f3(p: Problem, u):
    """F'''(psi) = -gamma + psi."""
    return -p.gamma + u


def inner(u: np.ndarray, v: np.ndarray) -> float:
    """<u, v>_N = (1/N) sum_x u(x) v(x) for real fields (paper §2)."""
    return float(np.mean(np.asarray(u, np.float64) * np.asarray(v, np.float64)))


def norm(u: np.ndarray) -> float:
    return float(np.sqrt(inner(u, u)))


def project(u: np.ndarray) -> np.ndarray:
    """P^T P: remove the k = 0 coefficient, i.e. the mean (paper §3, P = [0, I])."""
    u = np.asarray(u, dtype=np.float64)
    return u - u.mean()


def energy_parts(p: Problem, psi: np.ndarray, direct: bool = False):
    """(G, F): G = 1/2 sum_k Lambda_k |psi_hat_k|^2, F = (1/N) sum_x F(psi(x)).

    eq. `interaction_bulk_energy`: G's sum over k1 + k2 = 0 pairs psi_hat(k) with
    psi_hat(-k) = conj(psi_hat(k)) for a real field, giving |psi_hat_k|^2."""
    ph = fft.forward(psi, direct=direct)
    g = 0.5 * float(np.sum(lam(p) * (ph.real ** 2 + ph.imag ** 2)))
    f = float(np.mean(f0(p, np.asarray(psi, np.float64))))
    return g, f


def energy(p: Problem, psi: np.ndarray, direct: bool = False) -> float:
    """E = G + F (eq. `interaction_bulk_energy`)."""
    g, f = energy_parts(p, psi, direct)
    return g + f


def energy_derivatives(p: Problem, psi: np.ndarray):
    """(dE/dtau, dE/dgamma, [dE/dL_a per array axis]) of E = G + F (eq.
    `interaction_bulk_energy`) with the grid values of psi held fixed.

    F = (1/N) sum_x F(psi) depends on tau and gamma only: dF/dtau = <psi^2/2>_N,
    dF/dgamma = -<psi^3/6>_N, and not on the box.  G = 1/2 sum_k Lambda_k |psi_hat_k|^2
    depends on the box through Lambda_k = xi^2 (1 - |Bk|^2)^2 with (Bk)_a = 2 pi k_a / L_a:
    d|Bk|^2/dL_a = -2 (Bk)_a^2 / L_a, so dLambda_k/dL_a = 4 xi^2 (1 - |Bk|^2) (Bk)_a^2 / L_a.
    """
    psi = np.asarray(psi, np.float64)
    dtau = float(np.mean(psi ** 2 / 2.0))
    dgamma = float(-np.mean(psi ** 3 / 6.0))
    c2 = np.abs(fft.forward(psi)) ** 2
    t = 1.0 - bk_squared(p)
    dl = []
    for a, (m, length) in enumerate(zip(p.shape, p.box)):
        k = fft.wavenumbers(m).astype(np.float64) * (2.0 * np.pi / length)
        sh = [1] * len(p.shape)
        sh[a] = m
        qa = (k * k).reshape(sh)
        dl.append(float(np.sum(0.5 * c2 * 4.0 * p.xi ** 2 * t * qa) / length))
    return dtau, dgamma, dl


def apply_lam(p: Problem, u: np.ndarray, direct: bool = False) -> np.ndarray:
    """F^{-1} Lambda F u: the reciprocal-space diagonal applied to a physical field."""
    return fft.inverse(lam(p) * fft.forward(u, direct=direct), direct=direct)


def gradient(p: Problem, psi: np.ndarray, direct: bool = False) -> np.ndarray:
    """g = P [F^{-1} Lambda F psi + F'(psi)]  (grad G = Lambda Psi_hat and
    grad F = F_N Gamma F_N^{-1} Psi_hat of §2, expressed as a physical field)."""
    psi = np.asarray(psi, np.float64)
    return project(apply_lam(p, psi, direct) + f1(p, psi))


def hessvec(p: Problem, psi: np.ndarray, v: np.ndarray, direct: bool = False) -> np.ndarray:
    """H v = P [F^{-1} Lambda F v + F''(psi) v]  (grad^2 G = Lambda,
    grad^2 F = F_N Gamma' F_N^{-1} of §2; H = D + T of §3.2)."""
    psi = np.asarray(psi, np.float64)
    v = np.asarray(v, np.float64)
    return project(apply_lam(p, v, direct) + f2(p, psi) * v)


def apply_T(p: Problem, psi: np.ndarray, v: np.ndarray) -> np.ndarray:
    """T v = P F''(psi) v P^T: the physical-space diagonal part of H (§3.2)."""
    return project(f2(p, psi) * np.asarray(v, np.float64))


def apply_D(p: Problem, v: np.ndarray) -> np.ndarray:
    """D v = P Lambda P^T v: the reciprocal-space diagonal part of H (§3.2)."""
    return project(apply_lam(p, v))


def energy_from_coefficients(p: Problem, coeffs: dict) -> float:
    """E evaluated literally from eq. `interaction_bulk_energy` for a sparse spectrum.

    `coeffs` maps integer index vectors (per array axis) to Fourier coefficients
    psi_hat(k) of a real field (the set must be closed under k -> -k with
    conjugate coefficients).  The convolution sums run over all tuples from the
    support whose wavevectors add to exactly zero (no aliasing), which agrees with
    the pseudo-spectral value whenever the grid resolves 4x the largest |k|.
    This is an independent check of the physical-space evaluation.
    """
    keys = list(coeffs.keys())
    vals = np.array([coeffs[k] for k in keys], dtype=np.complex128)
    kv = np.array(keys, dtype=np.int64)
    scale = np.array([2.0 * np.pi / b for b in p.box])
    bk2 = np.sum((kv * scale) ** 2, axis=1)
    lam_k = p.xi ** 2 * (1.0 - bk2) ** 2
    index = {k: i for i, k in enumerate(keys)}
    n = len(keys)

    def neg(k):
        return tuple(-a for a in k)

    # two-mode sums: k1 + k2 = 0
    g = 0.0 + 0.0j
    s2 = 0.0 + 0.0j
    for i, k in enumerate(keys):
        j = index.get(neg(k))
        if j is not None:
            g += lam_k[i] * vals[i] * vals[j]
            s2 += vals[i] * vals[j]
    # three-mode sums: k1 + k2 + k3 = 0
    s3 = 0.0 + 0.0j
    for i in range(n):
        for j in range(n):
            k3 = neg(tuple(a + b for a, b in zip(keys[i], keys[j])))
            l = index.get(k3)
            if l is not None:
                s3 += vals[i] * vals[j] * vals[l]
    # four-mode sums: k1 + k2 + k3 + k4 = 0
    s4 = 0.0 + 0.0j
    for i in range(n):
        for j in range(n):
            kij = tuple(a + b for a, b in zip(keys[i], keys[j]))
            for l in range(n):
                k4 = neg(tuple(a + b for a, b in zip(kij, keys[l])))
                m = index.get(k4)
                if m is not None:
                    s4 += vals[i] * vals[j] * vals[l] * vals[m]
    e = 0.5 * g + p.tau / 2.0 * s2 - p.gamma / 6.0 * s3 + s4 / 24.0
    return float(e.real)
