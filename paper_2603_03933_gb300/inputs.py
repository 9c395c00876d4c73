"""Seeded synthetic inputs shared by the CUDA path, the oracle tests and the benchmark.

This module holds only input recipes: seeded Gaussian fields, sums of cosines over
wavevector sets (the Fourier-series initial phases of the paper's Table 2), and the
parameter sets of the workloads.  It contains none of the method's arithmetic (no
energy, gradient, Hessian, FFT or trust-region step), so both the CUDA path and the
oracle can consume the same arrays without sharing any computation.

Array convention: a d-dimensional field is a C-ordered float64 array whose last axis
is x (contiguous), i.e. shape (M, M) = [y][x] in 2D and (M, M, M) = [z][y][x] in 3D.
Box lengths are given per array axis in the same order.  Grid point i along an axis
of length L sits at x = L * i / M (the grid of the paper's §2), so a wavevector with
integer index k along that axis contributes the phase 2*pi*k*i/M.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    """One synthetic problem instance: grid, box, model parameters and initial field."""

    name: str
    shape: tuple
    box: tuple            # per array axis, same order as shape
    xi: float
    tau: float
    gamma: float
    phi0: np.ndarray = field(repr=False)

    @property
    def dim(self) -> int:
        return len(self.shape)

    @property
    def n_points(self) -> int:
        return int(np.prod(self.shape))


def remove_mean(a: np.ndarray) -> np.ndarray:
    """Return a - mean(a) in float64 (the mass constraint of the paper's §2)."""
    a = np.asarray(a, dtype=np.float64)
    return a - a.mean()


def gaussian_field(shape, sigma: float, seed: int) -> np.ndarray:
    """i.i.d. N(0, sigma^2) samples from numpy's PCG64 stream `seed`, mean removed."""
    rng = np.random.default_rng(seed)
    return remove_mean(sigma * rng.standard_normal(tuple(shape)))


def cosine_field(shape, kvecs, amp: float) -> np.ndarray:
    """sum_{k in kvecs} amp * cos(2*pi * sum_a k_a i_a / M_a).

    `kvecs` are integer index vectors given per array axis.  When the set is closed
    under k -> -k (every signed vector listed once), the sum equals
    sum_k amp * exp(2*pi*i k.i/M), i.e. a field whose Fourier coefficient is `amp`
    on every listed vector (the 12 {110} vectors at amp 0.1 peak at 1.2).
    """
    shape = tuple(shape)
    grids = np.meshgrid(*[np.arange(m) for m in shape], indexing="ij")
    out = np.zeros(shape, dtype=np.float64)
    for k in kvecs:
        ph = np.zeros(shape, dtype=np.float64)
        for a, m in enumerate(shape):
            ph += 2.0 * math.pi * k[a] * grids[a] / m
        out += amp * np.cos(ph)
    return out


def exp_field(shape, coeffs: dict) -> np.ndarray:
    """Real part of sum_k c_k exp(2*pi*i k.i/M) for a dict {index vector: coefficient}.

    This is the paper's Fourier-series construction of an initial phase (Table 2)
    with coefficients given explicitly for every signed vector.
    """
    shape = tuple(shape)
    grids = np.meshgrid(*[np.arange(m) for m in shape], indexing="ij")
    out = np.zeros(shape, dtype=np.complex128)
    for k, c in coeffs.items():
        ph = np.zeros(shape, dtype=np.float64)
        for a, m in enumerate(shape):
            ph += 2.0 * math.pi * k[a] * grids[a] / m
        out += c * np.exp(1j * ph)
    return out.real.copy()


def signed_permutations(base) -> list:
    """All distinct vectors obtained by permuting `base` and flipping signs."""
    out = set()
    for p in itertools.permutations(base):
        for s in itertools.product((1, -1), repeat=len(base)):
            out.add(tuple(int(a * b) for a, b in zip(p, s)))
    return sorted(out)


# Wavevector sets (integer index vectors) used by the workloads.
BCC110_INDEX = signed_permutations((2, 2, 0))      # 12 vectors, |k|^2 = 8
CUBIC211_INDEX = signed_permutations((2, 1, 1))    # 24 vectors, |k|^2 = 6
LAM_XI = [(1, 0, 0), (-1, 0, 0)]                   # paper Table 2, LAM
HEX_XI = [(0, 1, -1), (0, -1, 1), (1, 0, -1),      # paper Table 2, HEX
          (-1, 0, 1), (1, -1, 0), (-1, 1, 0)]


def table2_phase(phase: str, M: int) -> Workload:
    """The LAM / HEX initial phases of the paper's Table 2 on an M^3 grid.

    psi_hat = 0.3 on every vector of Xi; B = I/sqrt(2) (LAM) or I/sqrt(6) (HEX),
    so the cubic box side is 2*pi*sqrt(2) or 2*pi*sqrt(6) (A B^T = 2 pi I).
    Model parameters are those of Table 1 Example 1 (LAM) and Example 3 (HEX).
    """
    if phase == "LAM":
        xi_set, side, tau, gamma = LAM_XI, 2 * math.pi * math.sqrt(2), -0.35, 0.7
    elif phase == "HEX":
        xi_set, side, tau, gamma = HEX_XI, 2 * math.pi * math.sqrt(6), -0.28, 0.32
    else:
        raise ValueError(phase)
    # array axes are (z, y, x); the paper's vectors are (k1, k2, k3) along (x, y, z)
    coeffs = {(k[2], k[1], k[0]): 0.3 for k in xi_set}
    phi = exp_field((M, M, M), coeffs)
    return Workload(f"table2-{phase}-{M}^3", (M, M, M), (side,) * 3, 1.0, tau, gamma,
                    remove_mean(phi))


def config_2d_plain(M: int = 64, seed: int = 1) -> Workload:
    """2D LB, square box side 8*pi, xi=1, tau=-0.15, gamma=0.25, phi0 ~ N(0, 0.1^2)."""
    side = 8.0 * math.pi * (M / 64.0)
    return Workload(f"2d-{M}^2-plain", (M, M), (side, side), 1.0, -0.15, 0.25,
                    gaussian_field((M, M), 0.1, seed))


def config_3d_bcc(M: int = 64, seed: int = 2) -> Workload:
    """3D LB, cubic box side 4*pi*sqrt(2) (2x2x2 BCC cells, |q| = 1), xi=1, tau=-0.1,
    gamma=0.2, phi0 = 0.1 * sum cos over the 12 {110} vectors + N(0, 0.01^2), mean removed.
    The box is the same for every M; smaller M only lowers the resolution."""
    side = 4.0 * math.pi * math.sqrt(2.0)
    shape = (M, M, M)
    phi = cosine_field(shape, BCC110_INDEX, 0.1)
    rng = np.random.default_rng(seed)
    phi = phi + 0.01 * rng.standard_normal(shape)
    return Workload(f"3d-{M}^3-bcc", shape, (side,) * 3, 1.0, -0.1, 0.2, remove_mean(phi))


def config_3d_scale(M: int = 128, seed: int | None = None) -> Workload:
    """3D LB at scale: cubic box side 4*pi*sqrt(2), tau=-0.05, gamma=0.3,
    phi0 ~ N(0, 0.05^2), mean removed.  Seed 3 for 128^3, 4 for 256^3 by default."""
    if seed is None:
        seed = 3 if M <= 128 else 4
    side = 4.0 * math.pi * math.sqrt(2.0)
    shape = (M, M, M)
    return Workload(f"3d-{M}^3-scale", shape, (side,) * 3, 1.0, -0.05, 0.3,
                    gaussian_field(shape, 0.05, seed))


def config_3d_cubic211(M: int = 128, seed: int = 6, tau: float = -0.1,
                       gamma: float = 0.2) -> Workload:
    """Differentiation workload: cubic box side 2*pi*sqrt(8),
    phi0 = 0.1 * sum cos over the 24 {211} vectors + N(0, 0.01^2), mean removed.
    (tau, gamma) are not fixed by the workload description; (-0.1, 0.2) is used."""
    side = 2.0 * math.pi * math.sqrt(8.0)
    shape = (M, M, M)
    phi = cosine_field(shape, CUBIC211_INDEX, 0.1)
    rng = np.random.default_rng(seed)
    phi = phi + 0.01 * rng.standard_normal(shape)
    return Workload(f"3d-{M}^3-211", shape, (side,) * 3, 1.0, tau, gamma, remove_mean(phi))


def batched_sweep(n_instances: int = 256, seed: int = 5, sizes=(64, 128, 256, 512)):
    """Phase-diagram sweep: 2D instances of uneven sizes drawn uniformly from `sizes`,
    box side 8*pi*(M/64), tau ~ U[-0.3, 0], gamma ~ U[0, 0.5], phi0 ~ N(0, 0.1^2)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_instances):
        M = int(rng.choice(sizes))
        tau = float(rng.uniform(-0.3, 0.0))
        gamma = float(rng.uniform(0.0, 0.5))
        sub = int(rng.integers(0, 2**31 - 1))
        side = 8.0 * math.pi * (M / 64.0)
        out.append(Workload(f"sweep-{i}-{M}^2", (M, M), (side, side), 1.0, tau, gamma,
                            gaussian_field((M, M), 0.1, sub)))
    return out


def random_problem(shape, seed: int, sigma: float = 0.3, box=None,
                   xi: float = 1.0, tau: float = -0.2, gamma: float = 0.3) -> Workload:
    """A generic seeded instance for parity tests (any grid shape, optional box)."""
    shape = tuple(shape)
    if box is None:
        box = tuple(8.0 * math.pi * (m / 64.0) for m in shape)
    return Workload(f"random-{'x'.join(map(str, shape))}-s{seed}", shape, tuple(box),
                    xi, tau, gamma, gaussian_field(shape, sigma, seed))
