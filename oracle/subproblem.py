"""Oracle for the trust-region subproblem (paper §3.2): Algorithm 3 and the lambda rule.

Test infrastructure, not product code (see oracle/__init__.py).  FP64 throughout.

  * secular_lambda: the Lagrange-multiplier rule eq. `lambda_update_rule`:
    lambda = 0 if phi_k(0) <= r^2, else the root of phi_k(lambda) = r^2 reached by
    Newton's method from lambda_0 = 0, where
        phi_k(lambda) = sum_i b_i^2 / (1 + eta (D_ii + lambda))^2
    (the displayed formula before eq. `lambda_update_rule`).
  * imex_subproblem: Algorithm 3 (adaptive implicit-explicit iteration), step by
    step: b_k = d_k - eta (g + T d_k); lambda_{k+1} by the rule above;
    d_{k+1} = (I + eta (D + lambda_{k+1} I))^{-1} b_k (eq. `imex-scheme`,
    eq. `semi_implicit_2linear_system`); stop when ||g + (H + lambda I) d|| < eps_sub.
  * more_sorensen: the exact global minimiser of min_{||d|| <= r} g^T d + d^T H d / 2
    for a dense symmetric H (characterised by the optimality conditions of
    eq. `tr_subproblem_optimal_condition`), including the hard case; used as the
    reference that Algorithm 3 must reach (the global-optimality theorem of §3.2.1).

Readings: the paper gives no stopping rule for the Newton loop (it loops while
phi > r^2, which in exact arithmetic never ends because Newton from the left of the
root of a convex decreasing function approaches it monotonically from below).  Here
Newton stops when phi(lambda) - r^2 <= rtol * r^2, when the step is below
1e-15 * (1 + lambda), or after 100 steps.
"""
from __future__ import annotations

import numpy as np

from . import fft, lb


def secular_phi(c: np.ndarray, a: np.ndarray, eta: float, lam: float):
    """phi(lambda) and phi'(lambda) for phi = sum_i c_i / (a_i + eta*lambda)^2,
    with c_i = |b_i|^2 and a_i = 1 + eta*D_ii."""
    den = a + eta * lam
    t = c / (den * den)
    phi = float(np.sum(t))
    dphi = float(np.sum(-2.0 * eta * t / den))
    return phi, dphi


def secular_lambda(c: np.ndarray, a: np.ndarray, eta: float, r: float,
                   rtol: float = 1e-14, max_newton: int = 100, lam0: float = 0.0):
    """The rule of eq. `lambda_update_rule` by Newton from lam0 (0 in the paper).

    Returns (lambda, newton_steps, history) where history lists the Newton iterates.
    """
    r2 = r * r
    phi0, _ = secular_phi(c, a, eta, 0.0)
    if phi0 <= r2:
        return 0.0, 0, [0.0]
    lam = max(float(lam0), 0.0)
    phi, dphi = secular_phi(c, a, eta, lam)
    hist = [lam]
    steps = 0
    while steps < max_newton:
        if abs(phi - r2) <= rtol * r2:
            break
        lam_new = max(lam - (phi - r2) / dphi, 0.0)
        steps += 1
        hist.append(lam_new)
        if abs(lam_new - lam) <= 1e-15 * (1.0 + abs(lam_new)):
            lam = lam_new
            break
        lam = lam_new
        phi, dphi = secular_phi(c, a, eta, lam)
    return lam, steps, hist


def model_value(p: lb.Problem, psi, g, d) -> float:
    """f(d) = g^T d + d^T H d / 2 (eq. `tr_subproblem`) in the <.,.>_N metric."""
    return lb.inner(g, d) + 0.5 * lb.inner(d, lb.hessvec(p, psi, d))


def kkt_residual(p: lb.Problem, psi, g, d, lam: float) -> float:
    """||g + (H + lambda I) d|| (the stopping test of Algorithm 3)."""
    return lb.norm(g + lb.hessvec(p, psi, d) + lam * d)


def imex_subproblem(p: lb.Problem, psi: np.ndarray, g: np.ndarray, r: float,
                    eta: float = 0.1, eps_sub: float = 1e-13, max_iter: int = 20000,
                    d0: np.ndarray | None = None, record: bool = False, rel_tol: float = 0.0):
    """Algorithm 3 (adaptive implicit-explicit iteration) of the paper, in FP64.

    psi: the current iterate (physical field); g: the projected gradient there;
    r: trust-region radius; d0: initial point (default -r g / ||g||).
    The stop test is the paper's ||g + (H + lambda I) d|| < eps_sub; with rel_tol > 0 the
    iteration also stops once that residual is below rel_tol ||g|| (the relative form of
    the test, which the paper's absolute eps_sub leaves open; default off).
    Returns a dict with d, lambda, iterations, final residual and (if record)
    per-iteration histories of lambda_k, ||d_k||, f(d_k) and the residual.
    """
    psi = np.asarray(psi, np.float64)
    g = lb.project(np.asarray(g, np.float64))
    lam_k = lb.lam(p)
    a = 1.0 + eta * lam_k                       # diagonal of I + eta D in reciprocal space
    zero = np.zeros(p.shape, dtype=bool)
    zero[(0,) * len(p.shape)] = True            # the k = 0 mode removed by P (§3)
    if d0 is None:
        d = -r * g / lb.norm(g)
    else:
        d = lb.project(np.asarray(d0, np.float64))
    hist = {"lambda": [], "dnorm": [], "f": [], "res": [], "newton": []}
    tol = max(eps_sub, rel_tol * lb.norm(g))
    lam = 0.0
    res = np.inf
    it = 0
    for it in range(1, max_iter + 1):
        gbar = g + lb.apply_T(p, psi, d)        # g_bar_k = g + T d_k
        b = d - eta * gbar                      # b_k = d_k - eta g_bar_k
        bh = fft.forward(b)
        bh[zero] = 0.0
        c = (bh.real ** 2 + bh.imag ** 2)       # |[b_k]_i|^2 over the N-1 modes
        c[zero] = 0.0
        lam, nsteps, _ = secular_lambda(c[~zero], a[~zero], eta, r)
        dh = bh / (a + eta * lam)
        dh[zero] = 0.0
        d = fft.inverse(dh)
        res = kkt_residual(p, psi, g, d, lam)
        if record:
            hist["lambda"].append(lam)
            hist["dnorm"].append(lb.norm(d))
            hist["f"].append(model_value(p, psi, g, d))
            hist["res"].append(res)
            hist["newton"].append(nsteps)
        if res < tol:
            break
    out = {"d": d, "lambda": lam, "iterations": it, "residual": res,
           "converged": bool(res < tol)}
    if record:
        out["history"] = hist
    return out


# ---------------------------------------------------------------------------------
# Dense tools for small grids
# ---------------------------------------------------------------------------------

def zero_mean_basis(n: int) -> np.ndarray:
    """U (n x (n-1)) with orthonormal columns spanning {u : sum u = 0}.

    A field v = sqrt(n) U c has <v, v>_N = c^T c, so coordinates c carry the
    paper's Euclidean metric on the N-1 free Fourier coefficients."""
    ones = np.ones((n, 1)) / np.sqrt(n)
    q, _ = np.linalg.qr(np.hstack([ones, np.eye(n)[:, : n - 1]]))
    return q[:, 1:]


def dense_operator(p: lb.Problem, apply) -> np.ndarray:
    """Matrix A of a linear map on physical fields: column y = apply(e_y)."""
    n = p.n
    a = np.zeros((n, n))
    for y in range(n):
        e = np.zeros(n)
        e[y] = 1.0
        a[:, y] = apply(e.reshape(p.shape)).ravel()
    return a


def dense_hessian(p: lb.Problem, psi: np.ndarray):
    """(Hc, U): the Hessian in orthonormal zero-mean coordinates, Hc = U^T A U."""
    a = dense_operator(p, lambda v: lb.hessvec(p, psi, v))
    u = zero_mean_basis(p.n)
    hc = u.T @ a @ u
    return 0.5 * (hc + hc.T), u


def to_coords(u_basis: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Coordinates c of a zero-mean field v = sqrt(n) U c."""
    return u_basis.T @ np.asarray(v, np.float64).ravel() / np.sqrt(u_basis.shape[0])


def from_coords(u_basis: np.ndarray, c: np.ndarray, shape) -> np.ndarray:
    return (np.sqrt(u_basis.shape[0]) * (u_basis @ c)).reshape(shape)


def more_sorensen(h: np.ndarray, g: np.ndarray, r: float, hard_tol: float = 1e-12):
    """Exact global minimiser of g^T d + d^T h d / 2 over ||d|| <= r (dense, FP64).

    Uses h = Q diag(s) Q^T.  The optimality conditions of eq.
    `tr_subproblem_optimal_condition` (g + (h + lam I) d = 0, ||d|| <= r,
    lam (||d|| - r) = 0, h + lam I PSD) determine lam >= max(0, -s_1) with
    ||d(lam)|| = r unless the interior Newton point is feasible.  The root of
    sum_i gq_i^2 / (s_i + lam)^2 = r^2 is found by bisection to machine precision.
    Hard case (gq orthogonal to the s_1 eigenspace and ||d(-s_1)|| < r): lam = -s_1
    and d = d(-s_1) + t q_1 with ||d|| = r.
    Returns (d, lam, hard_case_flag).
    """
    s, q = np.linalg.eigh(h)
    gq = q.T @ g
    s1 = s[0]
    if s1 > 0:
        d = -q @ (gq / s)
        if np.linalg.norm(d) <= r:
            return d, 0.0, False

    def dnorm2(lam):
        return float(np.sum(gq ** 2 / (s + lam) ** 2))

    lo = max(0.0, -s1)
    # components in the (numerical) s_1 eigenspace
    deg = np.abs(s - s1) <= 1e-10 * max(1.0, abs(s1))
    if np.all(np.abs(gq[deg]) <= hard_tol * max(1.0, np.linalg.norm(g))) and s1 <= 0:
        keep = ~deg
        d_part = -q[:, keep] @ (gq[keep] / (s[keep] - s1))
        nrm = np.linalg.norm(d_part)
        if nrm < r:
            t = np.sqrt(r * r - nrm * nrm)
            return d_part + t * q[:, 0], -s1, True
    hi = lo + np.linalg.norm(g) / r + 1.0
    while dnorm2(hi) > r * r:
        hi = 2.0 * hi + 1.0
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if dnorm2(mid) > r * r:
            lo = mid
        else:
            hi = mid
    lam = 0.5 * (lo + hi)
    d = -q @ (gq / (s + lam))
    return d, lam, False


def random_ball_point(rng: np.random.Generator, shape, r: float) -> np.ndarray:
    """A zero-mean field drawn from a continuous distribution supported on the ball
    ||s|| <= r (the randomised initial point of the hard-case remark of §3.2):
    a Gaussian direction, projected and normalised, times r * U^(1/(N-1))."""
    v = lb.project(rng.standard_normal(tuple(shape)))
    n = int(np.prod(shape)) - 1
    rad = r * rng.uniform() ** (1.0 / n)
    return rad * v / lb.norm(v)
