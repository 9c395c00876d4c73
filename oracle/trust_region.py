"""Oracle for the IMEX-TR outer loop: Algorithm 1 (IMEX-TR) and Algorithm 2 (CONTRACT).

Test infrastructure, not product code (see oracle/__init__.py).  FP64 throughout.

Readings of the paper taken here (all listed in the design notes):
  * rho_j = (E(v_j) - E(v_j + s_j)) / ||s_j||^3 (Algorithm 1) is evaluated through
    the exact expansion of the quartic energy,
        E(v + s) - E(v) = <g, s> + G(s) + (1/N) sum_x s^2 (F''/2 + F''' s/6 + s^2/24),
    with G(s) = 1/2 sum_k Lambda_k |s_hat_k|^2, which avoids the cancellation of a
    difference of two O(1e-2) energies; `energy_drop_direct` keeps the literal form.
  * "||s_j|| = nu_j" is read as | ||s_j|| - nu_j | <= 1e-12 nu_j.
  * "lambda_j <= mu_j ||s_j||" is evaluated as lambda_j / ||s_j|| <= mu_j, the form of the
    mu update, so that after that update the test holds as the algorithm intends.
  * mu: the update Algorithm 1 makes when the previous ratio failed acts on the running mu;
    the CONTRACT branch leaves mu unchanged.
  * CONTRACT's linear systems (H + lambda~ I) s = -g are solved by preconditioned CG
    with preconditioner (Lambda + lambda~ + c)^{-1}, c = max(0, mean F''(psi)); the
    "find lambda~ in (lambda_j, lambda^)" step is a bisection on lambda~ (the ratio
    lambda~/||s(lambda~)|| increases with lambda~).
  * The last branch of CONTRACT returns gamma_C ||s_j|| (the paper prints gamma_C ||s||;
    the TRACE procedure it follows shrinks relative to the rejected step s_j).
  * Stop: ||g_j||_inf < eps with the max taken over physical grid values (this
    bounds the paper's max over Fourier coefficients from above).  With
    second_order=True the point is accepted only if lambda_min(H) >= -tol2; otherwise
    the next subproblem starts from a random point of the ball (the hard-case remark
    of §3.2), which is how a saddle with g = 0 is left.
"""
from __future__ import annotations

import numpy as np

from . import eig, fft, lb
from .subproblem import imex_subproblem, random_ball_point

PAPER_PARAMS = dict(gamma_c=0.5, gamma_e=2.0, gamma_lam=1.5, theta=1e-4, mu_lo=1.0,
                    mu_hi=1e5, mu0=1.0, r0=1.0, nu0=5.0, eps=1e-10, eta=0.1, eps_sub=1e-13)
"""Algorithm parameters printed in §4 (first paragraph)."""


def quad_energy(p: lb.Problem, s: np.ndarray) -> float:
    """G(s) = 1/2 sum_k Lambda_k |s_hat_k|^2."""
    sh = fft.forward(s)
    return 0.5 * float(np.sum(lb.lam(p) * (sh.real ** 2 + sh.imag ** 2)))


def energy_drop(p: lb.Problem, v: np.ndarray, g: np.ndarray, s: np.ndarray) -> float:
    """E(v) - E(v + s) by the exact quartic expansion (no cancellation)."""
    rem = s * s * (lb.f2(p, v) / 2.0 + lb.f3(p, v) * s / 6.0 + s * s / 24.0)
    return -(lb.inner(g, s) + quad_energy(p, s) + float(np.mean(rem)))


def energy_drop_direct(p: lb.Problem, v: np.ndarray, s: np.ndarray) -> float:
    """E(v) - E(v + s) as the literal difference of two energies."""
    return lb.energy(p, v) - lb.energy(p, v + s)


def pcg_shifted(p: lb.Problem, psi: np.ndarray, g: np.ndarray, shift: float,
                rtol: float = 1e-12, max_iter: int = 5000):
    """Solve (H + shift I) s = -g on zero-mean fields by preconditioned CG.

    Returns (s, iterations, final relative residual)."""
    psi = np.asarray(psi, np.float64)
    c = max(0.0, float(np.mean(lb.f2(p, psi))))
    pre = 1.0 / (lb.lam(p) + shift + c)

    def aop(v):
        return lb.hessvec(p, psi, v) + shift * v

    def prec(v):
        return lb.project(fft.inverse(pre * fft.forward(v)))

    b = -lb.project(g)
    bn = lb.norm(b)
    x = np.zeros_like(b)
    if bn == 0.0:
        return x, 0, 0.0
    r = b.copy()
    z = prec(r)
    d = z.copy()
    rz = lb.inner(r, z)
    it = 0
    for it in range(1, max_iter + 1):
        ad = aop(d)
        dad = lb.inner(d, ad)
        if dad <= 0.0:
            break
        al = rz / dad
        x = x + al * d
        r = r - al * ad
        if lb.norm(r) <= rtol * bn:
            break
        z = prec(r)
        rz_new = lb.inner(r, z)
        d = z + (rz_new / rz) * d
        rz = rz_new
    return x, it, lb.norm(r) / bn


def contract(p: lb.Problem, v, g, r, mu, s_j, lam_j, prm, log=None):
    """Algorithm 2 (CONTRACT): returns the new radius r_{j+1}."""
    sn = lb.norm(s_j)
    gn = lb.norm(g)
    if lam_j < prm["mu_lo"] * sn:
        lam_hat = lam_j + np.sqrt(prm["mu_lo"] * gn)
        s, _, _ = pcg_shifted(p, v, g, lam_hat)
        if lam_hat / lb.norm(s) <= prm["mu_hi"]:
            return lb.norm(s)
        lo, hi = lam_j, lam_hat
        s_mid = s
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            s_mid, _, _ = pcg_shifted(p, v, g, mid)
            ratio = mid / lb.norm(s_mid)
            if ratio < prm["mu_lo"]:
                lo = mid
            elif ratio > prm["mu_hi"]:
                hi = mid
            else:
                break
        return lb.norm(s_mid)
    lam_t = prm["gamma_lam"] * lam_j
    s, _, _ = pcg_shifted(p, v, g, lam_t)
    if lb.norm(s) >= prm["gamma_c"] * sn:
        return lb.norm(s)
    return prm["gamma_c"] * sn


def step_kind(rho: float, lam_j: float, sn: float, mu: float, nu: float, prm: dict) -> str:
    """The three branches of Algorithm 1 for the step s_j (||s_j|| = sn, multiplier lam_j):
    "accept" when rho_j >= theta and (lam_j <= mu_j ||s_j|| or ||s_j|| = nu_j); "contract"
    when rho_j < theta; "shrink" otherwise.  lam_j <= mu_j ||s_j|| is evaluated as
    lam_j / ||s_j|| <= mu_j, the form in which mu_j = max(mu, lam_j / ||s_j||) is updated after
    a failed ratio, so that the update's guarantee (the test then holds) survives rounding:
    the product form can miss by one ulp, and the shrink branch would then set
    r = lam_j / mu_j = ||s_j||, the same subproblem again."""
    if rho >= prm["theta"] and (lam_j / sn <= mu or abs(sn - nu) <= 1e-12 * nu):
        return "accept"
    if rho < prm["theta"]:
        return "contract"
    return "shrink"


def imex_tr(p: lb.Problem, v0: np.ndarray, params: dict | None = None, max_outer: int = 500,
            eps: float | None = None, second_order: bool = True, tol2: float = 1e-8,
            max_inner: int = 20000, eps_sub: float | None = None, seed: int = 0,
            log: list | None = None, sub_rel_tol: float = 0.0):
    """Algorithm 1 of the paper with the readings listed in the module docstring.

    Returns a dict with the final field, energy, ||g||_inf, lambda_min (if checked),
    outer/inner iteration counts and a per-iteration log (if `log` is a list).
    """
    prm = dict(PAPER_PARAMS)
    if params:
        prm.update(params)
    if eps is not None:
        prm["eps"] = eps
    if eps_sub is not None:
        prm["eps_sub"] = eps_sub
    rng = np.random.default_rng(seed)
    v = lb.project(np.asarray(v0, np.float64))
    r, nu, mu = prm["r0"], prm["nu0"], prm["mu0"]
    rho_prev = None
    inner_total = 0
    lam_min = None
    d0 = None
    status = "max_outer"
    j = 0
    for j in range(max_outer):
        g = lb.gradient(p, v)
        gmax = float(np.max(np.abs(g)))
        if gmax < prm["eps"] and d0 is None:
            if not second_order:
                status = "converged"
                break
            if p.n <= 1024:
                lam_min = float(eig.dense_eigs(p, v, count=1)[0][0])
            else:
                lam_min = eig.lanczos_lambda_min(p, v)["theta"]
            if lam_min >= -tol2:
                status = "converged"
                break
            d0 = random_ball_point(rng, p.shape, r)
        sub = imex_subproblem(p, v, g, r, prm["eta"], prm["eps_sub"], max_inner, d0=d0, rel_tol=sub_rel_tol)
        d0 = None
        inner_total += sub["iterations"]
        s, lam_j = sub["d"], sub["lambda"]
        sn = lb.norm(s)
        if j > 0 and rho_prev is not None and rho_prev < prm["theta"]:
            mu = max(mu, lam_j / sn)
        rho = energy_drop(p, v, g, s) / sn ** 3
        step = step_kind(rho, lam_j, sn, mu, nu, prm)
        if step == "accept":
            v = v + s
            nu_new = max(nu, prm["gamma_e"] * sn)
            r = min(nu_new, max(r, prm["gamma_e"] * sn))
            mu = max(mu, lam_j / sn)
            nu = nu_new
        elif step == "contract":
            r = contract(p, v, g, r, mu, s, lam_j, prm)
        else:
            r = min(nu, lam_j / mu)
        rho_prev = rho
        if log is not None:
            log.append({"j": j, "E": lb.energy(p, v), "gmax": gmax, "r": r, "nu": nu, "mu": mu,
                        "lambda": lam_j, "snorm": sn, "rho": rho, "inner": sub["iterations"],
                        "step": step})
    g = lb.gradient(p, v)
    return {"v": v, "E": lb.energy(p, v), "gmax": float(np.max(np.abs(g))),
            "lambda_min": lam_min, "outer": j, "inner": inner_total, "status": status}
