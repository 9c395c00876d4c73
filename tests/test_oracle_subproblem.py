"""Pins for the oracle TR-subproblem solver (paper §3.2, Algorithm 3 and the lambda rule)."""
import math

import numpy as np
import pytest
import scipy.optimize

from oracle import lb
from oracle import subproblem as sp
from paper_2603_03933_gb300 import inputs


def test_secular_newton_one_term_closed_form():
    # c / (a + eta lam)^2 = r^2  ->  lam = (sqrt(c)/r - a) / eta
    c, a, eta, r = np.array([9.0]), np.array([1.5]), 0.1, 0.5
    lam, steps, hist = sp.secular_lambda(c, a, eta, r)
    assert abs(lam - (3.0 / 0.5 - 1.5) / 0.1) < 1e-11
    assert steps >= 1


def test_secular_newton_matches_bracketing_root_and_is_monotone():
    rng = np.random.default_rng(3)
    c = rng.uniform(0, 1, 500) ** 4
    a = 1.0 + 0.1 * rng.uniform(0, 1e2, 500) ** 1.5
    eta, r = 0.1, 0.05
    assert float(np.sum(c / a ** 2)) > r * r       # the multiplier is positive
    lam, steps, hist = sp.secular_lambda(c, a, eta, r)
    f = lambda t: float(np.sum(c / (a + eta * t) ** 2)) - r * r
    ref = scipy.optimize.brentq(f, 0.0, 1e9, xtol=1e-14, rtol=1e-15)
    assert abs(lam - ref) <= 1e-12 * ref
    # Newton from 0 on a convex decreasing function increases monotonically
    assert all(b >= a_ for a_, b in zip(hist, hist[1:]))


def test_secular_zero_multiplier_inside_ball():
    c, a = np.array([0.01, 0.02]), np.array([1.0, 2.0])
    lam, steps, _ = sp.secular_lambda(c, a, 0.1, 1.0)
    assert lam == 0.0 and steps == 0


def test_more_sorensen_interior_is_newton_point():
    rng = np.random.default_rng(4)
    q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    h = q @ np.diag([1, 2, 3, 4, 5, 6.0]) @ q.T
    g = rng.standard_normal(6) * 0.1
    d, lam, hard = sp.more_sorensen(h, g, 10.0)
    assert lam == 0.0 and not hard
    assert np.allclose(d, np.linalg.solve(h, -g), atol=1e-13)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_more_sorensen_beats_brute_force_in_two_dims(seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((2, 2))
    h = a + a.T
    g = rng.standard_normal(2)
    r = 0.7
    d, lam, _ = sp.more_sorensen(h, g, r)
    f = lambda x: g @ x + 0.5 * x @ h @ x
    ang = np.linspace(0, 2 * np.pi, 200001)
    best = min(f(r * np.array([math.cos(t), math.sin(t)])) for t in ang[::50])
    pts = r * np.stack([np.cos(ang), np.sin(ang)], 1)
    vals = pts @ g + 0.5 * np.einsum("ij,jk,ik->i", pts, h, pts)
    best = min(best, vals.min())
    # interior stationary point, if it is a minimiser inside the ball
    if np.all(np.linalg.eigvalsh(h) > 0):
        xi = np.linalg.solve(h, -g)
        if np.linalg.norm(xi) <= r:
            best = min(best, f(xi))
    assert f(d) <= best + 1e-9
    assert np.linalg.norm(d) <= r * (1 + 1e-12)


def test_more_sorensen_hard_case():
    # H = diag(-1, 2), g = (0, 1): g has no component on the -1 eigenvector
    h = np.diag([-1.0, 2.0])
    g = np.array([0.0, 1.0])
    d, lam, hard = sp.more_sorensen(h, g, 2.0)
    assert hard and abs(lam - 1.0) < 1e-14
    assert abs(d[1] + 1.0 / 3.0) < 1e-14 and abs(abs(d[0]) - math.sqrt(4 - 1 / 9)) < 1e-13


def _nonconvex_problem():
    # box side 2 pi: |Bk| = |k|, so Lambda vanishes on the |k| = 1 modes and tau < 0
    # makes H indefinite near psi = 0
    w = inputs.random_problem((16, 16), 5, sigma=0.05, tau=-0.2, gamma=0.3,
                              box=(2 * math.pi, 2 * math.pi))
    return lb.Problem.from_workload(w), w.phi0


def _convex_problem():
    w = inputs.random_problem((8, 8), 3, sigma=0.8)
    return lb.Problem.from_workload(w), w.phi0


@pytest.mark.parametrize("which,r", [("convex", 0.05), ("convex", 1.0),
                                     ("nonconvex", 0.02), ("nonconvex", 0.05)])
def test_algorithm3_reaches_global_minimiser(which, r):
    p, psi = _convex_problem() if which == "convex" else _nonconvex_problem()
    g = lb.gradient(p, psi)
    hc, u = sp.dense_hessian(p, psi)
    gc = sp.to_coords(u, g)
    d_ms, lam_ms, _ = sp.more_sorensen(hc, gc, r)
    f_ms = gc @ d_ms + 0.5 * d_ms @ hc @ d_ms
    out = sp.imex_subproblem(p, psi, g, r, eta=0.1, eps_sub=1e-10, max_iter=60000, record=True)
    assert out["converged"]
    f_imex = sp.model_value(p, psi, g, out["d"])
    assert abs(f_imex - f_ms) <= 1e-9 * abs(f_ms)
    assert abs(out["lambda"] - lam_ms) <= 1e-6 * max(1.0, lam_ms)
    dc = sp.to_coords(u, out["d"])
    assert np.linalg.norm(dc - d_ms) <= 1e-6 * r
    # Corollary of §3.2: lambda_k >= 0, ||d_k|| <= r, lambda_k (||d_k|| - r) = 0
    h = out["history"]
    for lam_k, dn in zip(h["lambda"], h["dnorm"]):
        assert lam_k >= 0.0
        assert dn <= r * (1 + 1e-12)
        assert abs(lam_k * (dn - r)) <= 1e-10 * max(1.0, lam_k) * r
    # descent lemma of §3.2.1: eta = 0.1 <= 1/(||T|| + 2a) here, so f(d_k) decreases
    tnorm = float(np.max(np.abs(lb.f2(p, psi))))
    assert 0.1 < 1.0 / tnorm
    f = h["f"]
    assert all(b <= a_ + 1e-12 * abs(a_) for a_, b in zip(f, f[1:]))


def test_algorithm3_sign_invariant_on_lowest_eigenvector():
    # proof of the global-optimality theorem: d_k^(1) g^(1) <= 0 for all k
    p, psi = _nonconvex_problem()
    g = lb.gradient(p, psi)
    hc, u = sp.dense_hessian(p, psi)
    s, q = np.linalg.eigh(hc)
    assert s[0] < 0
    xi = sp.from_coords(u, q[:, 0], p.shape)
    g1 = lb.inner(xi, g)
    assert abs(g1) > 1e-8
    r = 0.3
    lam_k = lb.lam(p)
    a = 1.0 + 0.1 * lam_k
    d = -r * g / lb.norm(g)
    zero = np.zeros(p.shape, bool)
    zero[0, 0] = True
    from oracle import fft
    for _ in range(300):
        assert lb.inner(xi, d) * g1 <= 1e-15
        b = d - 0.1 * (g + lb.apply_T(p, psi, d))
        bh = fft.forward(b)
        c = np.abs(bh) ** 2
        lam, _, _ = sp.secular_lambda(c[~zero], a[~zero], 0.1, r)
        dh = bh / (a + 0.1 * lam)
        dh[zero] = 0
        d = fft.inverse(dh)


def test_random_ball_point_is_feasible_and_zero_mean():
    rng = np.random.default_rng(0)
    for _ in range(5):
        v = sp.random_ball_point(rng, (8, 8), 0.4)
        assert lb.norm(v) <= 0.4 + 1e-15
        assert abs(np.mean(v)) < 1e-16
