"""Pins for the oracle outer loop (paper §3.1, Algorithms 1 and 2)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import eig, lb
from oracle import subproblem as sp
from oracle import trust_region as tr
from paper_2603_03933_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def test_parameters_are_the_papers():
    with open(GOLDEN) as f:
        prm = json.load(f)["algorithm_parameters"]
    for k, v in tr.PAPER_PARAMS.items():
        assert prm[k] == v, k


def test_pcg_matches_dense_solve():
    w = inputs.random_problem((8, 8), 13, sigma=0.5)
    p = lb.Problem.from_workload(w)
    g = lb.gradient(p, w.phi0)
    hc, u = sp.dense_hessian(p, w.phi0)
    shift = 0.7 + max(0.0, -np.linalg.eigvalsh(hc)[0])
    s, it, rel = tr.pcg_shifted(p, w.phi0, g, shift)
    ref = np.linalg.solve(hc + shift * np.eye(hc.shape[0]), -sp.to_coords(u, g))
    assert np.allclose(sp.to_coords(u, s), ref, atol=1e-10 * np.linalg.norm(ref))


def test_exact_energy_drop_matches_direct_difference():
    w = inputs.random_problem((16, 16), 17, sigma=0.3)
    p = lb.Problem.from_workload(w)
    g = lb.gradient(p, w.phi0)
    for scale in (1e-1, 1.0):
        s = scale * inputs.gaussian_field(w.shape, 1.0, 18)
        a = tr.energy_drop(p, w.phi0, g, s)
        b = tr.energy_drop_direct(p, w.phi0, s)
        assert abs(a - b) <= 1e-12 * max(1.0, abs(b))


def test_imex_tr_reaches_second_order_stationary_point():
    # box side 2 pi on 16^2: |Bk| = |k|, tau < 0, started next to the saddle psi = 0
    w = inputs.random_problem((16, 16), 5, sigma=0.05, tau=-0.2, gamma=0.3,
                              box=(math.pi * 2, math.pi * 2))
    p = lb.Problem.from_workload(w)
    log = []
    out = tr.imex_tr(p, w.phi0, eps=1e-8, max_outer=60, max_inner=1000, log=log)
    assert out["status"] == "converged"
    assert out["gmax"] < 1e-8
    s, _ = eig.dense_eigs(p, out["v"], count=1)
    assert s[0] >= -1e-8                       # SP-II (paper §1 definition)
    # accepted steps never raise the energy
    e0 = lb.energy(p, w.phi0)
    es = [e0] + [l["E"] for l in log]
    assert all(b <= a + 1e-14 for a, b in zip(es, es[1:]))
    assert out["E"] < e0


# ---------------------------------------------------------------------------------
# Branch logic of Algorithm 2 (CONTRACT) and of the radius / multiplier updates of
# Algorithm 1, each pinned on a dense 8x8 problem where the linear systems of Algorithm 2
# are solved exactly by numpy.linalg.solve on the assembled Hessian.
# ---------------------------------------------------------------------------------

def _dense_case(seed=21, tau=0.4):
    # tau > 0 with a moderate field keeps H positive definite, so every shift >= 0 is valid
    w = inputs.random_problem((8, 8), seed, sigma=0.3, tau=tau, gamma=0.3, box=(2 * math.pi, 2 * math.pi))
    p = lb.Problem.from_workload(w)
    hc, u = sp.dense_hessian(p, w.phi0)
    assert np.linalg.eigvalsh(hc)[0] > 0.05
    return w, p, hc, u


def _snorm_dense(hc, u, g, shift):
    """||s|| of the solution of (H + shift I) s = -g (coordinates carry the <.,.>_N metric)."""
    c = np.linalg.solve(hc + shift * np.eye(hc.shape[0]), -sp.to_coords(u, g))
    return float(np.linalg.norm(c))


def _unit(field):
    return field / lb.norm(field)


def test_contract_first_branch_returns_norm_at_lambda_hat():
    # Algorithm 2, lambda_j < mu_lo ||s_j||: lambda^ = lambda_j + (mu_lo ||g||)^{1/2} and, when
    # lambda^ / ||s(lambda^)|| <= mu_hi, the new radius is ||s(lambda^)||
    w, p, hc, u = _dense_case()
    g = lb.gradient(p, w.phi0)
    prm = dict(tr.PAPER_PARAMS)
    lam_j, s_j = 0.1, 1.0 * _unit(g)               # 0.1 < 1 * 1
    lam_hat = lam_j + math.sqrt(prm["mu_lo"] * lb.norm(g))
    want = _snorm_dense(hc, u, g, lam_hat)
    assert lam_hat / want <= prm["mu_hi"]
    got = tr.contract(p, w.phi0, g, 1.0, 1.0, s_j, lam_j, prm)
    assert abs(got - want) <= 1e-9 * want
    # neither the second branch's candidates nor the shift without the square root give it
    for other in (_snorm_dense(hc, u, g, prm["gamma_lam"] * lam_j), prm["gamma_c"] * 1.0,
                  _snorm_dense(hc, u, g, lam_j + prm["mu_lo"] * lb.norm(g))):
        assert abs(other - want) > 1e-3 * want


def test_contract_first_branch_bisects_into_mu_window():
    # Algorithm 2, lambda^ / ||s(lambda^)|| > mu_hi: the radius is ||s(lambda~)|| for some
    # lambda~ in (lambda_j, lambda^) with mu_lo <= lambda~ / ||s(lambda~)|| <= mu_hi.  Any such
    # lambda~ is what the paper asks for; it is recovered here from the returned radius
    # (||s(lambda)|| decreases strictly in lambda) and the window checked.
    w, p, hc, u = _dense_case()
    g = lb.gradient(p, w.phi0)
    lam_j, s_j = 0.05, 1.0 * _unit(g)
    prm = dict(tr.PAPER_PARAMS)
    lam_hat = lam_j + math.sqrt(prm["mu_lo"] * lb.norm(g))
    ratio_hat = lam_hat / _snorm_dense(hc, u, g, lam_hat)
    ratio_lo = lam_j / _snorm_dense(hc, u, g, lam_j)
    prm["mu_lo"] = 1.0
    prm["mu_hi"] = 0.5 * ratio_hat                 # forces the search
    assert ratio_lo < prm["mu_lo"] < prm["mu_hi"] < ratio_hat
    got = tr.contract(p, w.phi0, g, 1.0, 1.0, s_j, lam_j, prm)
    from scipy.optimize import brentq
    lam_t = brentq(lambda x: _snorm_dense(hc, u, g, x) - got, lam_j, lam_hat, xtol=1e-14, rtol=1e-14)
    assert lam_j < lam_t < lam_hat
    ratio = lam_t / got
    assert prm["mu_lo"] * (1 - 1e-8) <= ratio <= prm["mu_hi"] * (1 + 1e-8)
    # the radius at lambda^ itself lies outside the window
    assert abs(got - _snorm_dense(hc, u, g, lam_hat)) > 1e-3 * got


def _g_for_step(p, phi, s_target, shift):
    # the gradient for which (H + shift I) s = -g has the solution s_target
    return -(lb.hessvec(p, phi, s_target) + shift * s_target)


def test_contract_second_branch_keeps_solution_norm():
    # Algorithm 2, lambda_j >= mu_lo ||s_j||: lambda~ = gamma_lam lambda_j; if
    # ||s(lambda~)|| >= gamma_C ||s_j|| the new radius is ||s(lambda~)||
    w, p, hc, u = _dense_case()
    prm = dict(tr.PAPER_PARAMS)
    lam_j, s_j = 2.0, 1.0 * _unit(inputs.gaussian_field((8, 8), 1.0, 31))
    s_t = 0.8 * _unit(inputs.gaussian_field((8, 8), 1.0, 32))      # 0.8 >= 0.5 * 1
    g = _g_for_step(p, w.phi0, s_t, prm["gamma_lam"] * lam_j)
    got = tr.contract(p, w.phi0, g, 1.0, 1.0, s_j, lam_j, prm)
    assert abs(got - 0.8) <= 1e-9
    assert abs(_snorm_dense(hc, u, g, prm["gamma_lam"] * lam_j) - 0.8) <= 1e-10


def test_contract_second_branch_floors_at_gamma_c_times_rejected_step():
    # ||s(lambda~)|| < gamma_C ||s_j||: the radius is gamma_C times the norm of the REJECTED
    # step s_j (the paper prints gamma_C ||s||, TRACE shrinks relative to s_j: reading of the
    # last branch), here 0.5 * 1.3, not 0.5 * 0.3
    w, p, hc, u = _dense_case()
    prm = dict(tr.PAPER_PARAMS)
    lam_j, s_j = 2.0, 1.3 * _unit(inputs.gaussian_field((8, 8), 1.0, 33))
    s_t = 0.3 * _unit(inputs.gaussian_field((8, 8), 1.0, 34))
    g = _g_for_step(p, w.phi0, s_t, prm["gamma_lam"] * lam_j)
    got = tr.contract(p, w.phi0, g, 1.0, 1.0, s_j, lam_j, prm)
    assert abs(got - 0.65) <= 1e-12


def _tr_case(params, max_outer):
    w = inputs.random_problem((8, 8), 11, sigma=0.3, tau=-0.2, gamma=0.3, box=(2 * math.pi, 2 * math.pi))
    p = lb.Problem.from_workload(w)
    log = []
    tr.imex_tr(p, w.phi0, params=params, max_outer=max_outer, eps=1e-12, second_order=False,
               max_inner=20000, eps_sub=1e-12, log=log)
    return w, p, log


def _check_first_step_is_global_minimiser(w, p, entry, r0):
    # the s_0 the branch logic acted on: the global minimiser of the subproblem (dense
    # More-Sorensen), its multiplier and the ratio from the literal energy difference
    g = lb.gradient(p, w.phi0)
    hc, u = sp.dense_hessian(p, w.phi0)
    c, lam, _ = sp.more_sorensen(hc, sp.to_coords(u, g), r0)
    s = sp.from_coords(u, c, w.shape)
    assert abs(entry["snorm"] - lb.norm(s)) <= 1e-8 * lb.norm(s)
    assert abs(entry["lambda"] - lam) <= 1e-7 * max(1.0, lam)
    rho = tr.energy_drop_direct(p, w.phi0, s) / lb.norm(s) ** 3
    assert abs(entry["rho"] - rho) <= 1e-6 * max(1.0, abs(rho))


def test_tr_step_accept_on_the_nu_boundary():
    # Algorithm 1: rho >= theta with ||s|| = nu (lambda > mu ||s||): accepted;
    # nu_1 = max(nu_0, gamma_E ||s||), r_1 = min(nu_1, max(r_0, gamma_E ||s||)),
    # mu_1 = max(mu_0, lambda / ||s||)
    w, p, log = _tr_case(dict(r0=0.01, nu0=0.01), 1)
    e = log[0]
    _check_first_step_is_global_minimiser(w, p, e, 0.01)
    assert e["step"] == "accept"
    assert e["lambda"] > 1.0 * e["snorm"] and e["rho"] >= 1e-4
    assert abs(e["snorm"] - 0.01) <= 1e-12 * 0.01
    assert e["nu"] == pytest.approx(0.02, rel=1e-12)
    assert e["r"] == pytest.approx(0.02, rel=1e-12)
    assert e["mu"] == pytest.approx(e["lambda"] / e["snorm"], rel=1e-12)
    assert e["E"] < lb.energy(p, w.phi0)


def test_tr_step_shrink_then_accept_without_mu_update():
    # j = 0: rho >= theta but lambda > mu_0 ||s|| and ||s|| < nu: the iterate stays, r_1 =
    # min(nu_0, lambda / mu_0), mu and nu unchanged.  j = 1: rho_0 >= theta, so mu is NOT
    # raised before the test; here lambda_1 <= mu_1 ||s_1|| anyway, so the step is accepted
    # with r_2 = min(nu, max(r_1, gamma_E ||s_1||)).
    w, p, log = _tr_case(dict(r0=0.01, mu0=1e4), 2)
    e0, e1 = log
    _check_first_step_is_global_minimiser(w, p, e0, 0.01)
    assert e0["step"] == "shrink"
    assert e0["rho"] >= 1e-4 and e0["lambda"] > 1e4 * e0["snorm"]
    assert e0["r"] == pytest.approx(e0["lambda"] / 1e4, rel=1e-12)
    assert e0["r"] < 5.0
    assert e0["nu"] == 5.0 and e0["mu"] == 1e4
    assert e0["E"] == pytest.approx(lb.energy(p, w.phi0), rel=1e-15)
    assert e1["step"] == "accept"
    assert e1["mu"] == 1e4                          # max(1e4, lambda_1 / ||s_1||) = 1e4
    assert abs(e1["snorm"] - e0["r"]) <= 1e-9 * e0["r"]     # the step fills the new radius
    assert e1["r"] == pytest.approx(min(5.0, max(e0["r"], 2.0 * e1["snorm"])), rel=1e-12)


def test_tr_step_contract_then_mu_update_forces_accept():
    # j = 0: a radius-5 step raises the energy (rho < theta): CONTRACT, first branch
    # (lambda_0 < mu_lo ||s_0||), r_1 = ||s(lambda^)||, nu and mu unchanged.  j = 1: rho_0 <
    # theta, so mu_1 = max(mu_0, lambda_1 / ||s_1||) BEFORE the acceptance test, which then
    # holds (lambda_1 <= mu_1 ||s_1||); without that update the step would be a shrink.
    w, p, log = _tr_case(dict(r0=5.0, nu0=5.0), 2)
    e0, e1 = log
    assert e0["step"] == "contract"
    assert e0["rho"] < 1e-4 and e0["lambda"] < 1.0 * e0["snorm"]
    assert e0["nu"] == 5.0 and e0["mu"] == 1.0
    g = lb.gradient(p, w.phi0)
    hc, u = sp.dense_hessian(p, w.phi0)
    lam_hat = e0["lambda"] + math.sqrt(lb.norm(g))
    want = _snorm_dense(hc, u, g, lam_hat)
    assert lam_hat / want <= 1e5
    assert e0["r"] == pytest.approx(want, rel=1e-8)
    assert e1["step"] == "accept"
    assert e1["lambda"] > 1.0 * e1["snorm"]          # mu_0 = 1 alone would not accept
    assert e1["mu"] == pytest.approx(e1["lambda"] / e1["snorm"], rel=1e-12)
    assert e1["r"] == pytest.approx(min(5.0, max(e0["r"], 2.0 * e1["snorm"])), rel=1e-12)
    assert e1["nu"] == pytest.approx(max(5.0, 2.0 * e1["snorm"]), rel=1e-12)


def test_step_kind_accepts_after_the_mu_update_despite_rounding():
    # Algorithm 1: after a failed ratio mu_j = max(mu, lambda_j / ||s_j||), so lambda_j <=
    # mu_j ||s_j|| holds and a step with rho_j >= theta is accepted.  For this pair the product
    # (lambda / s) * s rounds one ulp below lambda; evaluated as a product the test would
    # fail and the shrink branch would return r = lambda / mu = ||s||, the same subproblem.
    prm = dict(tr.PAPER_PARAMS)
    lam, sn = 0.21659939713061338, 0.4221165755827173
    mu = max(0.5, lam / sn)                          # the update after a failed ratio
    assert (lam / sn) * sn < lam                     # the rounding the test guards against
    assert tr.step_kind(0.5, lam, sn, mu, 5.0, prm) == "accept"
    # the other branches: a failed ratio contracts; lambda / ||s|| above mu (and ||s|| < nu)
    # shrinks; ||s|| = nu accepts whatever lambda is
    assert tr.step_kind(1e-5, lam, sn, mu, 5.0, prm) == "contract"
    assert tr.step_kind(0.5, lam, sn, 0.99 * lam / sn, 5.0, prm) == "shrink"
    assert tr.step_kind(0.5, lam, sn, 0.99 * lam / sn, sn, prm) == "accept"
    assert tr.step_kind(prm["theta"], lam, sn, mu, 5.0, prm) == "accept"   # rho = theta accepts

