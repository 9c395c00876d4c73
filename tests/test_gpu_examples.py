"""Examples 2 and 3 of the paper's Table 1 (§4.1) run through lb_imex_tr_solve.

Example 2: (tau, gamma) = (-0.001, 0.4), cubic box [0, 2 sqrt(2) pi]^3, LAM start.  The paper
reports that IMEX-TR reaches the BCC phase, an SP-II (first-order schemes end at the
disordered state), and prints no energy for it.  Checked: the end state is an SP-II whose
field carries the twelve {110} modes (|B k| = 1 in this box) at one common amplitude, with the
oracle's energy and gradient at the returned field; the same energy at 32^3 and 64^3 and in
both precisions (the state is band-limited, so the grid does not change it).  The exact LAM
start lies in the lamellar subspace, which the iteration preserves; the SP-II test at a
saddle of that subspace starts the next subproblem from a random point of the ball, and the
nearly-hard-case test does the same (hard_tol), which is how the run leaves it.

Example 3: (tau, gamma) = (-0.28, 0.32), cubic box [0, 2 sqrt(6) pi]^3, HEX start (Table 2).
From the exact HEX start the iteration converges to the HEX phase, an SP-II, at the energy the
paper prints for HEX, E = -8.02e-2 (three digits: |E + 0.0802| <= 5e-5); the paper's run left the
HEX basin for a network SP-II at -8.05e-2, which this start does not reach (the paper states
neither its grid nor its inner tolerances).  The end state carries the six HEX modes at equal
amplitude.
"""
import json
import os

import numpy as np
import pytest

from oracle import lb as olb
from paper_2603_03933_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"
PAPER = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


@pytest.fixture(scope="module")
def lbtr():
    from paper_2603_03933_gb300 import build, lbtr as mod
    build.build(force=False)
    mod.load()
    return mod


def _paper():
    with open(PAPER) as f:
        return json.load(f)


def _solve(lbtr, w, tau, gamma, hard_tol=1e-12, prec="fp64"):
    c = lbtr.lb_create_from_array_box(w.shape, w.box, 1.0, tau, gamma,
                                      lbtr.LB_FP64 if prec == "fp64" else lbtr.LB_MIXED)
    phi = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
    o = lbtr.default_tr_opts()
    o.eps, o.tol2, o.second_order, o.max_outer = 1e-8, 1e-8, 1, 400
    o.sub.max_iter, o.sub.eps_sub, o.sub.rel_tol = 5000, 0.0, 1e-4
    o.hard_tol = hard_tol
    info = lbtr.lb_imex_tr_solve(c, phi, opts=o)
    return info, phi.cpu().numpy()


@pytest.mark.parametrize("M", [32, 64])
def test_example3_hex_start_ends_at_the_hex_sp2_with_the_papers_energy(lbtr, M):
    pv = _paper()
    ex = pv["table1_examples"]["3"]
    w = inputs.table2_phase("HEX", M)
    assert (w.tau, w.gamma) == (ex["tau"], ex["gamma"])
    info, x = _solve(lbtr, w, w.tau, w.gamma)
    assert info["status"] == 0 and info["gmax"] < 1e-8 and info["lambda_min"] >= -1e-8
    assert abs(info["energy"] - pv["converged_energies"]["example3_hex"]) <= 5e-5
    # the oracle's energy and gradient at the returned field
    p = olb.Problem.from_workload(w)
    assert abs(olb.energy(p, x) - info["energy"]) <= 1e-12
    assert np.max(np.abs(olb.gradient(p, x))) < 1e-8
    amp = np.sort(np.abs(np.fft.fftn(x) / x.size).ravel())[::-1]
    assert np.allclose(amp[:6], amp[0], rtol=1e-6) and amp[6] < 0.05 * amp[0]


_BCC_E = {}


@pytest.mark.parametrize("M,prec", [(32, "fp64"), (64, "fp64"), (32, "mixed")])
def test_example2_lam_start_reaches_the_bcc_sp2(lbtr, M, prec):
    ex = _paper()["table1_examples"]["2"]
    w = inputs.table2_phase("LAM", M)                     # the LAM start of Table 2, side 2 sqrt(2) pi
    info, x = _solve(lbtr, w, ex["tau"], ex["gamma"], prec=prec)
    assert info["status"] == 0 and info["gmax"] < 1e-8 and info["lambda_min"] >= -1e-8
    p = olb.Problem.from_workload(inputs.Workload(w.name, w.shape, w.box, 1.0, ex["tau"], ex["gamma"], w.phi0))
    assert abs(olb.energy(p, x) - info["energy"]) <= 1e-12
    assert np.max(np.abs(olb.gradient(p, x))) < 1e-8
    assert info["energy"] < olb.energy(p, w.phi0) and info["energy"] < 0.0   # below the start and below phi = 0
    F = np.fft.fftn(x) / x.size
    order = np.argsort(np.abs(F).ravel())[::-1]
    amp = np.abs(F).ravel()[order]
    assert np.allclose(amp[:12], amp[0], rtol=1e-6) and amp[12] < 0.05 * amp[0]
    for i in order[:12]:
        k = sorted(abs(((i // s) % M + M // 2) % M - M // 2) for s in (M * M, M, 1))
        assert k == [0, 1, 1]                              # the {110} family
    _BCC_E[(M, prec)] = info["energy"]
    if len(_BCC_E) > 1:
        es = list(_BCC_E.values())
        assert max(es) - min(es) <= 1e-12


def test_example2_first_order_flow_ends_at_the_disordered_saddle(lbtr):
    # the semi-implicit gradient flow from the same start ends at phi = 0, a saddle whose
    # Hessian Lambda + tau has lambda_min = tau = -0.001 (on the |B k| = 1 modes): the paper's
    # finding that first-order schemes converge to the disordered state in Example 2
    ex = _paper()["table1_examples"]["2"]
    w = inputs.table2_phase("LAM", 32)
    c = lbtr.lb_create_from_array_box(w.shape, w.box, 1.0, ex["tau"], ex["gamma"], lbtr.LB_FP64)
    phi = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
    o = lbtr.default_sis_opts()
    o.dt, o.eps, o.max_steps, o.check_every = 1.0, 1e-8, 200000, 100
    info = lbtr.lb_sis_solve(c, phi, opts=o)
    assert info["status"] == 0 and info["gmax"] < 1e-8
    assert float(phi.abs().max()) < 1e-6 and abs(info["energy"]) < 1e-12
    lam = lbtr.lb_lambda_min(c, phi, raise_on_noconv=False)["lambda_min"]
    assert abs(lam - ex["tau"]) < 1e-8

