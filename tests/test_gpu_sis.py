"""The first-order gradient flow (lb_sis_solve) against the oracle's semi-implicit scheme.

A fixed number of steps (eps = 0) on 2D and 3D grids, including a 32^3 grid on the plane
kernels; FP64 in both precisions, tolerance 1e-11 relative in max norm for the field (FFT
rounding over 25 steps of a contraction), 1e-12 for the energy, 1e-9 for max |g|.  Argument errors are checked on the host path.
"""
import numpy as np
import pytest

from oracle import first_order as fo
from oracle import lb as olb
from paper_2603_03933_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def lbtr():
    from paper_2603_03933_gb300 import build, lbtr as mod
    build.build(force=False)
    mod.load()
    return mod


CASES = [
    (inputs.random_problem((32, 32), 51, sigma=0.3, box=(9.0, 7.0), tau=-0.15, gamma=0.25), 0.5, "fp64"),
    (inputs.random_problem((16, 16, 16), 52, sigma=0.3, box=(6.0, 6.5, 7.0), tau=-0.2, gamma=0.3), 1.0, "fp64"),
    (inputs.table2_phase("LAM", 32), 1.0, "mixed"),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_sis_steps_match_oracle(lbtr, case):
    w, dt, prec = CASES[case]
    p = olb.Problem.from_workload(w)
    ctx = lbtr.lb_create_from_array_box(w.shape, w.box, w.xi, w.tau, w.gamma,
                                        lbtr.LB_FP64 if prec == "fp64" else lbtr.LB_MIXED)
    phi = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
    o = lbtr.default_sis_opts()
    o.dt, o.eps, o.max_steps, o.check_every = dt, 0.0, 25, 7
    info = lbtr.lb_sis_solve(ctx, phi, opts=o, raise_on_noconv=False)
    assert info["status"] == 4 and info["steps"] == 25
    ref, steps, e, gmax = fo.sis_solve(p, w.phi0, dt, 0.0, 25)
    got = phi.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))
    assert abs(info["energy"] - e) <= 1e-12 * max(1.0, abs(e))
    # max |g| carries the field's rounding error times max Lambda (~1e3 on these grids)
    assert abs(info["gmax"] - gmax) <= 1e-9 * max(gmax, 1e-30)


def test_sis_converges_and_reports(lbtr):
    w = inputs.random_problem((16, 16), 53, sigma=0.3, box=(8.0, 8.0), tau=-0.2, gamma=0.3)
    ctx = lbtr.lb_create_from_array_box(w.shape, w.box, w.xi, w.tau, w.gamma, lbtr.LB_FP64)
    phi = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
    o = lbtr.default_sis_opts()
    o.eps = 1e-9
    info = lbtr.lb_sis_solve(ctx, phi, opts=o)
    assert info["status"] == 0 and info["gmax"] < 1e-9
    p = olb.Problem.from_workload(w)
    g = olb.gradient(p, phi.cpu().numpy())
    assert np.max(np.abs(g)) < 1e-9
    assert abs(info["energy"] - olb.energy(p, phi.cpu().numpy())) <= 1e-12


def test_sis_argument_errors(lbtr):
    w = inputs.random_problem((16, 16), 54)
    ctx = lbtr.lb_create_from_array_box(w.shape, w.box, w.xi, w.tau, w.gamma, lbtr.LB_FP64)
    phi = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
    o = lbtr.default_sis_opts()
    o.dt = 0.0
    with pytest.raises(lbtr.LBError):
        lbtr.lb_sis_solve(ctx, phi, opts=o)
    bad = torch.tensor(w.phi0 + 0.1, dtype=torch.float64, device=DEV)
    with pytest.raises(lbtr.LBError):
        lbtr.lb_sis_solve(ctx, bad)


def _amps(t):
    x = t.cpu().numpy()
    return np.sort(np.abs(np.fft.fftn(x) / x.size).ravel())[::-1]


def test_imex_tr_post_processing_of_the_first_order_trajectory(lbtr):
    # Example 1 of Table 1, (tau, gamma) = (-0.35, 0.7), LAM start on [0, 2 sqrt(2) pi]^3:
    # the first-order flow stays in the LAM basin and converges to a saddle; IMEX-TR
    # started from the initial point, an intermediate state or that saddle reaches the
    # same SP-II, the HEX phase (six modes of equal amplitude), at lower energy.
    w = inputs.table2_phase("LAM", 32)
    ctx = lbtr.lb_create_from_array_box(w.shape, w.box, 1.0, -0.35, 0.7, lbtr.LB_FP64)
    phi = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
    starts = {"initial": phi.clone()}
    o = lbtr.default_sis_opts()
    o.eps, o.max_steps, o.check_every = 1e-6, 20, 1
    lbtr.lb_sis_solve(ctx, phi, opts=o, raise_on_noconv=False)
    starts["intermediate"] = phi.clone()
    o.max_steps = 5000
    sis = lbtr.lb_sis_solve(ctx, phi, opts=o)
    starts["saddle"] = phi.clone()
    a = _amps(phi)
    assert sis["gmax"] < 1e-6
    assert abs(a[0] - a[1]) <= 1e-9 * a[0] and a[2] < 0.25 * a[0]          # LAM: one +-k pair leads
    assert lbtr.lb_lambda_min(ctx, phi, raise_on_noconv=False)["lambda_min"] < -0.1
    energies = []
    for name, st in starts.items():
        ph = st.clone()
        t = lbtr.default_tr_opts()
        t.eps, t.max_outer, t.hard_tol = 1e-8, 300, 1e-12
        t.sub.max_iter, t.eig.max_steps = 5000, 200
        info = lbtr.lb_imex_tr_solve(ctx, ph, opts=t, raise_on_noconv=False)
        assert info["status"] == 0 and info["gmax"] < 1e-8, name
        assert lbtr.lb_lambda_min(ctx, ph, raise_on_noconv=False)["lambda_min"] >= -1e-8, name
        a = _amps(ph)
        assert np.allclose(a[:6], a[0], rtol=1e-6) and a[6] < 0.05 * a[0], name
        energies.append(info["energy"])
    assert max(energies) - min(energies) <= 1e-10 and max(energies) < sis["energy"] - 0.1
