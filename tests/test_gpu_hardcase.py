"""The nearly hard case (the paper's §4, "Beyond the theoretical scope"): the LAM phase of
Example 1's domain at (tau, gamma) = (-0.09, 0.34), solved without the second-order escape,
once with the deterministic inner start -r g / ||g|| only and once with a random start on
every subproblem whose g^(1) (the component of g along the eigenvector of a negative
lambda_min) is below 1e-12.  The symmetric start makes g^(1) vanish, so the deterministic
run cannot leave the symmetric subspace and stops at a point that is not an SP-II; the
randomized run reaches the HEX phase, an SP-II, at the paper's energy E = -1.32e-2.  Both
runs are made at two resolutions of the same box (32^3 and 64^3), so that the end states
are properties of the iteration and not of one grid.
"""
import numpy as np
import pytest

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


def _solve(lbtr, hard_tol, M):
    w = inputs.table2_phase("LAM", M)
    c = lbtr.lb_create_from_array_box(w.shape, w.box, 1.0, -0.09, 0.34, lbtr.LB_FP64)
    phi = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
    o = lbtr.default_tr_opts()
    o.eps = 1e-8
    o.max_outer = 300
    o.second_order = 0
    o.hard_tol = hard_tol
    o.sub.max_iter = 5000
    o.eig.max_steps = 200
    info = lbtr.lb_imex_tr_solve(c, phi, opts=o, raise_on_noconv=False)
    lam = lbtr.lb_lambda_min(c, phi)["lambda_min"]
    x = phi.cpu().numpy()
    amp = np.sort(np.abs(np.fft.fftn(x) / x.size).ravel())[::-1]
    return info, lam, amp, x


@pytest.mark.parametrize("M", [32, 64])
def test_randomized_start_on_nearly_hard_subproblems_reaches_hex(lbtr, M):
    info, lam, amp, _ = _solve(lbtr, 1e-12, M)
    assert info["status"] == 0 and info["gmax"] < 1e-8
    assert info["randomized"] >= 1 and info["g1_min"] <= 1e-12
    assert lam >= -1e-8                                   # SP-II
    assert abs(info["energy"] - (-1.32e-2)) <= 0.01 * 1.32e-2
    # HEX: six modes (three +-k pairs) of equal amplitude carry the field
    assert np.allclose(amp[:6], amp[0], rtol=1e-6) and amp[6] < 0.05 * amp[0]


@pytest.mark.parametrize("M", [32, 64])
def test_deterministic_start_stops_at_a_point_that_is_not_sp2(lbtr, M):
    info, lam, _, x = _solve(lbtr, 0.0, M)
    assert info["status"] == 0 and info["randomized"] == 0
    # the point reached is the disordered state phi = 0: a critical point whose Hessian is
    # Lambda + tau (F''(0) = tau), so lambda_min = tau = -0.09, attained on the LAM
    # wavevectors (|B k| = 1, Lambda = 0), which lie on the grid at every resolution
    assert np.max(np.abs(x)) < 1e-6 and abs(info["energy"]) < 1e-12
    assert abs(lam - (-0.09)) < 1e-6
