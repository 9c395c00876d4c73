"""The one-launch inner loop of the subproblem (Algorithm 3 as one cooperative kernel,
k_imex3) at 128^3 in mixed precision, against the per-iteration launches of the same
algorithm (k_plane_mid + k_imex_lines, host polling between chunks of iterations).

Both take the same decisions from the same sums, in float, up to summation order: the
iterates differ by float rounding (bounded as in the fixed-iteration oracle parity,
4 eps_f (||d|| + eta ||g||)), and where the stop test ends both runs the iteration counts
agree to within the few iterations over which the residual sits near the threshold.  The
stall exit, the iteration cap and the barrier timeout behave as in the per-iteration form.
"""
import numpy as np
import pytest

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


def _setup(lbtr, w):
    phi = torch.tensor(w.phi0, dtype=torch.float32, device=DEV)
    ctx = lbtr.lb_create_from_array_box(w.shape, w.box, w.xi, w.tau, w.gamma, lbtr.LB_MIXED)
    g = torch.empty_like(phi)
    lbtr.lb_energy_grad(ctx, phi, g)
    return ctx, phi, g


def _norm(x):
    return float(torch.linalg.vector_norm(x.double()) / np.sqrt(x.numel()))


def _solve(lbtr, ctx, phi, g, r, persistent, **kw):
    lbtr.lb_set_persistent_subproblem(ctx, persistent)
    o = lbtr.default_sub_opts()
    for k, v in kw.items():
        setattr(o, k, v)
    d = torch.empty_like(phi)
    info = lbtr.lb_tr_subproblem(ctx, phi, g, r, d, opts=o, raise_on_noconv=False)
    return info, d


def test_available_only_at_128cubed_mixed(lbtr):
    for shape, prec, want in [((128, 128, 128), lbtr.LB_MIXED, True), ((128, 128, 128), lbtr.LB_FP64, False),
                              ((64, 64, 64), lbtr.LB_MIXED, False), ((128, 128), lbtr.LB_MIXED, False)]:
        box = (10.0,) * len(shape)
        ctx = lbtr.lb_create_from_array_box(shape, box, 1.0, -0.1, 0.2, prec)
        assert lbtr.lb_persistent_subproblem_available(ctx) == want
        lbtr.lb_set_persistent_subproblem(ctx, False)
        assert not lbtr.lb_persistent_subproblem_available(ctx)


@pytest.mark.parametrize("r,rel_tol", [(1.0, 1e-4), (0.05, 1e-5), (50.0, 1e-4)])
def test_converged_solve_matches_per_iteration_launches(lbtr, r, rel_tol):
    # r = 1: the boundary case with Newton steps of the multiplier rule; r = 50: an interior
    # solution (lambda = 0 from the first iteration on)
    w = inputs.config_3d_scale(128)
    ctx, phi, g = _setup(lbtr, w)
    ia, da = _solve(lbtr, ctx, phi, g, r, True, eps_sub=0.0, rel_tol=rel_tol, max_iter=5000)
    ib, db = _solve(lbtr, ctx, phi, g, r, False, eps_sub=0.0, rel_tol=rel_tol, max_iter=5000)
    assert ia["status"] == ib["status"] == 0 and ia["converged"] and ib["converged"]
    assert abs(ia["iterations"] - ib["iterations"]) <= max(3, ib["iterations"] // 100)
    gn = _norm(g)
    eps_f = 2.0 ** -24
    # both iterates meet the requested accuracy; they are two float iterates of the same
    # contraction, each within rel_tol ||g|| / (contraction margin) of the exact solution
    assert ia["rel_residual"] < rel_tol and ib["rel_residual"] < rel_tol
    assert abs(ia["lambda"] - ib["lambda"]) <= 1e-4 * (1 + ib["lambda"])
    # the same iteration in both forms: float rounding of the iterates (as in the fixed-
    # iteration parity) plus, per iteration by which the stop points differ, at most one
    # step d_{j+1} - d_j, whose size is eta times the residual (eq. imex-scheme)
    steps = abs(ia["iterations"] - ib["iterations"]) + 1
    assert _norm(da - db) <= 4 * eps_f * (_norm(db) + 0.1 * gn) + 2 * steps * 0.1 * rel_tol * gn
    assert _norm(da) <= r * (1 + 1e-5)
    if r == 50.0:
        assert ia["lambda"] == 0.0 and ib["lambda"] == 0.0
    # the model value reported with the iterate is the same quadratic model
    assert abs(ia["model_value"] - ib["model_value"]) <= 1e-4 * abs(ib["model_value"])


def test_returned_iterate_meets_the_tolerance(lbtr):
    # the returned d, written by the kernel's final z step and plane inverse, checked with the
    # oracle's FP64 Hessian on the same float-rounded inputs: the residual of the shifted
    # system g + (H + lambda) d meets the requested tolerance, and the multiplier satisfies
    # the Corollary's complementarity (lambda > 0 only with ||d|| = r)
    rel_tol = 1e-4
    w = inputs.config_3d_scale(128)
    ctx, phi, g = _setup(lbtr, w)
    info, d = _solve(lbtr, ctx, phi, g, 1.0, True, eps_sub=0.0, rel_tol=rel_tol, max_iter=5000)
    assert info["converged"] and info["rel_residual"] < rel_tol
    p = olb.Problem.from_workload(w)
    x = phi.double().cpu().numpy()
    dd = d.double().cpu().numpy()
    gg = g.double().cpu().numpy()
    res = gg + olb.hessvec(p, x, dd) + info["lambda"] * dd
    res -= res.mean()
    assert olb.norm(res) < rel_tol * olb.norm(gg)
    assert abs(dd.mean()) <= 1e-6 * olb.norm(dd)
    assert info["lambda"] >= 0.0
    if info["lambda"] > 0.0:
        assert abs(olb.norm(dd) - 1.0) <= 1e-5
    else:
        assert olb.norm(dd) <= 1.0 + 1e-5


def test_stall_and_cap_exits(lbtr):
    w = inputs.config_3d_scale(128)
    ctx, phi, g = _setup(lbtr, w)
    # a relative tolerance below float resolution: the stall exit (status NOCONV, stalled)
    info, _ = _solve(lbtr, ctx, phi, g, 1.0, True, eps_sub=0.0, rel_tol=1e-13, max_iter=20000)
    assert info["status"] == 4 and info["stalled"] and not info["converged"]
    assert info["iterations"] < 20000 and info["rel_residual"] > 1e-13
    # the cap: exactly max_iter iterations
    info, _ = _solve(lbtr, ctx, phi, g, 1.0, True, eps_sub=0.0, rel_tol=0.0, max_iter=7)
    assert info["status"] == 4 and not info["stalled"] and not info["converged"]
    assert info["iterations"] == 7


def test_barrier_timeout_is_reported_and_the_context_recovers(lbtr):
    w = inputs.config_3d_scale(128)
    ctx, phi, g = _setup(lbtr, w)
    lbtr.lb_set_persistent_subproblem(ctx, True)
    d = torch.empty_like(phi)
    lbtr.lb_set_barrier_budget(ctx, 1)
    with pytest.raises(lbtr.LBError) as e:
        lbtr.lb_tr_subproblem(ctx, phi, g, 1.0, d)
    assert e.value.status == 5
    lbtr.lb_set_barrier_budget(ctx, 0)
    o = lbtr.default_sub_opts()
    o.rel_tol = 1e-4
    info = lbtr.lb_tr_subproblem(ctx, phi, g, 1.0, d, opts=o)
    assert info["converged"]
