"""Bitwise repeatability (the race check of a library without a sanitizer): every reduction
sums its partials in a fixed order and no kernel accumulates floats with atomics, so the
same call on the same inputs must give the same bits.  A race in a transpose, a barrier or
a grid reduction would show up here as a difference between two runs.
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


def _ctx(lbtr, w, prec):
    return lbtr.lb_create_from_array_box(w.shape, w.box, w.xi, w.tau, w.gamma, prec)


@pytest.mark.parametrize("shape", [(128, 128, 128), (256, 256), (32, 32, 32)])
def test_hessvec_and_gradient_twice(lbtr, shape):
    w = inputs.random_problem(shape, 401, sigma=0.3)
    v = inputs.gaussian_field(shape, 1.0, 402)
    for prec, dt in ((lbtr.LB_MIXED, torch.float32), (lbtr.LB_FP64, torch.float64)):
        ctx = _ctx(lbtr, w, prec)
        phi = torch.tensor(w.phi0, dtype=dt, device=DEV)
        vt = torch.tensor(v, dtype=dt, device=DEV)
        outs = []
        for _ in range(2):
            hv = torch.empty_like(vt)
            g = torch.empty_like(phi)
            lbtr.lb_hessvec(ctx, phi, vt, hv)
            e, gmax = lbtr.lb_energy_grad(ctx, phi, g)
            outs.append((hv, g, e, gmax))
        torch.cuda.synchronize()
        (h0, g0, e0, m0), (h1, g1, e1, m1) = outs
        assert torch.equal(h0, h1) and torch.equal(g0, g1) and e0 == e1 and m0 == m1


def test_subproblem_twice(lbtr):
    # the fused cooperative IMEX kernel: grid barriers, secular Newton, stall test
    w = inputs.random_problem((32, 32, 32), 403, sigma=0.3, tau=-0.2, gamma=0.3)
    p = olb.Problem.from_workload(w)
    ctx = _ctx(lbtr, w, lbtr.LB_MIXED)
    phi32 = torch.tensor(w.phi0, dtype=torch.float32, device=DEV)
    g32 = torch.tensor(olb.gradient(p, phi32.double().cpu().numpy()), dtype=torch.float32, device=DEV)
    opts = lbtr.default_sub_opts()
    opts.eps_sub, opts.rel_tol, opts.max_iter = 0.0, 1e-5, 5000
    runs = []
    for _ in range(2):
        d = torch.empty_like(phi32)
        info = lbtr.lb_tr_subproblem(ctx, phi32, g32, 0.5, d, opts=opts, raise_on_noconv=False)
        runs.append((d, info))
    (d0, i0), (d1, i1) = runs
    assert torch.equal(d0, d1)
    assert (i0["iterations"], i0["lambda"], i0["newton_steps"]) == (i1["iterations"], i1["lambda"], i1["newton_steps"])
