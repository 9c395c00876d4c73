"""lb_hessvec_noalloc: the Hessian-vector product for callers that cannot allocate.

Callers whose host framework owns all device memory, or whose loops cannot afford the
device synchronisation of cudaMalloc, use this entry point instead of a context.  It
must give the same product as lb_hessvec (same tolerances as the parity tests), on
consecutive calls that share its fixed scratch array, and refuse grids beyond it.
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


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("shape,prec", [((64, 64), "fp64"), ((512, 512), "mixed"),
                                        ((16, 16, 16), "fp64"), ((32, 32, 32), "mixed"), ((64, 64, 64), "fp64")])
def test_noalloc_matches_hessvec_on_consecutive_calls(lbtr, shape, prec):
    p = lbtr.LB_FP64 if prec == "fp64" else lbtr.LB_MIXED
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 2e-5
    box_xyz = [7.0 + a for a in range(len(shape))]
    box_arr = box_xyz[::-1]
    for call in range(2):     # two calls in a row reuse the same scratch
        w = inputs.random_problem(shape, 500 + call, sigma=0.3, box=box_arr, tau=-0.1 - 0.05 * call)
        phi = torch.tensor(w.phi0, dtype=dt, device=DEV)
        v = torch.tensor(inputs.gaussian_field(shape, 1.0, 600 + call), dtype=dt, device=DEV)
        ctx = lbtr.lb_create(len(shape), shape[0], box_xyz, w.xi, w.tau, w.gamma, p)
        ref = torch.empty_like(v)
        lbtr.lb_hessvec(ctx, phi, v, ref)
        out = torch.full_like(v, float("nan"))
        lbtr.lb_hessvec_noalloc(len(shape), shape[0], box_xyz, w.xi, w.tau, w.gamma, p, phi, v, out)
        torch.cuda.synchronize()
        assert _rel(out.double().cpu().numpy(), ref.double().cpu().numpy()) < tol


def test_noalloc_rejects_grids_beyond_its_scratch(lbtr):
    shape = (128, 128, 128)
    z = torch.zeros(shape, dtype=torch.float32, device=DEV)
    with pytest.raises(lbtr.LBError) as e:
        lbtr.lb_hessvec_noalloc(3, 128, (5.0, 5.0, 5.0), 1.0, -0.1, 0.2, lbtr.LB_MIXED, z, z.clone(), z.clone())
    assert e.value.status == 8
