"""lb_hessvec_host: Hessian-vector products of host-resident fields through the C ABI, the
copies in and out overlapped with the products on three device staging slots.

Each product must equal the device-resident lb_hessvec of the same fields bit for bit (the
same kernels on the same values), for page-locked and for pageable host memory, for more
products than slots (slot reuse), in both precisions; one product is also checked against
the oracle.  Argument errors are reported, and an empty batch does nothing.
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


@pytest.mark.parametrize("shape,prec,count,pinned", [((128, 128, 128), "mixed", 7, True),
                                                     ((128, 128, 128), "mixed", 2, False),
                                                     ((64, 64, 64), "fp64", 5, True),
                                                     ((256, 256), "mixed", 4, True)])
def test_host_products_equal_device_products(lbtr, shape, prec, count, pinned):
    p = lbtr.LB_FP64 if prec == "fp64" else lbtr.LB_MIXED
    dt = torch.float64 if prec == "fp64" else torch.float32
    w = inputs.random_problem(shape, 21, sigma=0.2, box=tuple(float(10 + i) for i in range(len(shape))))
    ctx = lbtr.lb_create_from_array_box(w.shape, w.box, w.xi, w.tau, w.gamma, p)
    phi = torch.tensor(w.phi0, dtype=dt)
    vs = [torch.tensor(inputs.gaussian_field(w.shape, 1.0, 300 + i), dtype=dt) for i in range(count)]
    hvs = [torch.full_like(v, float("nan")) for v in vs]
    if pinned:
        phi, vs, hvs = phi.pin_memory(), [v.pin_memory() for v in vs], [h.pin_memory() for h in hvs]
    lbtr.lb_hessvec_host(ctx, phi, vs, hvs)
    phi_d = phi.to(DEV)
    for v, h in zip(vs, hvs):
        ref = torch.empty_like(phi_d)
        lbtr.lb_hessvec(ctx, phi_d, v.to(DEV), ref)
        torch.cuda.synchronize()
        assert torch.equal(h, ref.cpu())
    pr = olb.Problem.from_workload(w)
    want = olb.hessvec(pr, phi.double().numpy(), vs[-1].double().numpy())
    got = hvs[-1].double().numpy()
    assert np.max(np.abs(got - want)) <= (1e-12 if prec == "fp64" else 2e-5) * np.max(np.abs(want))


def test_host_entry_argument_errors(lbtr):
    w = inputs.random_problem((32, 32), 3, sigma=0.2)
    ctx = lbtr.lb_create_from_array_box(w.shape, w.box, w.xi, w.tau, w.gamma, lbtr.LB_FP64)
    phi = torch.tensor(w.phi0, dtype=torch.float64)
    v = torch.zeros_like(phi)
    lbtr.lb_hessvec_host(ctx, phi, [], [])                  # empty batch: nothing to do
    with pytest.raises(lbtr.LBError) as e:
        lbtr.lb_hessvec_host(ctx, phi, [v], [v])             # output aliases its input
    assert e.value.status == 1
    with pytest.raises(ValueError):
        lbtr.lb_hessvec_host(ctx, phi.to(DEV), [v], [torch.empty_like(v)])
