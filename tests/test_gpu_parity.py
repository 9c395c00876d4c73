"""Parity of the CUDA path with the FP64 oracle on seeded inputs (calls go through the C ABI).

Tolerances: FP64 path - energy 1e-12 relative, gradient 1e-10 relative max-norm,
Hessian-vector product 1e-12 relative max-norm.  MIXED path - inputs are rounded to
float32 and the oracle runs on the rounded values in FP64; energy 1e-6 relative,
gradient and Hv 2e-5 relative max-norm (float32 FFTs, double reductions).  MIXED
subproblem: the float iteration stops at a relative residual, so d is checked against a
bound derived from that residual and the model value f(d) against the exact minimum.
"""
import math

import numpy as np
import pytest

from oracle import lb as olb
from oracle import subproblem as osp
from paper_2603_03933_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lbtr():
    from paper_2603_03933_gb300 import build, lbtr as mod
    build.build(force=False)
    mod.load()
    return mod


DEV = "cuda:0"

GRIDS = [
    ((8, 8), None), ((16, 16), None), ((32, 32), (5.0, 9.0)), ((64, 64), None), ((128, 128), None),
    ((256, 256), None), ((512, 512), None),
    ((8, 8, 8), None), ((16, 16, 16), (5.0, 6.0, 7.0)), ((32, 32, 32), None), ((64, 64, 64), None),
    ((128, 128, 128), None),
]


def _ctx(lbtr, w, prec):
    return lbtr.lb_create_from_array_box(w.shape, w.box, w.xi, w.tau, w.gamma, prec)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("shape,box", GRIDS)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_hessvec_parity(lbtr, shape, box, prec):
    w = inputs.random_problem(shape, 101, sigma=0.3, box=box)
    v = inputs.gaussian_field(shape, 1.0, 102)
    dt = torch.float64 if prec == "fp64" else torch.float32
    phi_t = torch.tensor(w.phi0, dtype=dt, device=DEV)
    v_t = torch.tensor(v, dtype=dt, device=DEV)
    phi_in = phi_t.double().cpu().numpy()
    v_in = v_t.double().cpu().numpy()
    ctx = _ctx(lbtr, w, lbtr.LB_FP64 if prec == "fp64" else lbtr.LB_MIXED)
    hv = torch.empty_like(v_t)
    lbtr.lb_hessvec(ctx, phi_t, v_t, hv)
    torch.cuda.synchronize()
    p = olb.Problem.from_workload(w)
    # the library takes v as given (zero mean up to rounding); the oracle's H applies P to it
    ref = olb.hessvec(p, phi_in, v_in - v_in.mean())
    err = _rel(hv.double().cpu().numpy(), ref)
    assert err < (1e-12 if prec == "fp64" else 2e-5), err


@pytest.mark.parametrize("shape,box", GRIDS)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_energy_gradient_parity(lbtr, shape, box, prec):
    w = inputs.random_problem(shape, 201, sigma=0.3, box=box)
    dt = torch.float64 if prec == "fp64" else torch.float32
    phi_t = torch.tensor(w.phi0, dtype=dt, device=DEV)
    phi_in = phi_t.double().cpu().numpy()
    ctx = _ctx(lbtr, w, lbtr.LB_FP64 if prec == "fp64" else lbtr.LB_MIXED)
    g = torch.empty_like(phi_t)
    e, gmax = lbtr.lb_energy_grad(ctx, phi_t, g)
    p = olb.Problem.from_workload(w)
    e_ref = olb.energy(p, phi_in)
    g_ref = olb.gradient(p, phi_in)
    assert abs(e - e_ref) / abs(e_ref) < (1e-12 if prec == "fp64" else 1e-6)
    assert _rel(g.double().cpu().numpy(), g_ref) < (1e-10 if prec == "fp64" else 2e-5)
    assert abs(gmax - np.max(np.abs(g_ref))) <= (1e-10 if prec == "fp64" else 2e-5) * np.max(np.abs(g_ref))


def test_energy_closed_form_lamellar(lbtr):
    # Table 2 LAM on 16^3: E = (Lambda_q + tau) A^2 + A^4 / 4 with Lambda_q = 1/4, A = 0.3
    w = inputs.table2_phase("LAM", 16)
    ctx = _ctx(lbtr, w, lbtr.LB_FP64)
    phi = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
    e, _ = lbtr.lb_energy_grad(ctx, phi)
    assert abs(e - (-0.006975)) < 1e-14


def test_energy_rejects_nonzero_mean(lbtr):
    w = inputs.random_problem((16, 16), 3)
    ctx = _ctx(lbtr, w, lbtr.LB_FP64)
    phi = torch.tensor(w.phi0 + 0.01, dtype=torch.float64, device=DEV)
    with pytest.raises(lbtr.LBError) as e:
        lbtr.lb_energy_grad(ctx, phi)
    assert e.value.status == 2


def test_energy_rejects_nan(lbtr):
    w = inputs.random_problem((16, 16), 3)
    ctx = _ctx(lbtr, w, lbtr.LB_FP64)
    a = w.phi0.copy()
    a[3, 4] = np.nan
    phi = torch.tensor(a, dtype=torch.float64, device=DEV)
    with pytest.raises(lbtr.LBError) as e:
        lbtr.lb_energy_grad(ctx, phi)
    assert e.value.status == 3


SUB_CASES = [
    # shape, box, sigma, tau, gamma, r, eps_sub, max_iter
    ((16, 16), (2 * math.pi, 2 * math.pi), 0.05, -0.2, 0.3, 0.05, 1e-10, 4000),
    ((16, 16), (2 * math.pi, 2 * math.pi), 0.05, -0.2, 0.3, 0.02, 1e-10, 4000),
    ((8, 8), None, 0.8, -0.2, 0.3, 1.0, 1e-10, 4000),
    ((8, 8, 8), (4.0, 5.0, 6.0), 0.3, -0.2, 0.3, 0.1, 1e-10, 3000),
    ((64, 64), None, 0.1, -0.15, 0.25, 1.0, 1e-11, 600),
]


@pytest.mark.parametrize("case", SUB_CASES)
def test_subproblem_parity_fp64(lbtr, case):
    shape, box, sig, tau, gam, r, eps, mi = case
    w = inputs.random_problem(shape, 301, sigma=sig, tau=tau, gamma=gam, box=box)
    p = olb.Problem.from_workload(w)
    g_ref = olb.gradient(p, w.phi0)
    ref = osp.imex_subproblem(p, w.phi0, g_ref, r, eta=0.1, eps_sub=eps, max_iter=mi)
    ctx = _ctx(lbtr, w, lbtr.LB_FP64)
    phi = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
    g = torch.tensor(g_ref, dtype=torch.float64, device=DEV)
    d = torch.empty_like(phi)
    opts = lbtr.default_sub_opts()
    opts.eps_sub = eps
    opts.max_iter = mi
    info = lbtr.lb_tr_subproblem(ctx, phi, g, r, d, opts=opts, raise_on_noconv=False)
    assert info["converged"] == ref["converged"]
    assert abs(info["iterations"] - ref["iterations"]) <= 1
    dd = d.cpu().numpy()
    assert _rel(dd, ref["d"]) < 1e-8
    assert abs(info["lambda"] - ref["lambda"]) <= 1e-8 * max(1.0, ref["lambda"])
    assert olb.norm(dd) <= r * (1 + 1e-12)
    f_ref = osp.model_value(p, w.phi0, g_ref, ref["d"])
    assert abs(info["model_value"] - f_ref) <= 1e-10 * abs(f_ref)


@pytest.mark.parametrize("case", SUB_CASES[:4])
def test_subproblem_parity_mixed(lbtr, case):
    shape, box, sig, tau, gam, r, eps, mi = case
    w = inputs.random_problem(shape, 301, sigma=sig, tau=tau, gamma=gam, box=box)
    p = olb.Problem.from_workload(w)
    phi32 = torch.tensor(w.phi0, dtype=torch.float32, device=DEV)
    phi_in = phi32.double().cpu().numpy()
    g_ref = olb.gradient(p, phi_in)
    g32 = torch.tensor(g_ref, dtype=torch.float32, device=DEV)
    ref = osp.imex_subproblem(p, phi_in, g32.double().cpu().numpy(), r, eta=0.1, eps_sub=1e-12, max_iter=20000)
    ctx = _ctx(lbtr, w, lbtr.LB_MIXED)
    d = torch.empty_like(phi32)
    opts = lbtr.default_sub_opts()
    opts.eps_sub = 0.0
    opts.rel_tol = 1e-5
    opts.max_iter = 20000
    info = lbtr.lb_tr_subproblem(ctx, phi32, g32, r, d, opts=opts)
    assert info["converged"]
    dd = d.double().cpu().numpy()
    # The float iteration stops at a residual of 1e-5 ||g||; the distance to the exact
    # minimiser is then bounded by that residual over sigma_min(H + lambda I).
    hc, u = osp.dense_hessian(p, phi_in)
    s1 = float(np.linalg.eigvalsh(hc)[0])
    gap = s1 + ref["lambda"]
    gn = olb.norm(g_ref)
    bound = 3.0 * opts.rel_tol * gn / max(gap, 1e-300) + 1e-5 * olb.norm(ref["d"])
    assert olb.norm(dd - ref["d"]) <= bound
    assert olb.norm(dd) <= r * (1 + 1e-5)
    # the model value, which is what the trust-region step needs, is quadratic in that error
    f_ref = osp.model_value(p, phi_in, g_ref, ref["d"])
    f_gpu = osp.model_value(p, phi_in, g_ref, dd)
    # no feasible point beats the exact minimiser: scale d back into the ball first
    # (float rounding can leave ||d|| a few ulps above r)
    d_in = dd * min(1.0, r / olb.norm(dd))
    assert osp.model_value(p, phi_in, g_ref, d_in) >= f_ref - 1e-9 * abs(f_ref)
    assert abs(f_gpu - f_ref) <= 1e-5 * abs(f_ref)
    assert abs(info["model_value"] - f_gpu) <= 1e-5 * abs(f_ref)



@pytest.fixture(scope="module")
def scale256():
    # the 256^3 scale workload; phi and v are float32-representable with zero mean so that
    # one oracle evaluation serves both precisions
    w = inputs.config_3d_scale(256)
    phi = inputs.remove_mean(w.phi0.astype(np.float32).astype(np.float64))
    v = inputs.gaussian_field(w.shape, 1.0, 104).astype(np.float32).astype(np.float64)
    p = olb.Problem.from_workload(w)
    return (w, phi, v, olb.hessvec(p, phi, v - v.mean()), olb.gradient(p, phi), olb.energy(p, phi))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_hessvec_and_gradient_parity_256cubed(lbtr, scale256, prec):
    # 3D grids above 128^3 take the register row kernels and the persistent line passes
    w, phi, v, hv_ref, g_ref, e_ref = scale256
    dt = torch.float64 if prec == "fp64" else torch.float32
    phi_t = torch.tensor(phi, dtype=dt, device=DEV)
    v_t = torch.tensor(v, dtype=dt, device=DEV)
    ctx = _ctx(lbtr, w, lbtr.LB_FP64 if prec == "fp64" else lbtr.LB_MIXED)
    hv = torch.empty_like(v_t)
    lbtr.lb_hessvec(ctx, phi_t, v_t, hv)
    g = torch.empty_like(phi_t)
    e, _ = lbtr.lb_energy_grad(ctx, phi_t, g)
    torch.cuda.synchronize()
    fp64 = prec == "fp64"
    assert _rel(hv.double().cpu().numpy(), hv_ref) < (1e-12 if fp64 else 2e-5)
    assert _rel(g.double().cpu().numpy(), g_ref) < (1e-10 if fp64 else 2e-5)
    assert abs(e - e_ref) <= (1e-12 if fp64 else 1e-6) * abs(e_ref)
