"""The C-ABI library builds for sm_103a, loads, and exports every declared entry point."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbtr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_03933_gb300 import build, lbtr
    build.build(force=False)
    return lbtr.load()


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for n in ("lb_energy_grad", "lb_hessvec", "lb_tr_subproblem", "lb_lambda_min", "lb_imex_tr_solve"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2603_03933_gb300 import lbtr
    bound = {n for n, _, _ in lbtr.SIGNATURES}
    assert set(declared_functions()) == bound


def test_default_options_match_the_paper(lib):
    from paper_2603_03933_gb300 import lbtr
    o = lbtr.default_tr_opts()
    assert (o.gamma_c, o.gamma_e, o.gamma_lam, o.theta) == (0.5, 2.0, 1.5, 1e-4)
    assert (o.mu_lo, o.mu_hi, o.mu0, o.r0, o.nu0, o.eps) == (1.0, 1e5, 1.0, 1.0, 5.0, 1e-10)
    assert (o.sub.eta, o.sub.eps_sub) == (0.1, 1e-13)


def test_default_first_order_options(lib):
    from paper_2603_03933_gb300 import lbtr
    o = lbtr.default_sis_opts()
    assert (o.dt, o.eps, o.max_steps, o.check_every) == (1.0, 1e-8, 10000, 10)


def test_create_rejects_bad_sizes_without_a_gpu(lib):
    # argument validation happens before any CUDA call
    from paper_2603_03933_gb300 import lbtr
    for dim, n in ((4, 64), (2, 48), (3, 512), (2, 4)):
        with pytest.raises(lbtr.LBError) as e:
            lbtr.lb_create(dim, n, (1.0, 1.0, 1.0), 1.0, -0.1, 0.2)
        assert e.value.status == 8
    with pytest.raises(lbtr.LBError) as e:
        lbtr.lb_create(2, 64, (0.0, 1.0), 1.0, -0.1, 0.2)
    assert e.value.status == 1


def test_batch_solve_binding_checks_fields_before_the_call():
    # host-side marshalling errors are raised before anything reaches the library
    torch = pytest.importorskip("torch")
    from paper_2603_03933_gb300 import lbtr
    b = lbtr.Batch(None, [(2, 16), (2, 16)], lbtr.LB_FP64)
    with pytest.raises(ValueError):
        lbtr.lb_batch_tr_solve(b, [torch.zeros(256, dtype=torch.float64)])
    with pytest.raises(ValueError):      # host tensors are not device fields
        lbtr.lb_batch_tr_solve(b, [torch.zeros(256, dtype=torch.float64)] * 2)
