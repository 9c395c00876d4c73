"""GPU tests of lb_lambda_min and lb_imex_tr_solve against the oracle (through the C ABI)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import eig as oeig
from oracle import lb as olb
from paper_2603_03933_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_solves.json")


@pytest.fixture(scope="module")
def lbtr():
    from paper_2603_03933_gb300 import build, lbtr as mod
    build.build(force=False)
    mod.load()
    return mod


def _ctx(lbtr, w, prec):
    return lbtr.lb_create_from_array_box(w.shape, w.box, w.xi, w.tau, w.gamma, prec)


@pytest.mark.parametrize("sig,tau", [(0.05, -0.2), (0.6, -0.05)])
def test_lambda_min_matches_dense_fp64(lbtr, sig, tau):
    w = inputs.random_problem((16, 16), 8, sigma=sig, tau=tau, gamma=0.3, box=(2 * math.pi, 2 * math.pi))
    p = olb.Problem.from_workload(w)
    s, _ = oeig.dense_eigs(p, w.phi0, count=2)
    ctx = _ctx(lbtr, w, lbtr.LB_FP64)
    phi = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
    vec = torch.empty_like(phi)
    o = lbtr.default_eig_opts()
    o.max_steps = 255
    o.tol = 1e-7
    info = lbtr.lb_lambda_min(ctx, phi, vec=vec, opts=o, raise_on_noconv=False)
    assert info["lambda_min"] >= s[0] - 1e-9            # Rayleigh-Ritz upper bound
    assert abs(info["lambda_min"] - s[0]) <= 1e-8 * max(1.0, abs(s[0]))
    assert np.sign(info["kappa_min"]) == np.sign(s[0])  # congruence keeps the inertia
    u = vec.cpu().numpy()
    assert abs(olb.norm(u) - 1.0) < 1e-10
    # the returned vector is an approximate eigenvector of the oracle's H
    r = olb.hessvec(p, w.phi0, u) - info["lambda_min"] * u
    assert olb.norm(r) <= max(1e-6, 2 * info["residual"])


def test_lambda_min_zero_field_closed_form(lbtr):
    # phi = 0: H = D + tau I, lambda_min = tau + min_{k != 0} Lambda_k (= tau here: |Bk| = 1 exists)
    shape, box = (32, 32), (2 * math.pi, 2 * math.pi)
    w = inputs.Workload("zero", shape, box, 1.0, -0.3, 0.2, np.zeros(shape))
    ctx = _ctx(lbtr, w, lbtr.LB_FP64)
    phi = torch.zeros(shape, dtype=torch.float64, device=DEV)
    info = lbtr.lb_lambda_min(ctx, phi, raise_on_noconv=False)
    assert abs(info["lambda_min"] - (-0.3)) < 1e-9


@pytest.mark.parametrize("shape,box", [((32, 32), (2 * math.pi, 2 * math.pi)), ((16, 16, 16), (4.0, 5.0, 6.0))])
def test_lambda_min_matches_oracle_lanczos(lbtr, shape, box):
    w = inputs.random_problem(shape, 9, sigma=0.1, tau=-0.1, gamma=0.3, box=box)
    p = olb.Problem.from_workload(w)
    ref = oeig.lanczos_lambda_min(p, w.phi0, k_max=300, tol=1e-8)
    ctx = _ctx(lbtr, w, lbtr.LB_FP64)
    phi = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
    o = lbtr.default_eig_opts()
    o.max_steps = 300
    o.tol = 1e-8
    info = lbtr.lb_lambda_min(ctx, phi, opts=o, raise_on_noconv=False)
    assert abs(info["lambda_min"] - ref["theta"]) <= 1e-7 * max(1.0, abs(ref["theta"]))


def test_lambda_min_mixed_precision(lbtr):
    w = inputs.random_problem((32, 32), 9, sigma=0.1, tau=-0.1, gamma=0.3, box=(2 * math.pi, 2 * math.pi))
    p = olb.Problem.from_workload(w)
    phi32 = torch.tensor(w.phi0, dtype=torch.float32, device=DEV)
    ref = oeig.lanczos_lambda_min(p, phi32.double().cpu().numpy(), k_max=300, tol=1e-8)
    ctx = _ctx(lbtr, w, lbtr.LB_MIXED)
    o = lbtr.default_eig_opts()
    o.tol = 1e-4
    info = lbtr.lb_lambda_min(ctx, phi32, opts=o, raise_on_noconv=False)
    assert abs(info["lambda_min"] - ref["theta"]) <= 1e-5 * max(1.0, abs(ref["theta"]))
    assert np.sign(info["kappa_min"]) == np.sign(ref["theta"])


def test_barrier_timeout_returns_status_without_hang(lbtr):
    # A grid-barrier budget of one cycle makes every waiting block give up at once; the
    # call must return LB_ERR_TIMEOUT and the context must stay usable afterwards.  The
    # grid is 16^3 so that the fused iteration spans several CTAs (a one-CTA grid never
    # waits at its barriers).
    w = inputs.random_problem((16, 16, 16), 3, sigma=0.3)
    p = olb.Problem.from_workload(w)
    ctx = _ctx(lbtr, w, lbtr.LB_FP64)
    phi = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
    g = torch.tensor(olb.gradient(p, w.phi0), dtype=torch.float64, device=DEV)
    d = torch.empty_like(phi)
    lbtr.lb_set_barrier_budget(ctx, 1)
    with pytest.raises(lbtr.LBError) as e:
        lbtr.lb_tr_subproblem(ctx, phi, g, 0.05, d)
    assert e.value.status == 5
    lbtr.lb_set_barrier_budget(ctx, 0)
    info = lbtr.lb_tr_subproblem(ctx, phi, g, 0.05, d)
    assert info["converged"]


def _golden(name):
    if not os.path.exists(GOLDEN):
        pytest.skip("oracle golden solves not generated")
    with open(GOLDEN) as f:
        data = json.load(f)
    if name not in data:
        pytest.skip(f"golden {name} missing")
    return data[name]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_tr_solve_small_matches_oracle(lbtr, prec):
    ref = _golden("2d_16_nonconvex")
    w = inputs.random_problem((16, 16), 5, sigma=0.05, tau=-0.2, gamma=0.3, box=(2 * math.pi, 2 * math.pi))
    p = olb.Problem.from_workload(w)
    ctx = _ctx(lbtr, w, lbtr.LB_FP64 if prec == "fp64" else lbtr.LB_MIXED)
    phi = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
    o = lbtr.default_tr_opts()
    o.eps = 1e-8
    o.max_outer = 200
    info = lbtr.lb_imex_tr_solve(ctx, phi, opts=o)
    v = phi.cpu().numpy()
    # checks made by the oracle on the returned field
    assert np.max(np.abs(olb.gradient(p, v))) < 1e-8
    s, _ = oeig.dense_eigs(p, v, count=1)
    assert s[0] >= -1e-8                                  # second-order stationary
    assert abs(info["energy"] - olb.energy(p, v)) < 1e-12
    assert abs(info["energy"] - ref["energy"]) < 1e-8     # the oracle's own solve


def test_tr_solve_2d_64_plain_matches_oracle(lbtr):
    # 2D LB, 64^2, box 8 pi, tau -0.15, gamma 0.25, phi0 ~ N(0, 0.1^2): ||g||_inf < 1e-8 and
    # lambda_min >= -1e-8; energy within 1e-8 of the oracle's own solve
    ref = _golden("2d_64_plain")
    w = inputs.config_2d_plain(64)
    p = olb.Problem.from_workload(w)
    ctx = _ctx(lbtr, w, lbtr.LB_FP64)
    phi = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
    o = lbtr.default_tr_opts()
    o.eps = 1e-8
    o.tol2 = 1e-8
    o.max_outer = 300
    info = lbtr.lb_imex_tr_solve(ctx, phi, opts=o)
    v = phi.cpu().numpy()
    assert np.max(np.abs(olb.gradient(p, v))) < 1e-8
    assert info["lambda_min"] is not None and info["lambda_min"] >= -1e-8
    assert abs(info["energy"] - olb.energy(p, v)) < 1e-12
    assert abs(info["energy"] - ref["energy"]) < 1e-8


def test_tr_solve_3d_bcc_mixed_matches_fp64(lbtr):
    # 3D BCC workload on 32^3 (the 64^3 box at half resolution keeps the test short):
    # the mixed path (float inner iterations) reaches the FP64 path's energy to 1e-8
    w = inputs.config_3d_bcc(32)
    p = olb.Problem.from_workload(w)
    out = {}
    for prec in ("fp64", "mixed"):
        ctx = _ctx(lbtr, w, lbtr.LB_FP64 if prec == "fp64" else lbtr.LB_MIXED)
        phi = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
        o = lbtr.default_tr_opts()
        o.eps = 1e-8
        o.max_outer = 300
        o.sub.rel_tol = 1e-6
        info = lbtr.lb_imex_tr_solve(ctx, phi, opts=o)
        v = phi.cpu().numpy()
        assert np.max(np.abs(olb.gradient(p, v))) < 1e-8
        assert abs(info["energy"] - olb.energy(p, v)) < 1e-12
        out[prec] = info
    assert abs(out["mixed"]["energy"] - out["fp64"]["energy"]) < 1e-8
    assert (out["mixed"]["lambda_min"] >= -1e-8) == (out["fp64"]["lambda_min"] >= -1e-8)


def test_tr_checkpoint_resume_repeats_the_solve(lbtr, tmp_path):
    # a solve cut after four outer iterations (checkpoints after the 2nd and 4th) and resumed
    # from its files ends where the uninterrupted solve ends, iteration for iteration
    w = inputs.random_problem((16, 16), 5, sigma=0.05, tau=-0.2, gamma=0.3, box=(2 * math.pi, 2 * math.pi))
    ctx = _ctx(lbtr, w, lbtr.LB_FP64)
    o = lbtr.default_tr_opts()
    o.eps, o.max_outer = 1e-8, 200
    straight = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
    ref = lbtr.lb_imex_tr_solve(ctx, straight, opts=o)
    assert ref["outer"] > 4
    path = str(tmp_path / "tr").encode()
    o.checkpoint_path, o.checkpoint_every, o.max_outer = path, 2, 4
    phi = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
    cut = lbtr.lb_imex_tr_solve(ctx, phi, opts=o, raise_on_noconv=False)
    assert cut["status"] == 4 and cut["outer"] == 4
    saved = np.load(path.decode() + ".npy")
    assert np.array_equal(saved, phi.cpu().numpy())
    o.resume, o.max_outer = 1, 200
    resumed = torch.zeros_like(phi)                      # the start comes from the files
    info = lbtr.lb_imex_tr_solve(ctx, resumed, opts=o)
    assert info["outer"] == ref["outer"] and info["inner"] == ref["inner"]
    assert (info["accepted"], info["contracted"], info["shrunk"]) == (ref["accepted"], ref["contracted"], ref["shrunk"])
    assert np.max(np.abs(resumed.cpu().numpy() - straight.cpu().numpy())) <= 1e-13
    assert abs(info["energy"] - ref["energy"]) <= 1e-14


def test_tr_resume_refuses_a_checkpoint_of_another_grid(lbtr, tmp_path):
    w = inputs.random_problem((16, 16), 6, sigma=0.05, tau=-0.2, gamma=0.3)
    ctx = _ctx(lbtr, w, lbtr.LB_FP64)
    path = str(tmp_path / "other")
    np.save(path + ".npy", np.zeros((32, 32)))
    with open(path + ".json", "w") as f:
        f.write('{"format": 1, "dim": 2, "n": 32, "j": 1, "r": 1, "nu": 5, "mu": 1, "rho_prev": 0, '
                '"have_rho": 0, "random_next": 0, "rstream": 1, "accepted": 0, "contracted": 0, "shrunk": 0, '
                '"randomized": 0, "inner": 0, "g1_min": NaN}\n')
    o = lbtr.default_tr_opts()
    o.checkpoint_path, o.resume = path.encode(), 1
    phi = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
    with pytest.raises(lbtr.LBError) as e:
        lbtr.lb_imex_tr_solve(ctx, phi, opts=o)
    assert e.value.status == 1


def test_tr_resume_refuses_a_checkpoint_of_another_problem(lbtr, tmp_path):
    # a checkpoint written for tau = -0.2 is not resumed by a context built for tau = -0.1
    # on the same grid and box
    w = inputs.random_problem((16, 16), 5, sigma=0.05, tau=-0.2, gamma=0.3, box=(2 * math.pi, 2 * math.pi))
    ctx = _ctx(lbtr, w, lbtr.LB_FP64)
    o = lbtr.default_tr_opts()
    path = str(tmp_path / "tr").encode()
    o.eps, o.checkpoint_path, o.checkpoint_every, o.max_outer = 1e-8, path, 1, 2
    phi = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
    lbtr.lb_imex_tr_solve(ctx, phi, opts=o, raise_on_noconv=False)
    other = inputs.random_problem((16, 16), 5, sigma=0.05, tau=-0.1, gamma=0.3, box=(2 * math.pi, 2 * math.pi))
    ctx2 = _ctx(lbtr, other, lbtr.LB_FP64)
    o.resume, o.max_outer = 1, 200
    with pytest.raises(lbtr.LBError) as e:
        lbtr.lb_imex_tr_solve(ctx2, torch.zeros_like(phi), opts=o)
    assert e.value.status == 1 and "tau" in str(e.value)
    # the matching context resumes
    info = lbtr.lb_imex_tr_solve(ctx, torch.zeros_like(phi), opts=o)
    assert info["status"] == 0


def _trace_lines(err_text):
    out = []
    for line in err_text.splitlines():
        line = line.strip()
        if line.startswith("{\"j\""):
            out.append(json.loads(line))
    return out


@pytest.mark.parametrize("params,steps", [(dict(r0=5.0, nu0=5.0), ["contract", "accept"]),
                                          (dict(r0=0.01, mu0=1e4), ["shrink", "accept"]),
                                          (dict(r0=0.01, nu0=0.01), ["accept", "accept"])])
def test_tr_trajectory_matches_oracle_branch_by_branch(lbtr, capfd, monkeypatch, params, steps):
    # Algorithm 1's first two outer iterations on an 8x8 problem, GPU (FP64, per-iteration
    # trace) against the oracle: the same branch each time, and r, nu, mu, lambda, ||s||, rho
    # of every iteration (inner solves to 1e-12, CONTRACT solves to 1e-10 relative)
    from oracle import trust_region as otr
    w = inputs.random_problem((8, 8), 11, sigma=0.3, tau=-0.2, gamma=0.3, box=(2 * math.pi, 2 * math.pi))
    p = olb.Problem.from_workload(w)
    log = []
    otr.imex_tr(p, w.phi0, params=params, max_outer=2, eps=1e-12, second_order=False, max_inner=20000,
                eps_sub=1e-12, log=log)
    assert [e["step"] for e in log] == steps
    ctx = _ctx(lbtr, w, lbtr.LB_FP64)
    o = lbtr.default_tr_opts()
    for k, v in params.items():
        setattr(o, k, v)
    o.eps, o.max_outer, o.second_order = 1e-12, 2, 0
    o.sub.eps_sub, o.sub.max_iter = 1e-12, 20000
    monkeypatch.setenv("LBTR_TRACE", "1")
    phi = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
    capfd.readouterr()
    lbtr.lb_imex_tr_solve(ctx, phi, opts=o, raise_on_noconv=False)
    torch.cuda.synchronize()
    tr = _trace_lines(capfd.readouterr().err)
    assert len(tr) == 2
    prev = (0, 0, 0)
    for e, g in zip(log, tr):
        cnt = (g["acc"], g["con"], g["shr"])
        kind = ["accept", "contract", "shrink"][[c - q for c, q in zip(cnt, prev)].index(1)]
        prev = cnt
        assert kind == e["step"]
        for key, gk in (("r", "r"), ("nu", "nu"), ("mu", "mu"), ("lambda", "lambda"), ("snorm", "snorm"),
                        ("rho", "rho")):
            # the trace prints 6 significant digits
            assert abs(g[gk] - e[key]) <= 1e-5 * max(abs(e[key]), 1e-12) + 1e-12, (key, g[gk], e[key])


def _c2_opts(lbtr, case):
    o = lbtr.default_tr_opts()
    o.eps, o.tol2, o.max_outer, o.second_order = 1e-8, 1e-8, 200, 1
    if case == "3d_64_bcc_rel":
        o.sub.eps_sub, o.sub.rel_tol, o.sub.max_iter = 0.0, 1e-4, 2000
    else:
        o.sub.eps_sub, o.sub.rel_tol, o.sub.max_iter = 1e-10, 0.0, 5000
    return o


@pytest.mark.parametrize("case,prec", [("3d_64_bcc_rel", "fp64"), ("3d_64_bcc_rel", "mixed"),
                                       ("3d_64_bcc_abs", "fp64")])
def test_tr_solve_3d_64_bcc_matches_oracle(lbtr, case, prec):
    # the 64^3 BCC workload solved to ||g||_inf < 1e-8 with the second-order test, with the
    # inner settings of the oracle's own solve: the energy within 1e-8 of the oracle's and the
    # same sign of lambda_min (|lambda_min| <= 1e-8 counts as >= 0)
    ref = _golden(case)
    w = inputs.config_3d_bcc(64)
    p = olb.Problem.from_workload(w)
    ctx = _ctx(lbtr, w, lbtr.LB_FP64 if prec == "fp64" else lbtr.LB_MIXED)
    phi = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
    info = lbtr.lb_imex_tr_solve(ctx, phi, opts=_c2_opts(lbtr, case))
    v = phi.cpu().numpy()
    assert np.max(np.abs(olb.gradient(p, v))) < 1e-8
    assert abs(info["energy"] - olb.energy(p, v)) < 1e-12
    assert abs(info["energy"] - ref["energy"]) < 1e-8
    assert (info["lambda_min"] >= -1e-8) == (ref["lambda_min"] >= -1e-8)
