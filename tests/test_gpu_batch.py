"""Batches of independent problems (the phase-diagram sweep) through lb_batch_hessvec.

Every product of the batch must equal the product of the same problem through its own
context (lb_hessvec: the same transforms; the 2D problems run in one persistent launch
whose sums differ from the single-problem kernels' only in summation order), on the
recording call, on a replay of the recorded graph, and after new field pointers force a
new recording; one member of every grid size is also checked against the oracle.  The
tuner's table must be complete and its choice must give the same products.
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


def _members():
    ws = inputs.batched_sweep(12, seed=11, sizes=(16, 32, 64, 128, 256, 512))
    ws.append(inputs.random_problem((32, 32, 32), 12, sigma=0.3, box=(5.0, 6.0, 7.0)))
    ws.append(inputs.random_problem((64, 64, 64), 13, sigma=0.3))
    return ws


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("persistent", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_matches_single_problem_products(lbtr, prec, persistent):
    p = lbtr.LB_FP64 if prec == "fp64" else lbtr.LB_MIXED
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 1e-6
    ws = _members()
    probs = [(w.dim, w.shape[0], list(w.box)[::-1], w.xi, w.tau, w.gamma) for w in ws]
    batch = lbtr.lb_batch_create(probs, p)
    assert len(batch) == len(ws)
    lbtr.lb_batch_set_launch(batch, persistent)
    phis = [torch.tensor(w.phi0, dtype=dt, device=DEV) for w in ws]
    vs = [torch.tensor(inputs.gaussian_field(w.shape, 1.0, 900 + i), dtype=dt, device=DEV) for i, w in enumerate(ws)]
    refs = []
    for w, phi, v in zip(ws, phis, vs):
        c = lbtr.lb_create_from_array_box(w.shape, w.box, w.xi, w.tau, w.gamma, p)
        hv = torch.empty_like(v)
        lbtr.lb_hessvec(c, phi, v, hv)
        refs.append(hv)
    torch.cuda.synchronize()
    for call in range(3):
        # calls 0 and 1 share pointers (record, replay); call 2 uses new outputs (record anew)
        hvs = [torch.full_like(v, float("nan")) for v in vs] if call != 1 else hvs
        if call == 1:
            for h in hvs:
                h.fill_(float("nan"))
        lbtr.lb_batch_hessvec(batch, phis, vs, hvs)
        torch.cuda.synchronize()
        for i, (h, r) in enumerate(zip(hvs, refs)):
            assert _rel(h.double().cpu().numpy(), r.double().cpu().numpy()) <= tol, (call, i)
    # one member of every grid size (the 2D ones run in the persistent launch, the 3D ones
    # as graph branches) against the oracle (parity tolerances)
    first = {}
    for i, w in enumerate(ws):
        first.setdefault(w.shape, i)
    for i in sorted(first.values()):
        w = ws[i]
        pr = olb.Problem.from_workload(w)
        ref = olb.hessvec(pr, phis[i].double().cpu().numpy(), vs[i].double().cpu().numpy())
        assert _rel(hvs[i].double().cpu().numpy(), ref) <= (1e-12 if prec == "fp64" else 2e-5)


def test_batch_rejects_bad_fields(lbtr):
    ws = _members()[:2]
    probs = [(w.dim, w.shape[0], list(w.box)[::-1], w.xi, w.tau, w.gamma) for w in ws]
    batch = lbtr.lb_batch_create(probs, lbtr.LB_FP64)
    f = [torch.zeros(w.shape, dtype=torch.float64, device=DEV) for w in ws]
    with pytest.raises(lbtr.LBError) as e:
        lbtr.lb_batch_hessvec(batch, f, f, f)          # outputs alias inputs
    assert e.value.status == 1


def test_batch_tr_solve_matches_individual_solves(lbtr):
    # eight 2D problems of two sizes across (tau, gamma), solved on four host threads; each
    # must end where the single-problem driver ends (same stop test, same SP-II check)
    ws = [w for w in inputs.batched_sweep(8, seed=11, sizes=(16, 32))]
    probs = [(w.dim, w.shape[0], list(w.box)[::-1], w.xi, w.tau, w.gamma) for w in ws]
    batch = lbtr.lb_batch_create(probs, lbtr.LB_FP64)
    o = lbtr.default_tr_opts()
    o.eps, o.max_outer = 1e-8, 300
    phis = [torch.tensor(w.phi0, dtype=torch.float64, device=DEV) for w in ws]
    infos = lbtr.lb_batch_tr_solve(batch, phis, opts=o, nthreads=4)
    for w, ph, info in zip(ws, phis, infos):
        ctx = lbtr.lb_create_from_array_box(w.shape, w.box, w.xi, w.tau, w.gamma, lbtr.LB_FP64)
        ref = torch.tensor(w.phi0, dtype=torch.float64, device=DEV)
        r = lbtr.lb_imex_tr_solve(ctx, ref, opts=o)
        assert info["status"] == 0 and info["gmax"] < 1e-8
        assert abs(info["energy"] - r["energy"]) <= 1e-9 * max(1.0, abs(r["energy"]))
        p = olb.Problem.from_workload(w)
        x = ph.cpu().numpy()
        assert np.max(np.abs(olb.gradient(p, x))) < 1e-8
        assert abs(olb.energy(p, x) - info["energy"]) <= 1e-12


def test_batch_tr_solve_rejects_aliased_fields(lbtr):
    ws = inputs.batched_sweep(2, seed=12, sizes=(16,))
    probs = [(w.dim, w.shape[0], list(w.box)[::-1], w.xi, w.tau, w.gamma) for w in ws]
    batch = lbtr.lb_batch_create(probs, lbtr.LB_FP64)
    ph = torch.tensor(ws[0].phi0, dtype=torch.float64, device=DEV)
    with pytest.raises(lbtr.LBError):
        lbtr.lb_batch_tr_solve(batch, [ph, ph])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_tune_keeps_products_and_reports_its_table(lbtr, prec):
    p = lbtr.LB_FP64 if prec == "fp64" else lbtr.LB_MIXED
    dt = torch.float64 if prec == "fp64" else torch.float32
    ws = inputs.batched_sweep(24, seed=5, sizes=(64, 128, 256, 512))
    probs = [(w.dim, w.shape[0], list(w.box)[::-1], w.xi, w.tau, w.gamma) for w in ws]
    batch = lbtr.lb_batch_create(probs, p)
    phis = [torch.tensor(w.phi0, dtype=dt, device=DEV) for w in ws]
    vs = [torch.tensor(inputs.gaussian_field(w.shape, 1.0, 700 + i), dtype=dt, device=DEV) for i, w in enumerate(ws)]
    hvs = [torch.empty_like(v) for v in vs]
    lbtr.lb_batch_hessvec(batch, phis, vs, hvs)
    torch.cuda.synchronize()
    before = [h.clone() for h in hvs]
    table = lbtr.lb_batch_tune(batch, phis, vs, hvs, replays=3)
    cands = table["candidates"]
    assert len(cands) >= 3 and cands[0]["strategy"] == "grouped"
    assert any(c["strategy"] == "persistent" for c in cands)
    assert all(c["us"] > 0 and c["row_blocks_per_task"] in (1, 4) for c in cands)
    assert all(c["ctas_per_sm"] >= 1 for c in cands if c["strategy"] == "persistent")
    best = min(range(len(table["candidates"])), key=lambda k: table["candidates"][k]["us"])
    assert table["chosen"] == best
    for h in hvs:
        h.fill_(float("nan"))
    lbtr.lb_batch_hessvec(batch, phis, vs, hvs)           # records anew with the chosen launch
    torch.cuda.synchronize()
    for h, r in zip(hvs, before):
        # the grouped launches and the persistent one sum F''(phi) v in different orders
        assert _rel(h.double().cpu().numpy(), r.double().cpu().numpy()) <= (1e-12 if prec == "fp64" else 1e-6)
    w = ws[-1]
    pr = olb.Problem.from_workload(w)
    ref = olb.hessvec(pr, phis[-1].double().cpu().numpy(), vs[-1].double().cpu().numpy())
    assert _rel(hvs[-1].double().cpu().numpy(), ref) <= (1e-12 if prec == "fp64" else 2e-5)
