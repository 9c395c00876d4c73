"""Pins for the oracle outer loop (paper §3.1, Algorithms 1 and 2)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import eig, lb
from oracle import subproblem as sp
from oracle import trust_region as tr
from paper_2603_03933_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def test_parameters_are_the_papers():
    with open(GOLDEN) as f:
        prm = json.load(f)["algorithm_parameters"]
    for k, v in tr.PAPER_PARAMS.items():
        assert prm[k] == v, k


def test_pcg_matches_dense_solve():
    w = inputs.random_problem((8, 8), 13, sigma=0.5)
    p = lb.Problem.from_workload(w)
    g = lb.gradient(p, w.phi0)
    hc, u = sp.dense_hessian(p, w.phi0)
    shift = 0.7 + max(0.0, -np.linalg.eigvalsh(hc)[0])
    s, it, rel = tr.pcg_shifted(p, w.phi0, g, shift)
    ref = np.linalg.solve(hc + shift * np.eye(hc.shape[0]), -sp.to_coords(u, g))
    assert np.allclose(sp.to_coords(u, s), ref, atol=1e-10 * np.linalg.norm(ref))


def test_exact_energy_drop_matches_direct_difference():
    w = inputs.random_problem((16, 16), 17, sigma=0.3)
    p = lb.Problem.from_workload(w)
    g = lb.gradient(p, w.phi0)
    for scale in (1e-1, 1.0):
        s = scale * inputs.gaussian_field(w.shape, 1.0, 18)
        a = tr.energy_drop(p, w.phi0, g, s)
        b = tr.energy_drop_direct(p, w.phi0, s)
        assert abs(a - b) <= 1e-12 * max(1.0, abs(b))


def test_imex_tr_reaches_second_order_stationary_point():
    # box side 2 pi on 16^2: |Bk| = |k|, tau < 0, started next to the saddle psi = 0
    w = inputs.random_problem((16, 16), 5, sigma=0.05, tau=-0.2, gamma=0.3,
                              box=(math.pi * 2, math.pi * 2))
    p = lb.Problem.from_workload(w)
    log = []
    out = tr.imex_tr(p, w.phi0, eps=1e-8, max_outer=60, max_inner=1000, log=log)
    assert out["status"] == "converged"
    assert out["gmax"] < 1e-8
    s, _ = eig.dense_eigs(p, out["v"], count=1)
    assert s[0] >= -1e-8                       # SP-II (paper §1 definition)
    # accepted steps never raise the energy
    e0 = lb.energy(p, w.phi0)
    es = [e0] + [l["E"] for l in log]
    assert all(b <= a + 1e-14 for a, b in zip(es, es[1:]))
    assert out["E"] < e0
