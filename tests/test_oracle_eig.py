"""Pins for the oracle lambda_min (dense and preconditioned Lanczos)."""
import math

import numpy as np
import pytest

from oracle import eig, lb
from paper_2603_03933_gb300 import inputs


def test_dense_lambda_min_at_zero_field_closed_form():
    # psi = 0: H = D + tau I, lambda_min = tau + min_{k != 0} Lambda_k
    shape, box = (16, 16), (8 * math.pi * 16 / 64,) * 2
    p = lb.Problem(shape, box, 1.0, -0.15, 0.25)
    s, _ = eig.dense_eigs(p, np.zeros(shape), count=3)
    k = np.fft.fftfreq(16, 1 / 16)
    kk = (2 * math.pi / box[0]) ** 2 * (k[:, None] ** 2 + k[None, :] ** 2)
    lam = (1 - kk) ** 2
    lam[0, 0] = np.inf
    # eigh's absolute error scales with the largest eigenvalue (~(|Bk|_max)^4)
    assert abs(s[0] - (-0.15 + lam.min())) < 1e-14 * np.max(lam[np.isfinite(lam)])


@pytest.mark.parametrize("sigma_field,tau", [(0.05, -0.2), (0.6, -0.05)])
def test_lanczos_matches_dense(sigma_field, tau):
    w = inputs.random_problem((16, 16), 8, sigma=sigma_field, tau=tau, gamma=0.3,
                              box=(2 * math.pi, 2 * math.pi))
    p = lb.Problem.from_workload(w)
    s, vecs = eig.dense_eigs(p, w.phi0, count=2)
    out = eig.lanczos_lambda_min(p, w.phi0, k_max=255, tol=1e-9)
    assert out["theta"] >= s[0] - 1e-10          # Rayleigh-Ritz value is an upper bound
    assert abs(out["theta"] - s[0]) <= 1e-8 * max(1.0, abs(s[0]))
    assert np.sign(out["kappa"]) == np.sign(s[0])  # Sylvester inertia of the congruence


def test_lanczos_zero_field_closed_form():
    shape, box = (16, 16), (2 * math.pi, 2 * math.pi)
    p = lb.Problem(shape, box, 1.0, -0.3, 0.2)
    out = eig.lanczos_lambda_min(p, np.zeros(shape), k_max=200, tol=1e-10)
    assert abs(out["theta"] - (-0.3)) < 1e-9
