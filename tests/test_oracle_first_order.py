"""Pins of the first-order (semi-implicit gradient-flow) oracle.

* One step on a single cosine mode against the closed form from the power-reduction
  identities cos^2 = (1 + cos 2t) / 2 and cos^3 = (3 cos t + cos 3t) / 4: the step
  keeps the modes k0, 2 k0 and 3 k0 only, each divided by its own 1 + dt Lambda.
* Energy decreases monotonically along a trajectory from a random field (dt small
  against 1 / max |F''|).
* A fixed point is a zero of g: a converged run has max |g| below the tolerance and a
  further step moves it by at most dt times that.
"""
import math

import numpy as np

from oracle import first_order as fo
from oracle import lb
from paper_2603_03933_gb300 import inputs


def test_single_mode_step_matches_closed_form():
    m, k0, a, dt = 32, 2, 0.4, 0.7
    length = 2 * math.pi * 1.7
    p = lb.Problem((m, m), (length * 1.3, length), 1.0, -0.2, 0.35)
    x = np.arange(m) * length / m
    th = 2 * math.pi * k0 * x / length
    psi = np.broadcast_to(a * np.cos(th), (m, m)).copy()
    out = fo.sis_step(p, psi, dt)

    def lam_k(k):      # Lambda at wavevector (0, k) on the last (x) axis
        return (1.0 - (2 * math.pi * k / length) ** 2) ** 2

    # projected F'(psi) = (tau a + a^3/8) cos t - (gamma a^2 / 4) cos 2t + (a^3 / 24) cos 3t
    g1 = lam_k(k0) * a + p.tau * a + a ** 3 / 8
    g2 = -p.gamma * a * a / 4
    g3 = a ** 3 / 24
    want = (a - dt * g1 / (1 + dt * lam_k(k0))) * np.cos(th) \
        - dt * g2 / (1 + dt * lam_k(2 * k0)) * np.cos(2 * th) \
        - dt * g3 / (1 + dt * lam_k(3 * k0)) * np.cos(3 * th)
    assert np.max(np.abs(out - want[None, :])) < 1e-14


def test_energy_decreases_along_the_trajectory():
    w = inputs.random_problem((24, 24), 41, sigma=0.2, box=(9.0, 7.0), tau=-0.15, gamma=0.25)
    p = lb.Problem.from_workload(w)
    psi = w.phi0
    e = [lb.energy(p, psi)]
    for _ in range(40):
        psi = fo.sis_step(p, psi, 0.5)
        e.append(lb.energy(p, psi))
        assert abs(psi.mean()) < 1e-15
    assert all(b < a for a, b in zip(e, e[1:]))


def test_converged_point_is_a_zero_of_the_gradient():
    w = inputs.random_problem((16, 16), 42, sigma=0.3, box=(8.0, 8.0), tau=-0.2, gamma=0.3)
    p = lb.Problem.from_workload(w)
    psi, steps, e, gmax = fo.sis_solve(p, w.phi0, 1.0, 1e-9, 20000)
    assert gmax < 1e-9 and steps > 0
    assert e < lb.energy(p, w.phi0)
    assert np.max(np.abs(fo.sis_step(p, psi, 1.0) - psi)) <= 1e-9
