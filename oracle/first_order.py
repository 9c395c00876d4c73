"""Oracle for the first-order gradient-flow solver used before IMEX-TR post-processing.

Test infrastructure, not product code (see oracle/__init__.py).  FP64 throughout.

§4 compares IMEX-TR with gradient-flow schemes, among them the semi-implicit scheme
(SIS), and §4 "Robustness to initial conditions" starts IMEX-TR from three states of
a first-order trajectory: its initial point, an intermediate state and the saddle it
converges to.  The paper does not print the scheme; the reading taken here treats the
gradient flow d psi / dt = -g(psi) (g in the <.,.>_N metric of §2) with the same split
as the IMEX subproblem solver of §3.2: the reciprocal diagonal D = Lambda implicitly and
the bulk term F'(psi) explicitly,

    (psi_{n+1} - psi_n) / dt = -(D psi_{n+1} + P F'(psi_n)),

i.e. psi_{n+1} = psi_n - dt (I + dt D)^{-1} g(psi_n), with the k = 0 coefficient held at
zero.  Its fixed points are exactly the zeros of g.
"""
from __future__ import annotations

import numpy as np

from . import fft, lb


def sis_step(p: lb.Problem, psi: np.ndarray, dt: float) -> np.ndarray:
    """One step psi - dt (I + dt Lambda)^{-1} g(psi), k = 0 removed."""
    psi = np.asarray(psi, np.float64)
    g = lb.gradient(p, psi)
    gh = fft.forward(g)
    upd = fft.inverse(gh / (1.0 + dt * lb.lam(p)))
    return psi - dt * lb.project(upd)


def sis_solve(p: lb.Problem, psi: np.ndarray, dt: float, eps: float, max_steps: int):
    """Steps until max_x |g| < eps (tested before each step) or max_steps steps.

    Returns (psi, steps taken, energy, max |g|) at the returned point."""
    psi = np.asarray(psi, np.float64).copy()
    steps = 0
    while True:
        g = lb.gradient(p, psi)
        gmax = float(np.max(np.abs(g)))
        if gmax < eps or steps >= max_steps:
            return psi, steps, lb.energy(p, psi), gmax
        psi = sis_step(p, psi, dt)
        steps += 1
