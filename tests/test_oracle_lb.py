"""Pins for the oracle energy, gradient and Hessian-vector product (paper §2).

Each check comes from outside the oracle's own formulas: closed forms, the paper's
Fourier-space convolution sums evaluated by enumeration, exact finite-difference
identities of polynomials, and the structure H = D + T at psi = 0.
"""
import math

import numpy as np
import pytest

from oracle import lb
from oracle.subproblem import dense_hessian
from paper_2603_03933_gb300 import inputs


def lamellar_closed_form(lam_q, tau, amp):
    # psi = 2A cos(q.x): <psi^2> = 2A^2, <psi^3> = 0, <psi^4> = 6A^4, G = Lambda_q A^2
    return (lam_q + tau) * amp ** 2 + amp ** 4 / 4.0


@pytest.mark.parametrize("tau,gamma,expect", [(-0.35, 0.7, -0.006975),
                                                (-0.001, 0.4, 0.024435),
                                                (-0.09, 0.34, 0.016425)])
@pytest.mark.parametrize("m", [8, 16])
def test_lamellar_energy_closed_form(tau, gamma, expect, m):
    # Table 2 LAM: psi_hat = 0.3 at k = +-(1,0,0), B = I/sqrt(2) -> |Bk|^2 = 1/2, Lambda = 1/4
    w = inputs.table2_phase("LAM", m)
    p = lb.Problem(w.shape, w.box, 1.0, tau, gamma)
    e = lb.energy(p, w.phi0)
    assert abs(e - lamellar_closed_form(0.25, tau, 0.3)) < 1e-15
    assert abs(e - expect) < 1e-15


@pytest.mark.parametrize("xi", [1.0, 1.7])
def test_lamellar_closed_form_rectangular_box_and_xi(xi):
    # single mode along the short axis of a rectangular 2D box
    shape, box = (16, 32), (3.0, 11.0)
    amp = 0.21
    coeffs = {(1, 0): amp, (-1, 0): amp}
    psi = inputs.exp_field(shape, coeffs)
    p = lb.Problem(shape, box, xi, -0.2, 0.5)
    q2 = (2 * math.pi / box[0]) ** 2
    expect = lamellar_closed_form(xi ** 2 * (1 - q2) ** 2, -0.2, amp)
    assert abs(lb.energy(p, psi) - expect) < 1e-14


@pytest.mark.parametrize("phase", ["HEX"])
def test_multimode_energy_matches_convolution_sums(phase):
    # eq. interaction_bulk_energy evaluated literally over the sparse support
    w = inputs.table2_phase(phase, 16)
    p = lb.Problem.from_workload(w)
    coeffs = {(k[2], k[1], k[0]): 0.3 for k in inputs.HEX_XI}
    e_grid = lb.energy(p, w.phi0)
    e_sum = lb.energy_from_coefficients(p, coeffs)
    assert abs(e_grid - e_sum) < 1e-14
    # the cubic (gamma) term is active for HEX: triads k1+k2+k3 = 0 exist
    p0 = lb.Problem(p.shape, p.box, p.xi, p.tau, 0.0)
    assert abs(lb.energy(p, w.phi0) - lb.energy(p0, w.phi0)) > 1e-3


def test_bcc_energy_matches_convolution_sums():
    w = inputs.config_3d_bcc(16)
    phi = inputs.remove_mean(inputs.cosine_field(w.shape, inputs.BCC110_INDEX, 0.1))
    p = lb.Problem.from_workload(w)
    e_sum = lb.energy_from_coefficients(p, {k: 0.1 for k in inputs.BCC110_INDEX})
    assert abs(lb.energy(p, phi) - e_sum) < 1e-14
    assert abs(e_sum - (-0.00535)) < 1e-6


def _richardson_slope(fun, h):
    d1 = (fun(h) - fun(-h)) / (2 * h)
    d2 = (fun(2 * h) - fun(-2 * h)) / (4 * h)
    return (4 * d1 - d2) / 3


@pytest.mark.parametrize("shape,box", [((16, 16), None), ((8, 16), (5.0, 9.0)),
                                       ((8, 8, 8), None), ((4, 8, 16), (3.0, 5.0, 7.0))])
def test_gradient_is_exact_derivative_of_energy(shape, box):
    # E(psi + t v) is a quartic polynomial in t, so the Richardson combination of two
    # central differences is exact up to rounding.
    w = inputs.random_problem(shape, 11, sigma=0.4, box=box)
    p = lb.Problem.from_workload(w)
    v = inputs.gaussian_field(shape, 1.0, 12)
    g = lb.gradient(p, w.phi0)
    slope = _richardson_slope(lambda t: lb.energy(p, w.phi0 + t * v), 0.05)
    assert abs(slope - lb.inner(g, v)) <= 1e-10 * max(1.0, abs(slope))
    assert abs(np.mean(g)) < 1e-14 * max(1.0, np.max(np.abs(g)))


@pytest.mark.parametrize("shape,box", [((16, 16), None), ((8, 8, 8), (4.0, 6.0, 5.0))])
def test_hessvec_is_exact_derivative_of_gradient(shape, box):
    # g(psi + t v) is a cubic polynomial in t: Richardson central differences are exact.
    w = inputs.random_problem(shape, 21, sigma=0.4, box=box)
    p = lb.Problem.from_workload(w)
    v = inputs.gaussian_field(shape, 1.0, 22)
    hv = lb.hessvec(p, w.phi0, v)
    fd = _richardson_slope(lambda t: lb.gradient(p, w.phi0 + t * v), 0.05)
    assert np.max(np.abs(fd - hv)) <= 1e-9 * np.max(np.abs(hv))
    u = inputs.gaussian_field(shape, 1.0, 23)
    # symmetry <u, Hv> = <Hu, v>
    assert abs(lb.inner(u, hv) - lb.inner(lb.hessvec(p, w.phi0, u), v)) < 1e-10 * np.max(np.abs(hv))
    assert abs(np.mean(hv)) < 1e-13 * np.max(np.abs(hv))


def test_hessian_at_zero_field_is_lambda_plus_tau():
    # psi = 0: F'' = tau, so H = D + tau I on zero-mean fields; eigenvalues Lambda_k + tau, k != 0
    shape, box = (8, 8), (7.0, 7.0)
    p = lb.Problem(shape, box, 1.3, -0.17, 0.4)
    hc, _ = dense_hessian(p, np.zeros(shape))
    got = np.sort(np.linalg.eigvalsh(hc))
    k = np.fft.fftfreq(8, 1.0 / 8)
    kk = (2 * np.pi / 7.0) ** 2 * (k[:, None] ** 2 + k[None, :] ** 2)
    expect = np.sort((1.3 ** 2 * (1 - kk) ** 2 - 0.17).ravel()[1:])
    assert np.allclose(got, expect, atol=1e-11 * np.max(np.abs(expect)))


def test_t_and_d_split_sum_to_hessian():
    w = inputs.random_problem((8, 16), 31)
    p = lb.Problem.from_workload(w)
    v = inputs.gaussian_field(w.shape, 1.0, 32)
    h = lb.hessvec(p, w.phi0, v)
    assert np.allclose(lb.apply_D(p, v) + lb.apply_T(p, w.phi0, v), h, atol=1e-12 * np.max(np.abs(h)))


# ---- derivatives with respect to tau, gamma and the box (differentiation workload) ----

def _with(p, **kw):
    d = dict(shape=p.shape, box=p.box, xi=p.xi, tau=p.tau, gamma=p.gamma)
    d.update(kw)
    return lb.Problem(**d)


@pytest.mark.parametrize("shape,box", [((8, 8, 8), (5.0, 6.0, 7.0)), ((16, 16), (9.0, 6.5))])
def test_energy_derivatives_match_central_differences(shape, box):
    # E is linear in tau and gamma, so their central differences are exact up to rounding;
    # along L_a the central difference has an h^2 error (h = 1e-4 L_a relative, tol 1e-6).
    w = inputs.random_problem(shape, 21, sigma=0.4, box=box, tau=-0.15, gamma=0.35)
    p = lb.Problem.from_workload(w)
    dtau, dgamma, dl = lb.energy_derivatives(p, w.phi0)
    h = 1e-3
    fd_tau = (lb.energy(_with(p, tau=p.tau + h), w.phi0) - lb.energy(_with(p, tau=p.tau - h), w.phi0)) / (2 * h)
    fd_gam = (lb.energy(_with(p, gamma=p.gamma + h), w.phi0) - lb.energy(_with(p, gamma=p.gamma - h), w.phi0)) / (2 * h)
    assert abs(fd_tau - dtau) <= 1e-10 * max(1.0, abs(dtau))
    assert abs(fd_gam - dgamma) <= 1e-10 * max(1.0, abs(dgamma))
    for a in range(len(shape)):
        hl = 1e-4 * box[a]
        bp = list(box); bp[a] += hl
        bm = list(box); bm[a] -= hl
        fd = (lb.energy(_with(p, box=tuple(bp)), w.phi0) - lb.energy(_with(p, box=tuple(bm)), w.phi0)) / (2 * hl)
        assert abs(fd - dl[a]) <= 1e-6 * max(abs(dl[a]), 1e-3), (a, fd, dl[a])


def test_box_derivative_of_a_single_mode_closed_form():
    # psi = 2A cos(2 pi k x / L_x): G = Lambda_q A^2 with q = (2 pi k / L_x)^2, so
    # dE/dL_x = A^2 xi^2 2 (1 - q) 2 q / L_x and dE/dL_y = 0
    m, k, amp, xi, lx, ly = 16, 3, 0.2, 1.3, 11.0, 7.0
    x = np.arange(m)
    psi = np.tile(2 * amp * np.cos(2 * np.pi * k * x / m), (m, 1))        # [y][x]
    p = lb.Problem((m, m), (ly, lx), xi, -0.1, 0.2)
    _, _, dl = lb.energy_derivatives(p, psi)
    q = (2 * np.pi * k / lx) ** 2
    assert abs(dl[1] - amp ** 2 * xi ** 2 * 4 * (1 - q) * q / lx) <= 1e-12
    assert abs(dl[0]) <= 1e-14


def test_211_cosines_are_stationary_in_the_box_at_unit_reciprocal_length():
    # the 24 {211} vectors have |k|^2 = 6, so on the cubic box of side 2 pi sqrt(6) every
    # mode sits at |Bk| = 1, where Lambda and dLambda/dL vanish: dE/dL = 0 on every axis,
    # while the differentiation workload's side 2 pi sqrt(8) is not stationary
    m = 8
    psi = inputs.remove_mean(inputs.cosine_field((m, m, m), inputs.CUBIC211_INDEX, 0.1))
    side6, side8 = 2 * math.pi * math.sqrt(6.0), 2 * math.pi * math.sqrt(8.0)
    _, _, dl6 = lb.energy_derivatives(lb.Problem((m,) * 3, (side6,) * 3, 1.0, -0.1, 0.2), psi)
    _, _, dl8 = lb.energy_derivatives(lb.Problem((m,) * 3, (side8,) * 3, 1.0, -0.1, 0.2), psi)
    assert max(abs(v) for v in dl6) <= 1e-14
    assert min(abs(v) for v in dl8) > 1e-4
