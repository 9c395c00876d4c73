"""Pins for the oracle FFT (paper §2 discrete Fourier transform)."""
import numpy as np
import pytest

from oracle import fft


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 8, 16, 32])
def test_fft_matches_direct_dft(m):
    rng = np.random.default_rng(m)
    x = rng.standard_normal((3, m)) + 1j * rng.standard_normal((3, m))
    for sign in (-1, 1):
        a = fft.fft_axis(x, 1, sign)
        b = fft.dft_axis(x, 1, sign)
        assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("shape", [(8,), (4, 16), (8, 4, 2), (16, 16)])
def test_fft_matches_numpy_library(shape):
    rng = np.random.default_rng(1)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    for a in range(len(shape)):
        assert np.allclose(fft.fft_axis(x, a, -1), np.fft.fft(x, axis=a), atol=1e-12)
        assert np.allclose(fft.fft_axis(x, a, +1), np.fft.ifft(x, axis=a) * shape[a], atol=1e-12)


def test_paper_normalisation_and_parseval():
    # psi_hat = (1/N) sum psi e^{-ikx}: sum_k |psi_hat|^2 = <psi, psi>_N
    rng = np.random.default_rng(2)
    psi = rng.standard_normal((8, 16))
    ph = fft.forward(psi)
    assert np.isclose(np.sum(np.abs(ph) ** 2), np.mean(psi ** 2), rtol=1e-13)
    assert np.allclose(fft.inverse(ph), psi, atol=1e-13)
    assert np.allclose(fft.forward(psi, direct=True), ph, atol=1e-14)


def test_single_cosine_has_two_coefficients():
    m = 16
    i = np.arange(m)
    psi = np.cos(2 * np.pi * 3 * i / m)
    ph = fft.forward(psi)
    expect = np.zeros(m, complex)
    expect[3] = 0.5
    expect[m - 3] = 0.5
    assert np.allclose(ph, expect, atol=1e-15)


def test_delta_transform_is_flat():
    psi = np.zeros((4, 8))
    psi[0, 0] = 1.0
    assert np.allclose(fft.forward(psi), 1.0 / 32.0, atol=1e-16)


def test_wavenumbers_follow_paper_set():
    # K_M = {k : -M/2 <= k < M/2}
    assert list(fft.wavenumbers(8)) == [0, 1, 2, 3, -4, -3, -2, -1]
    assert list(fft.wavenumbers(5)) == [0, 1, 2, -2, -1]
