"""Oracle FFT: the discrete Fourier transform of the paper's §2, written out plainly.

Test infrastructure, not product code (see oracle/__init__.py).

The paper defines the discrete Fourier coefficients of a grid function as
    psi_hat(k) = <psi, e^{i(Bk)^T x}>_N = (1/N) sum_x psi(x) e^{-i (Bk)^T x}
(§2, the formula closing the discrete-orthogonality paragraph) and the expansion
    psi(x) = sum_k psi_hat(k) e^{i (Bk)^T x}.
On the grid x = A(i/M) with A B^T = 2 pi I the phase (Bk)^T x equals 2 pi k.i / M,
so the forward transform is the plain DFT with sign -1 scaled by 1/N and the inverse
is the unscaled DFT with sign +1.  Array index k in [0, M) stands for the wavenumber
k if k < M/2 and k - M otherwise (the paper's set K_M = {-M/2 <= k < M/2}).

Two independent implementations are kept:
  * dft_axis: the O(M^2) definition, a matrix of exp(sign * 2 pi i j k / M);
  * fft_axis: an iterative radix-2 Cooley-Tukey transform (bit reversal, then
    log2(M) butterfly stages), used for speed on power-of-two lengths.
Tests pin fft_axis against dft_axis and against numpy.fft (a separate library).
"""
from __future__ import annotations

import numpy as np


def dft_axis(x: np.ndarray, axis: int, sign: int) -> np.ndarray:
    """Unscaled DFT along `axis`: y[k] = sum_j x[j] exp(sign * 2 pi i j k / M)."""
    x = np.asarray(x, dtype=np.complex128)
    m = x.shape[axis]
    j = np.arange(m)
    mat = np.exp(sign * 2j * np.pi * np.outer(j, j) / m)
    xm = np.moveaxis(x, axis, -1)
    y = xm @ mat.T          # y[..., k] = sum_j x[..., j] mat[k, j]
    return np.moveaxis(y, -1, axis)


def _bit_reverse_perm(m: int) -> np.ndarray:
    bits = m.bit_length() - 1
    idx = np.arange(m)
    rev = np.zeros(m, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def fft_axis(x: np.ndarray, axis: int, sign: int) -> np.ndarray:
    """Unscaled DFT along `axis` by iterative radix-2 Cooley-Tukey (power-of-two M).

    Other lengths fall back to the O(M^2) definition.
    """
    x = np.asarray(x, dtype=np.complex128)
    m = x.shape[axis]
    if m & (m - 1) != 0:
        return dft_axis(x, axis, sign)
    if m == 1:
        return x.copy()
    xm = np.moveaxis(x, axis, -1)
    lead = xm.shape[:-1]
    y = xm[..., _bit_reverse_perm(m)].reshape(-1, m).copy()
    size = 2
    while size <= m:
        half = size // 2
        w = np.exp(sign * 2j * np.pi * np.arange(half) / size)
        blocks = y.reshape(y.shape[0], m // size, size)
        even = blocks[:, :, :half].copy()
        odd = blocks[:, :, half:] * w
        blocks[:, :, :half] = even + odd
        blocks[:, :, half:] = even - odd
        y = blocks.reshape(y.shape[0], m)
        size *= 2
    y = y.reshape(lead + (m,))
    return np.moveaxis(y, -1, axis)


def forward(psi: np.ndarray, direct: bool = False) -> np.ndarray:
    """psi_hat = (1/N) sum_x psi(x) e^{-i (Bk)^T x} over every axis (paper §2)."""
    out = np.asarray(psi, dtype=np.complex128)
    tr = dft_axis if direct else fft_axis
    for a in range(out.ndim):
        out = tr(out, a, -1)
    return out / out.size


def inverse(psi_hat: np.ndarray, direct: bool = False, real: bool = True) -> np.ndarray:
    """psi(x) = sum_k psi_hat(k) e^{i (Bk)^T x} over every axis (paper §2).

    With real=True the imaginary part, which is rounding noise for a Hermitian
    spectrum, is dropped."""
    out = np.asarray(psi_hat, dtype=np.complex128)
    tr = dft_axis if direct else fft_axis
    for a in range(out.ndim):
        out = tr(out, a, +1)
    return out.real.copy() if real else out


def wavenumbers(m: int) -> np.ndarray:
    """Signed integer wavenumber of each array index: k if k < M/2 else k - M."""
    k = np.arange(m)
    return np.where(k < (m + 1) // 2 if m % 2 else k < m // 2, k, k - m)
