"""Own discrete Fourier transforms for the oracle (float64 / complex128).

The paper computes the second-order source "with FFTs" (Sec. 2.1, Eq. second-ini)
and goes back and forth between Fourier and configuration space (Sec. 3).
Conventions (a reading: the paper fixes none):
  forward  F[n] = sum_x f[x] exp(-2 pi i n x / N)          (unnormalised)
  inverse  f[x] = (1/N) sum_n F[n] exp(+2 pi i n x / N)
so that a derivative d/dx becomes a multiplication by i k, k = 2 pi n / L.

Power-of-two lengths use an iterative radix-2 decimation-in-time FFT
(bit-reversal permutation, then log2 N butterfly stages) written here.
Other lengths (96, 192) use the plain O(N^2) DFT as a matrix product.
"""
from __future__ import annotations

import numpy as np

__all__ = ["fft_axis", "fftn", "ifftn", "dft_matrix"]


def _bit_reverse_perm(n: int) -> np.ndarray:
    bits = n.bit_length() - 1
    idx = np.arange(n)
    rev = np.zeros(n, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def dft_matrix(n: int, sign: int) -> np.ndarray:
    """W[k, x] = exp(sign * 2 pi i k x / n), exponent reduced mod n exactly."""
    kx = np.outer(np.arange(n), np.arange(n)) % n
    return np.exp(sign * 2j * np.pi * kx / n)


def _radix2(x: np.ndarray, sign: int) -> np.ndarray:
    """Radix-2 DIT along the last axis of x (complex128, length a power of two)."""
    n = x.shape[-1]
    x = x[..., _bit_reverse_perm(n)]
    lead = x.shape[:-1]
    m = 1
    while m < n:
        w = np.exp(sign * 1j * np.pi * np.arange(m) / m)      # exp(sign 2 pi i j / (2m))
        blocks = x.reshape(lead + (n // (2 * m), 2, m))
        even = blocks[..., 0, :]
        odd = blocks[..., 1, :] * w
        x = np.stack((even + odd, even - odd), axis=-2).reshape(lead + (n,))
        m *= 2
    return x


def fft_axis(a: np.ndarray, axis: int, inverse: bool = False) -> np.ndarray:
    """1-D transform of `a` along `axis` (inverse includes the 1/N factor)."""
    x = np.moveaxis(np.asarray(a, dtype=np.complex128), axis, -1)
    n = x.shape[-1]
    sign = +1 if inverse else -1
    if n & (n - 1) == 0:
        y = _radix2(np.ascontiguousarray(x), sign)
    else:
        y = x @ dft_matrix(n, sign).T
    if inverse:
        y = y / n
    return np.moveaxis(y, -1, axis)


def fftn(a: np.ndarray) -> np.ndarray:
    """Forward 3-D transform (all axes), unnormalised."""
    y = np.asarray(a, dtype=np.complex128)
    for ax in range(y.ndim):
        y = fft_axis(y, ax)
    return y


def ifftn(a: np.ndarray) -> np.ndarray:
    """Inverse 3-D transform (all axes), with the 1/N^3 factor."""
    y = np.asarray(a, dtype=np.complex128)
    for ax in range(y.ndim):
        y = fft_axis(y, ax, inverse=True)
    return y
