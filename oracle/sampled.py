"""Oracle values at full problem size, on samples (test infrastructure only).

At 512^3 the step-by-step oracle of `lpt2.py` (its own radix-2 FFT on full complex
arrays) does not fit a test's time and memory.  These functions compute the same
quantities, in float64 and by the same definitions, only where a test samples them:

  delta_k_modes      delta(k) = DFT[w](k) sqrt(P_lin N^3 / V) at given modes, by the
                     direct DFT sum over every cell (Sec. 3 "linear density field";
                     DC / Nyquist rule as in lpt2.delta_k).
  displacements_at   Psi1 and Psi2 at given Lagrangian cells (Sec. 2.1, Eq. second-ini,
                     Sec. 2.4 factorisation).  The six phi_ij and S need every cell, so
                     they are made with a library real FFT (scipy.fft) as a step; Psi1
                     and Psi2 at the sampled cells are then direct inverse-DFT sums over
                     every mode of the half spectrum.
  power_spectrum_rfft the shell P(k), mean |k| and mode counts of lpt2.power_spectrum,
                     from a library real FFT with the half spectrum weighted for its
                     conjugate partners.

Each is pinned in tests/test_oracle_sampled.py against the full-grid oracle (itself
pinned against closed forms and brute force) at sizes where both run.  Only tests/
use this module.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

from . import cosmology as cm
from . import growth as gr
from . import lpt2

__all__ = ["delta_k_modes", "displacements_at", "power_spectrum_rfft", "noise_grid"]

_WORKERS = -1   # all host cores for the library FFT


def noise_grid(n: int, seed: int, chunk_rows: int = 16) -> np.ndarray:
    """The Philox white noise on the full grid (float64), generated in x-slabs."""
    from . import philox
    out = np.empty((n, n, n), dtype=np.float64)
    per = chunk_rows * n * n
    for x0 in range(0, n, chunk_rows):
        out[x0:x0 + chunk_rows] = philox.gaussian_noise(n, seed, first=x0 * n * n, count=per,
                                                        as_float64=True).reshape(-1, n, n)
    return out


def _scale(n: int, box: float, cosmo, kmag: np.ndarray) -> np.ndarray:
    amp = cm.pk_amplitude(cosmo)
    return np.sqrt(cm.pk_linear(cosmo, kmag, amp) * n ** 3 / box ** 3)


def _is_zeroed(n: int, m: np.ndarray) -> np.ndarray:
    """DC or any |n_i| = N/2 (rows of mode numbers m, shape (..., 3))."""
    return np.all(m == 0, axis=-1) | np.any(np.abs(m) == n // 2, axis=-1)


def delta_k_modes(n: int, box: float, cosmo, noise: np.ndarray, modes) -> np.ndarray:
    """delta(k) at the integer modes `modes` (shape (M, 3), entries in [-N/2, N/2)),
    by the direct sum sum_x w(x) exp(-2 pi i n.x / N) times sqrt(P N^3 / V)."""
    modes = np.asarray(modes, dtype=np.int64)
    x = np.arange(n)
    out = np.zeros(len(modes), dtype=np.complex128)
    kf = 2.0 * np.pi / box
    for j, m in enumerate(modes):
        if _is_zeroed(n, m[None, :])[0]:
            continue
        ex, ey, ez = (np.exp(-2j * np.pi * m[c] * x / n) for c in range(3))
        s = (noise @ ez.real) + 1j * (noise @ ez.imag)   # sum over z (real products: no complex copy)
        s = s @ ey                                       # over y
        out[j] = np.dot(s, ex)                           # over x
        out[j] *= _scale(n, box, cosmo, np.array(kf * np.sqrt(float(m @ m))))
    return out


def _half_kgrid(n: int, box: float):
    m = lpt2.mode_numbers(n)
    mz = np.arange(n // 2 + 1)
    kf = 2.0 * np.pi / box
    kx = (kf * m)[:, None, None]
    ky = (kf * m)[None, :, None]
    kz = (kf * mz)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    nyq_xy = np.abs(m) == n // 2
    zero = nyq_xy[:, None, None] | nyq_xy[None, :, None] | (mz == n // 2)[None, None, :] | (k2 == 0.0)
    return (kx, ky, kz), k2, zero


def _point_sum(half: np.ndarray, n: int, cell) -> float:
    """Real inverse DFT (1/N^3 normalised) of a half spectrum at one grid point:
    f(x) = (1/N^3) sum over every mode, the kz > 0 (and < N/2) modes standing for
    themselves and their conjugates."""
    ix, iy, iz = cell
    idx = np.arange(n)
    ex = np.exp(2j * np.pi * idx * ix / n)   # index idx stands for mode idx or idx - N: same phase
    ey = np.exp(2j * np.pi * idx * iy / n)
    ez = np.exp(2j * np.pi * np.arange(n // 2 + 1) * iz / n)
    w = np.full(n // 2 + 1, 2.0)
    w[0] = 1.0
    w[n // 2] = 1.0
    s = np.einsum("ijk,k->ij", half, ez * w)
    s = np.einsum("ij,j->i", s, ey)
    return float(np.real(np.dot(s, ex))) / n ** 3


def displacements_at(n: int, box: float, cosmo, noise: np.ndarray, tables: dict, cells):
    """Psi1 and Psi2 (each shape (M, 3), components x, y, z) at the Lagrangian cells
    `cells` (shape (M, 3)), by the steps of lpt2.displacements."""
    kv, k2, zero = _half_kgrid(n, box)
    kmag = np.sqrt(k2)
    safe = np.where(zero, 1.0, k2)
    dk = sfft.rfftn(noise, workers=_WORKERS)
    with np.errstate(divide="ignore", invalid="ignore"):
        dk *= np.where(zero, 0.0, _scale(n, box, cosmo, np.where(zero, 1.0, kmag)))
    pot1 = np.where(zero, 0.0, dk / safe)                       # phi1(k) = delta / k^2
    del dk
    d1 = gr.interp_lnk(tables["k"], tables["D1"], np.where(zero, 1.0, kmag))
    # S(x) = phi_xx phi_yy + (phi_xx + phi_yy) phi_zz - phi_xy^2 - phi_xz^2 - phi_yz^2
    def phi(a, b):
        return sfft.irfftn(-kv[a] * kv[b] * pot1, s=(n, n, n), workers=_WORKERS)
    S = phi(0, 0)
    T = S.copy()
    f = phi(1, 1)
    S *= f
    T += f
    f = phi(2, 2)
    S += T * f
    del T
    for a, b in ((0, 1), (0, 2), (1, 2)):
        f = phi(a, b)
        S -= f * f
    del f
    Sk = sfft.rfftn(S, workers=_WORKERS)
    del S
    d2 = gr.interp_lnk(tables["k"], tables["D2"], np.where(zero, 1.0, kmag))
    phi2 = np.where(zero, 0.0, -Sk * d2 / safe)
    del Sk
    cells = np.asarray(cells, dtype=np.int64)
    psi1 = np.zeros((len(cells), 3))
    psi2 = np.zeros((len(cells), 3))
    for c in range(3):
        h1 = 1j * kv[c] * d1 * pot1
        h2 = 1j * kv[c] * phi2
        for j, cell in enumerate(cells):
            psi1[j, c] = _point_sum(h1, n, cell)
            psi2[j, c] = _point_sum(h2, n, cell)
    return psi1, psi2


def power_spectrum_rfft(n: int, box: float, delta: np.ndarray, n_shells: int = 32):
    """Shell P(k) of lpt2.power_spectrum from the half spectrum of a real field: the
    kz = 0 and kz = N/2 planes count once, every other kz twice (its conjugate)."""
    dk = sfft.rfftn(delta, workers=_WORKERS)
    p = box ** 3 * (dk.real ** 2 + dk.imag ** 2) / float(n) ** 6
    del dk
    m = lpt2.mode_numbers(n).astype(np.int64)
    mz = np.arange(n // 2 + 1, dtype=np.int64)
    n2 = m[:, None, None] ** 2 + m[None, :, None] ** 2 + mz[None, None, :] ** 2
    M = 4 * n_shells * n_shells * n2
    r = np.floor(np.sqrt(M.astype(np.float64))).astype(np.int64)
    r = np.where((r + 1) ** 2 <= M, r + 1, r)
    r = np.where(r * r > M, r - 1, r)                            # isqrt(M)
    b = np.where((n2 > 0) & (4 * n2 < n * n), r // n, -1)
    w = np.full(n // 2 + 1, 2.0)
    w[0] = 1.0
    w[n // 2] = 1.0
    w = np.broadcast_to(w[None, None, :], b.shape)
    kmag = (2.0 * np.pi / box) * np.sqrt(n2.astype(np.float64))
    sel = b >= 0
    bs = b[sel]
    cnt = np.bincount(bs, weights=w[sel], minlength=n_shells)
    psum = np.bincount(bs, weights=(w * p)[sel], minlength=n_shells)
    ksum = np.bincount(bs, weights=(w * kmag)[sel], minlength=n_shells)
    ok = cnt > 0
    return (np.where(ok, psum / np.maximum(cnt, 1), 0.0), np.where(ok, ksum / np.maximum(cnt, 1), 0.0),
            np.rint(cnt).astype(np.int64))
