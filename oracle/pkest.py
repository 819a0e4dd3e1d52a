"""P(k) estimator refinements (oracle, float64; test infrastructure only): CIC window
deconvolution and interlacing, the refinements Sec. 4 leaves out of its P(k) (a raw CIC
estimate; Sefusatti et al. 2016 describe both).

  CIC window of a mode n (integers in [-N/2, N/2)): W(n) = prod_i sinc^2(pi n_i / N),
  sinc(x) = sin(x) / x.  Deconvolution divides |delta(k)|^2 by W^2.
  Interlacing: a second CIC grid of the particles shifted by +h/2 along every axis
  (h = L/N); the two spectra are combined as delta(k) = [F1(k) + F2(k) e^{i pi (nx+ny+nz)/N}] / 2,
  which cancels the odd aliasing images of the first grid.
Shells, normalisation and mode counts as lpt2.power_spectrum.
"""
from __future__ import annotations

import numpy as np

from . import fft as offt
from . import lpt2

__all__ = ["cic_window", "interlaced_spectrum", "power_spectrum_est"]


def cic_window(n: int) -> np.ndarray:
    """W(n) on the full grid, (N, N, N)."""
    m = lpt2.mode_numbers(n).astype(np.float64)
    x = np.pi * m / n
    s = np.ones_like(x)
    nz = m != 0
    s[nz] = (np.sin(x[nz]) / x[nz]) ** 2
    return s[:, None, None] * s[None, :, None] * s[None, None, :]


def interlaced_spectrum(n: int, box: float, pos: np.ndarray) -> np.ndarray:
    """Combined DFT of the CIC density contrast of pos (3, Np) and of pos shifted by +h/2."""
    h = box / n
    F1 = offt.fftn(lpt2.cic_density(n, box, pos))
    F2 = offt.fftn(lpt2.cic_density(n, box, np.mod(pos + 0.5 * h, box)))
    m = lpt2.mode_numbers(n)
    ph = np.exp(1j * np.pi * (m[:, None, None] + m[None, :, None] + m[None, None, :]) / n)
    return 0.5 * (F1 + F2 * ph)


def power_spectrum_est(n: int, box: float, pos: np.ndarray, n_shells: int = 32,
                       deconvolve: bool = False, interlace: bool = False):
    """(P, mean |k|, counts) per shell of the CIC estimate of pos with the refinements."""
    F = interlaced_spectrum(n, box, pos) if interlace else offt.fftn(lpt2.cic_density(n, box, pos))
    p = box ** 3 * np.abs(F) ** 2 / float(n) ** 6
    if deconvolve:
        p = p / cic_window(n) ** 2
    b = lpt2.shell_index(n, n_shells).ravel()
    _, k2, _ = lpt2.kvectors(n, box)
    kmag = np.sqrt(k2).ravel()
    sel = b >= 0
    cnt = np.bincount(b[sel], minlength=n_shells).astype(np.int64)
    psum = np.bincount(b[sel], weights=p.ravel()[sel], minlength=n_shells)
    ksum = np.bincount(b[sel], weights=kmag[sel], minlength=n_shells)
    with np.errstate(invalid="ignore", divide="ignore"):
        return (np.where(cnt > 0, psum / np.maximum(cnt, 1), 0.0),
                np.where(cnt > 0, ksum / np.maximum(cnt, 1), 0.0), cnt)
