"""Pins of oracle/pkest.py (CIC deconvolution and interlacing of the P(k) estimator)."""
import numpy as np
import pytest

from oracle import fft as offt
from oracle import lpt2, pkest


def test_interlacing_of_one_particle_on_a_corner():
    """A particle on a cell corner fills one cell of the first grid; shifted by h/2 it
    spreads 1/8 over the 8 cells around the same corner, so the combined DFT is
    (N^3/2) e^{-i k.x} [1 + prod_i cos(pi n_i / N)] for every k != 0 (delta contrast of one
    particle: rho N^3 - 1, the -1 only at k = 0)."""
    n, box = 8, 16.0
    h = box / n
    x = np.array([3, 5, 6], dtype=np.float64)
    F = pkest.interlaced_spectrum(n, box, (x * h).reshape(3, 1))
    m = lpt2.mode_numbers(n)
    M = np.stack(np.meshgrid(m, m, m, indexing="ij"))
    want = 0.5 * n ** 3 * np.exp(-2j * np.pi * np.tensordot(x, M, axes=1) / n) * (
        1.0 + np.prod(np.cos(np.pi * M / n), axis=0))
    want[0, 0, 0] = F[0, 0, 0]
    np.testing.assert_allclose(F, want, atol=1e-9 * n ** 3)


def test_cic_window_values():
    n = 16
    W = pkest.cic_window(n)
    assert W[0, 0, 0] == 1.0
    x = np.pi * 3 / n
    assert abs(W[3, 0, 0] - (np.sin(x) / x) ** 2) < 1e-15
    assert abs(W[-3, 2, 0] - (np.sin(x) / x) ** 2 * (np.sin(np.pi * 2 / n) / (np.pi * 2 / n)) ** 2) < 1e-15


def test_raw_cic_shot_noise_is_the_aliased_window_sum():
    """Uniform random particles: the expected raw CIC |delta(k)|^2 (shot noise) is
    (V / Np) sum over aliases of W^2 = (V / Np) prod_i [1 - (2/3) sin^2(pi n_i / N)]
    (Jing 2005); shell means agree within their statistical error."""
    n, box, npart = 32, 100.0, 400000
    rng = np.random.default_rng(3)
    pos = rng.random((3, npart)) * box
    p, _, cnt = pkest.power_spectrum_est(n, box, pos, 8)
    m = lpt2.mode_numbers(n)
    f = 1.0 - (2.0 / 3.0) * np.sin(np.pi * m / n) ** 2
    want_grid = box ** 3 / npart * f[:, None, None] * f[None, :, None] * f[None, None, :]
    b = lpt2.shell_index(n, 8).ravel()
    sel = b >= 0
    want = np.bincount(b[sel], weights=want_grid.ravel()[sel], minlength=8) / np.maximum(cnt, 1)
    ok = cnt > 50
    # exponential scatter per mode: relative error of a shell mean ~ 1/sqrt(count)
    assert np.all(np.abs(p[ok] / want[ok] - 1) < 6 / np.sqrt(cnt[ok] / 2)), (p / want)


def test_deconvolved_and_interlaced_shot_noise_is_flatter():
    """Deconvolution lifts the raw shot noise toward V/Np; with interlacing the odd
    images cancel and the deconvolved estimate stays closest to V/Np at high k."""
    n, box, npart = 32, 100.0, 400000
    pos = np.random.default_rng(4).random((3, npart)) * box
    flat = box ** 3 / npart
    raw, _, cnt = pkest.power_spectrum_est(n, box, pos, 8)
    dec, _, _ = pkest.power_spectrum_est(n, box, pos, 8, deconvolve=True)
    both, _, _ = pkest.power_spectrum_est(n, box, pos, 8, deconvolve=True, interlace=True)
    hi = slice(5, 8)
    assert np.all(raw[hi] < 0.8 * flat)
    assert np.all(np.abs(both[hi] / flat - 1) < np.abs(dec[hi] / flat - 1))
