"""Pins of oracle/sampled.py (full-size values on samples) against the full-grid
oracle, itself pinned against closed forms and brute force, at sizes both run."""
import numpy as np
import pytest

import workloads as W
from oracle import growth, lpt2, philox, sampled


def test_noise_grid_is_the_philox_field():
    n = 16
    np.testing.assert_array_equal(sampled.noise_grid(n, 5, chunk_rows=4).ravel(),
                                  philox.gaussian_noise(n, 5, as_float64=True))


@pytest.mark.parametrize("n,box", [(16, 64.0), (32, 200.0)])
def test_delta_k_modes_match_full_grid(n, box):
    c = W.COSMO.replace(fr0_abs=1e-5)
    noise = sampled.noise_grid(n, 3)
    full = lpt2.delta_k(n, box, c, noise)
    rng = np.random.default_rng(1)
    modes = rng.integers(-n // 2, n // 2, size=(10, 3))
    modes = np.vstack([modes, [[0, 0, 0], [1, 0, 0], [0, -1, 3], [-n // 2, 2, 1], [3, 2, n // 2 - 1]]])
    got = sampled.delta_k_modes(n, box, c, noise, modes)
    want = full[modes[:, 0] % n, modes[:, 1] % n, modes[:, 2] % n]
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-10 * np.abs(full).max())
    assert got[10] == 0 and got[13] == 0          # DC and a Nyquist mode are zeroed


def test_displacements_at_match_full_grid():
    n, box = 32, 128.0
    c = W.COSMO.replace(fr0_abs=1e-5)
    tables = growth.growth_tables(c, 1.0, n_steps=128)
    noise = sampled.noise_grid(n, 2)
    dk = lpt2.delta_k(n, box, c, noise)
    psi1, psi2, _, _ = lpt2.displacements(n, box, dk, tables)
    cells = np.array([[0, 0, 0], [5, 17, 31], [31, 1, 16], [12, 30, 7]])
    g1, g2 = sampled.displacements_at(n, box, c, noise, tables, cells)
    for j, (x, y, z) in enumerate(cells):
        np.testing.assert_allclose(g1[j], psi1[:, x, y, z], rtol=1e-9, atol=1e-12 * np.abs(psi1).max())
        np.testing.assert_allclose(g2[j], psi2[:, x, y, z], rtol=1e-9, atol=1e-10 * np.abs(psi2).max())


@pytest.mark.parametrize("n,ns", [(32, 16), (64, 32), (64, 7)])
def test_power_spectrum_rfft_matches_full_grid(n, ns):
    rng = np.random.default_rng(n + ns)
    delta = rng.standard_normal((n, n, n))
    p0, k0, c0 = lpt2.power_spectrum(n, 100.0, delta, ns)
    p1, k1, c1 = sampled.power_spectrum_rfft(n, 100.0, delta, ns)
    np.testing.assert_array_equal(c1, c0)
    np.testing.assert_allclose(p1, p0, rtol=1e-10)
    np.testing.assert_allclose(k1, k0, rtol=1e-12)
