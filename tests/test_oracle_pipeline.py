"""Pins of the oracle's pipeline steps: closed forms, invariants and brute force."""
import math

import numpy as np

import workloads as W
from oracle import cosmology as cm
from oracle import fft as of
from oracle import growth as gr
from oracle import lpt2


def flat_tables(d1=1.0, d2=1.0):
    k = gr.k_table()
    return dict(k=k, D1=np.full(k.size, d1), D2=np.full(k.size, d2))


def grid(n, box):
    x = np.arange(n) * box / n
    return np.meshgrid(x, x, x, indexing="ij")


def test_source_vanishes_for_plane_symmetric_field():
    n, box = 32, 100.0
    rng = np.random.default_rng(0)
    dk = np.zeros((n, n, n), complex)
    line = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    dk[:, 0, 0] = line                     # depends on x only
    dk = of.fftn(of.ifftn(dk).real)        # keep it a real field
    _, _, zero = lpt2.kvectors(n, box)
    dk[zero] = 0
    psi1, psi2, S, phi = lpt2.displacements(n, box, dk, flat_tables())
    assert np.max(np.abs(S)) < 1e-12 * np.max(np.abs(phi["xx"])) ** 2
    assert np.max(np.abs(psi2)) < 1e-12
    assert np.max(np.abs(psi1[1:])) < 1e-12


def test_source_closed_form_cos_cos():
    """phi = cos(ka x) cos(kb y): S = phi_xx phi_yy - phi_xy^2 in closed form, and
    Psi2 = D2 grad phi2 with laplacian(phi2) = S solved by hand."""
    n, box = 32, 64.0
    ma, mb = 3, 5
    ka, kb = 2 * np.pi * ma / box, 2 * np.pi * mb / box
    X, Y, Z = grid(n, box)
    phi = np.cos(ka * X) * np.cos(kb * Y)
    delta = (ka ** 2 + kb ** 2) * phi          # phi_,ii = -delta
    d2 = -0.37
    psi1, psi2, S, _ = lpt2.displacements(n, box, of.fftn(delta), flat_tables(1.7, d2))
    want_S = ka ** 2 * kb ** 2 * (np.cos(ka * X) ** 2 * np.cos(kb * Y) ** 2
                                  - np.sin(ka * X) ** 2 * np.sin(kb * Y) ** 2)
    np.testing.assert_allclose(S, want_S, atol=1e-12 * np.abs(want_S).max())
    np.testing.assert_allclose(psi1[0], -1.7 * ka * np.sin(ka * X) * np.cos(kb * Y), atol=1e-12)
    np.testing.assert_allclose(psi1[1], -1.7 * kb * np.cos(ka * X) * np.sin(kb * Y), atol=1e-12)
    c = ka ** 2 * kb ** 2 / 2
    np.testing.assert_allclose(psi2[0], d2 * c * np.sin(2 * ka * X) / (2 * ka), atol=1e-12)
    np.testing.assert_allclose(psi2[1], d2 * c * np.sin(2 * kb * Y) / (2 * kb), atol=1e-12)
    np.testing.assert_allclose(psi2[2], 0.0, atol=1e-12)
    # S is even in phi
    _, _, S2, _ = lpt2.displacements(n, box, of.fftn(-delta), flat_tables(1.7, d2))
    np.testing.assert_allclose(S2, S, atol=1e-13)


def test_psi1_single_mode_with_table_growth():
    c = W.COSMO
    n, box = 32, 128.0
    t = gr.growth_tables(c)
    m0 = np.array([2, -3, 1])
    k0 = 2 * np.pi * m0 / box
    X, Y, Z = grid(n, box)
    ph = k0[0] * X + k0[1] * Y + k0[2] * Z + 0.3
    delta = 0.7 * np.cos(ph)
    psi1, _, _, _ = lpt2.displacements(n, box, of.fftn(delta), t)
    kk = np.sqrt(k0 @ k0)
    d1 = gr.interp_lnk(t["k"], t["D1"], kk)
    for i in range(3):
        np.testing.assert_allclose(psi1[i], -0.7 * d1 * k0[i] / kk ** 2 * np.sin(ph), atol=1e-12)


def test_delta_k_is_noise_times_sqrt_pk_and_zeroes_nyquist():
    c = W.COSMO
    n, box = 16, 64.0
    w = W.white_noise(n, 5).astype(np.float64)
    dk = lpt2.delta_k(n, box, c, w)
    ref = np.fft.fftn(w)                     # library transform, independent of the oracle FFT
    m = lpt2.mode_numbers(n)
    kf = 2 * np.pi / box
    for (i, j, l) in [(1, 0, 0), (3, 5, 2), (15, 1, 7), (0, 0, 3)]:
        k = kf * math.sqrt(m[i] ** 2 + m[j] ** 2 + m[l] ** 2)
        want = ref[i, j, l] * math.sqrt(cm.pk_linear(c, k) * n ** 3 / box ** 3)
        assert abs(dk[i, j, l] - want) < 1e-10 * abs(want)
    assert dk[0, 0, 0] == 0 and np.all(dk[n // 2] == 0) and np.all(dk[:, n // 2] == 0)
    assert np.all(dk[:, :, n // 2] == 0)
    # Hermitian: the inverse is real
    assert np.max(np.abs(of.ifftn(dk).imag)) < 1e-12 * np.max(np.abs(of.ifftn(dk).real))


def test_cic_conservation_and_corner_particles():
    n, box = 8, 16.0
    q = np.indices((n, n, n)).reshape(3, -1).astype(float) * (box / n)
    d = lpt2.cic_density(n, box, q)
    np.testing.assert_allclose(d, 0.0, atol=1e-14)          # one particle per cell corner
    one = np.array([[0.5], [0.5], [0.5]]) * (box / n)       # centre of cell 0
    rho = (lpt2.cic_density(n, box, one) + 1) / n ** 3      # mass per cell / (N^3/N_p)
    got = rho.reshape(n, n, n)
    assert abs(got[:2, :2, :2].sum() - 1.0) < 1e-14
    np.testing.assert_allclose(got[:2, :2, :2], 0.125, atol=1e-15)
    edge = np.array([[box - 0.25 * box / n], [0.0], [0.0]])  # wraps around x
    g2 = ((lpt2.cic_density(n, box, edge) + 1) / n ** 3).reshape(n, n, n)
    assert abs(g2[n - 1, 0, 0] - 0.25) < 1e-14 and abs(g2[0, 0, 0] - 0.75) < 1e-14
    pos = W.random_positions(n, box, 3).astype(np.float64)
    assert abs(lpt2.cic_density(n, box, pos).sum()) < 1e-10


def test_shell_index_brute_force():
    for n, ns in [(16, 32), (32, 32), (24, 7)]:
        b = lpt2.shell_index(n, ns)
        m = lpt2.mode_numbers(n)
        for i in range(n):
            for j in range(n):
                for l in range(n):
                    n2 = m[i] ** 2 + m[j] ** 2 + m[l] ** 2
                    if n2 == 0 or 4 * n2 >= n * n:
                        want = -1
                    else:   # largest b with b * (N / (2 ns)) <= |n|
                        want = math.isqrt(4 * ns * ns * n2) // n
                    assert b[i, j, l] == want


def test_power_spectrum_single_mode_and_counts():
    n, box = 32, 100.0
    X, Y, Z = grid(n, box)
    m0 = (3, 1, 0)
    k0 = 2 * np.pi * np.array(m0) / box
    A = 0.25
    delta = A * np.cos(k0[0] * X + k0[1] * Y)
    pk, km, cnt = lpt2.power_spectrum(n, box, delta, 32)
    b = math.isqrt(4 * 32 * 32 * (9 + 1)) // n
    want = 2 * (box ** 3 * A * A / 4) / cnt[b]            # two modes +-m0 in shell b
    assert abs(pk[b] - want) < 1e-12 * want
    assert np.all(pk[np.arange(32) != b] < 1e-20)
    nm = lpt2.mode_numbers(n)
    n2 = nm[:, None, None] ** 2 + nm[None, :, None] ** 2 + nm[None, None, :] ** 2
    assert cnt.sum() == np.count_nonzero((n2 > 0) & (4 * n2 < n * n))
    assert cnt[0] == 0


def test_full_run_64_gr_vs_mg_and_statistics():
    inst = W.oracle_64()
    r = lpt2.run(inst.n, inst.box, inst.cosmo, seed=inst.seed)
    # displacement field is curl-free gradient: Psi1 rms follows sum over modes of D1^2 P/k^2
    _, k2, zero = lpt2.kvectors(inst.n, inst.box)
    assert np.isfinite(r["pk"]).all() and r["n_modes"].sum() > 0
    # Psi2 opposes nothing in particular, but its size is ~ (3/7) of Psi1^2 / cell scale
    assert 0.05 < r["psi2"].std() / r["psi1"].std() < 0.5
    # linear delta variance: sum |delta_k|^2/N^6 equals the realised field variance
    dreal = of.ifftn(r["delta_k"]).real
    assert abs(np.sum(np.abs(r["delta_k"]) ** 2) / inst.n ** 6 - dreal.var()) < 1e-10
