"""Pins of oracle/fullsource.py (the full source term S1..S4 of Sec. 3) against Eq.
full-d2 evaluated for explicit triangles, the GR limit and plane-wave identities."""
import numpy as np
import pytest

import workloads as W
from oracle import fullsource as fs
from oracle import growth, lpt2

N, BOX, A = 16, 100.0, 1.0


def _two_mode_field(n, modes, amps):
    """Full complex delta0(k) with entries at +-each mode (a real field)."""
    dk = np.zeros((n, n, n), dtype=np.complex128)
    for m, z in zip(modes, amps):
        dk[m[0] % n, m[1] % n, m[2] % n] += z
        dk[-m[0] % n, -m[1] % n, -m[2] % n] += np.conj(z)
    return dk


@pytest.fixture(scope="module")
def setup():
    c = W.COSMO.replace(fr0_abs=1e-4)           # F4: large MG effect at these k
    tab = growth.growth_tables(c, A, n_steps=256)
    d1gr = fs.d1_gr_norm(c, A, n_steps=256)
    return c, tab, d1gr


@pytest.mark.parametrize("n1,n2", [((1, 2, 0), (0, 1, 3)), ((2, 0, 1), (1, -3, 2)), ((3, 1, 1), (-1, 2, -4))])
def test_two_mode_source_is_eq_full_d2(setup, n1, n2):
    """For delta0 = two cosines, DFT[S1+..+S4] at k = k1 + k2 equals -(1/N^3) times the
    right-hand side of Eq. full-d2 for the triangle (k1, k2) times delta0(k1) delta0(k2)
    (the -1/2 of the Poisson normalisation, twice for the two orderings)."""
    c, tab, d1gr = setup
    z1, z2 = 3.0 + 1.0j, -2.0 + 0.5j
    dk = _two_mode_field(N, [n1, n2], [z1, z2])
    S = fs.source_terms(N, BOX, c, A, dk, tab, d1gr)
    kf = 2 * np.pi / BOX
    k1, k2 = kf * np.array(n1, float), kf * np.array(n2, float)
    D = lambda k: float(growth.interp_lnk(tab["k"], tab["D1"], np.sqrt(k @ k)))
    K = fs.full_d2_kernel(c, A, k1, k2, D(k1), D(k2))
    m = (np.array(n1) + np.array(n2)) % N
    got = (S[0] + S[1] + S[2] + S[3])[m[0], m[1], m[2]]
    want = -K * z1 * z2 / N ** 3
    assert abs(got - want) <= 1e-10 * abs(want), (got, want)
    # each term separately is non-zero (the pin exercises all four)
    assert all(abs(X[m[0], m[1], m[2]]) > 1e-6 * abs(want) for X in S[:4])
    # GR: sin^2(theta) with D1_GR
    cg = c.replace(fr0_abs=0.0)
    KG = fs.full_d2_kernel(cg, A, k1, k2, d1gr, d1gr)
    assert abs(S[4][m[0], m[1], m[2]] - (-KG * z1 * z2 / N ** 3)) <= 1e-10 * abs(KG * z1 * z2 / N ** 3)


def test_self_pair_of_one_mode(setup):
    """A single cosine: at 2 k1 only the ordered pair (k1, k1) contributes, half the
    two-ordering value; the GR source vanishes (sin theta = 0)."""
    c, tab, d1gr = setup
    n1, z1 = (1, 2, 1), 1.5 - 0.7j
    dk = _two_mode_field(N, [n1], [z1])
    S = fs.source_terms(N, BOX, c, A, dk, tab, d1gr)
    kf = 2 * np.pi / BOX
    k1 = kf * np.array(n1, float)
    D = float(growth.interp_lnk(tab["k"], tab["D1"], np.sqrt(k1 @ k1)))
    K = fs.full_d2_kernel(c, A, k1, k1, D, D)
    m = (2 * np.array(n1)) % N
    got = (S[0] + S[1] + S[2] + S[3])[m[0], m[1], m[2]]
    assert abs(got - (-0.5 * K * z1 * z1 / N ** 3)) <= 1e-10 * abs(K * z1 * z1 / N ** 3)
    assert np.abs(S[4]).max() <= 1e-12 * np.abs(got)


def test_gr_limit_ratio_is_one():
    """|fR0| -> 0: mu - 1 ~ k^2 / (3 m^2) and the M2 and m^2 terms vanish like |fR0|; at
    1e-16 every deviation is below 1e-9 at these k."""
    c = W.COSMO.replace(fr0_abs=1e-16)
    tab = growth.growth_tables(c, A, n_steps=128)
    d1gr = fs.d1_gr_norm(c, A, n_steps=128)
    n, box = 16, 64.0
    dk = lpt2.delta_k(n, box, c, W.white_noise(n, 4))
    mean, sig, cnt = fs.source_ratio(n, box, c, A, dk, tab, d1gr, n_bins=8)
    ok = cnt > 0
    np.testing.assert_allclose(mean[ok], 1.0, atol=1e-6)
    assert np.all(sig[ok] < 1e-6)


def test_t1_ratio_limits(setup):
    c, tab, d1gr = setup
    # large scales: mu -> 1, D1 -> D1_GR, the M2 term -> 0
    assert abs(fs.t1_ratio(c, A, np.array([1e-3]), tab, d1gr)[0] - 1.0) < 1e-3
    # it is exactly the T1 kernel ratio of Eq. full-d2
    k = 0.5
    kh = k / np.sqrt(2.0)
    k1, k2 = np.array([kh, 0, 0]), np.array([0, kh, 0])
    D = float(growth.interp_lnk(tab["k"], tab["D1"], kh))
    want = fs.full_d2_kernel(c, A, k1, k2, D, D) / fs.full_d2_kernel(c.replace(fr0_abs=0.0), A, k1, k2, d1gr, d1gr)
    assert abs(fs.t1_ratio(c, A, np.array([k]), tab, d1gr)[0] - want) <= 1e-12 * abs(want)
