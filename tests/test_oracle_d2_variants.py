"""Pins of the D2 triangle variants of oracle/growth.py (Sec. 3 triangle comparison):
the braces equal Eq. full-d2 for the explicit triangle (through fullsource.full_d2_kernel,
itself pinned by two-mode source fields), their d/dln|fR0| equals finite differences, and
the growth tables meet the Einstein-de Sitter closed forms for every variant."""
import numpy as np
import pytest

import workloads as W
from oracle import cosmology as cm
from oracle import fullsource as fs
from oracle import growth as gr

EDS = W.COSMO.replace(omega_m=1.0, omega_l=0.0, fr0_abs=0.0)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 7, 8])
@pytest.mark.parametrize("k,a", [(0.05, 1.0), (0.4, 0.7), (2.0, 0.5)])
def test_braces_are_eq_full_d2_of_the_triangle(variant, k, a):
    c = W.COSMO.replace(fr0_abs=1e-5)
    k1, k2, ct = gr.triangle(np.array(k), variant)
    st = np.sqrt(1.0 - ct * ct)
    v1 = np.array([float(k1), 0.0, 0.0])
    v2 = float(k2) * np.array([ct, st, 0.0])
    assert abs(np.linalg.norm(v1 + v2) - k) <= 1e-12 * k
    assert abs(np.linalg.norm(v1) / np.linalg.norm(v2) - gr.VARIANTS[variant][0]) <= 1e-12
    want = fs.full_d2_kernel(c, a, v1, v2, 1.0, 1.0) / (cm.four_pi_g_rho(c, a) * st * st)
    got = float(gr.d2_braces(c, np.array(k), a, variant))
    assert abs(got - want) <= 1e-12 * abs(want), (got, want)


def test_winther_and_gr_braces():
    c = W.COSMO.replace(fr0_abs=1e-5)
    k = np.array([0.01, 0.3, 3.0])
    np.testing.assert_array_equal(gr.d2_braces(c, k, 0.8, 5), gr.d2_braces(c, k, 0.8, 0))
    np.testing.assert_array_equal(gr.d2_braces(c, k, 0.8, 6), 1.0)


@pytest.mark.parametrize("variant", [0, 1, 3, 4, 7, 8])
def test_brace_tangent_is_the_derivative(variant):
    c = W.COSMO.replace(fr0_abs=1e-5)
    k = np.array([0.02, 0.2, 1.0, 5.0])
    _, t = gr.d2_braces(c, k, 0.9, variant, tangent=True)
    h = 1e-4
    bp = gr.d2_braces(c.replace(fr0_abs=1e-5 * np.exp(h)), k, 0.9, variant)
    bm = gr.d2_braces(c.replace(fr0_abs=1e-5 * np.exp(-h)), k, 0.9, variant)
    np.testing.assert_allclose(t, (bp - bm) / (2 * h), rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("variant", range(10))
def test_eds_gr_every_variant(variant):
    t = gr.growth_tables(EDS, 1.0, k=np.array([1e-3, 0.1, 1.0]), n_steps=2048, variant=variant)
    np.testing.assert_allclose(t["D2"], -3.0 / 7.0, rtol=1e-10)


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5, 7, 8])
def test_eds_mu_four_thirds_every_variant_is_t1(variant):
    """m^2 -> 0: mu = 4/3 at every k, the m^2/Pi and M2 terms vanish, the braces are
    (4/3) sin^2 theta / sin^2 theta and D1 is scale-independent: every triangle gives the
    T1 solution, itself pinned to the closed form (test_oracle_growth)."""
    # |fR0| = 1e40: m^2 / (k1/a)^2 must vanish also for the squeezed k1 = 1e-3 k2 (at
    # |fR0| = 1e30 it is 2e-8 at a_init for k = 0.05, enough to move D2 by 6e-10)
    c = EDS.replace(fr0_abs=1e40)
    k = np.array([0.05, 1.0])
    t1 = gr.growth_tables(c, 1.0, k=k, n_steps=1024, variant=0)
    tv = gr.growth_tables(c, 1.0, k=k, n_steps=1024, variant=variant)
    np.testing.assert_allclose(tv["D2"], t1["D2"], rtol=1e-12)


def test_variant_tangents_match_finite_differences():
    c = W.COSMO.replace(fr0_abs=1e-5)
    k = np.array([0.01, 0.1, 0.5, 2.0])
    t = gr.growth_tables(c, 1.0, k=k, n_steps=256, variant=3)
    h = 1e-4
    tp = gr.growth_tables(c.replace(fr0_abs=1e-5 * np.exp(h)), 1.0, k=k, n_steps=256, variant=3)
    tm = gr.growth_tables(c.replace(fr0_abs=1e-5 * np.exp(-h)), 1.0, k=k, n_steps=256, variant=3)
    np.testing.assert_allclose(t["dD2"], (tp["D2"] - tm["D2"]) / (2 * h), rtol=1e-5, atol=1e-12)
    np.testing.assert_allclose(t["dD1"], (tp["D1"] - tm["D1"]) / (2 * h), rtol=1e-5, atol=1e-12)


def test_winther_overestimates_t1_at_small_scales():
    """Sec. 3: D1(k)^2 instead of D1(k/sqrt2)^2 gives a larger |D2| where D1 grows with k."""
    c = W.COSMO.replace(fr0_abs=1e-4)
    k = np.array([1e-3, 1.0])
    t1 = gr.growth_tables(c, 1.0, k=k, n_steps=256, variant=0)
    tw = gr.growth_tables(c, 1.0, k=k, n_steps=256, variant=5)
    assert abs(tw["D2"][0] / t1["D2"][0] - 1) < 1e-4
    assert abs(tw["D2"][1]) > abs(t1["D2"][1])


def test_squeezed_braces_reach_the_k1_to_zero_limit():
    """k1 -> 0 at 90 deg: Pi(k1) -> m^2, Pi(k2) -> Pi(k), so the braces of Eq. full-d2
    tend to mu(k) - (2/27) 4 pi G rho (k^2/a^2) M2 / (m^2 Pi(k)^2); r = 1e-3 is within
    O(r^2) of that limit."""
    c = W.COSMO.replace(fr0_abs=1e-5)
    k = np.array([0.01, 0.2, 1.0, 4.0])
    for a in (0.5, 1.0):
        q, msq = (k / a) ** 2, cm.m2(c, a)
        P = q + msq
        lim = 1.0 + q / (3.0 * P) - (2.0 / 27.0) * cm.four_pi_g_rho(c, a) * q * cm.M2(c, a) / (msq * P * P)
        np.testing.assert_allclose(gr.d2_braces(c, k, a, 8), lim, rtol=1e-5)


def test_lcdm_fit_variant():
    """Eq. lcdm-fit as a D2 variant: exact -3/7 D1^2 in Einstein-de Sitter (above); in
    LCDM GR within the fit's own accuracy of the D2 equation (1.5e-3, as pinned against
    the Bouchet form in test_oracle_growth); its tangent is the finite difference."""
    c = W.COSMO.replace(fr0_abs=0.0)
    k = np.array([0.01, 1.0])
    for a in (0.5, 1.0):
        fit = gr.growth_tables(c, a, k=k, n_steps=1024, variant=gr.BOUCHET)
        ode = gr.growth_tables(c, a, k=k, n_steps=1024, variant=0)
        np.testing.assert_allclose(fit["D1"], ode["D1"], rtol=1e-14)
        np.testing.assert_allclose(fit["D2"], ode["D2"], rtol=1.5e-3)
    cm5 = W.COSMO.replace(fr0_abs=1e-5)
    t = gr.growth_tables(cm5, 0.8, k=k, n_steps=256, variant=gr.BOUCHET)
    h = 1e-4
    tp = gr.growth_tables(cm5.replace(fr0_abs=1e-5 * np.exp(h)), 0.8, k=k, n_steps=256, variant=gr.BOUCHET)
    tm = gr.growth_tables(cm5.replace(fr0_abs=1e-5 * np.exp(-h)), 0.8, k=k, n_steps=256, variant=gr.BOUCHET)
    np.testing.assert_allclose(t["dD2"], (tp["D2"] - tm["D2"]) / (2 * h), rtol=1e-5, atol=1e-12)


def test_d2_fit_comparison_of_fig_d2fit():
    """Fig. d2fit: T1 D2 / (-3/7 D1^2) divided by Omega_m(a)^(-1/143) for |fR0| = 1e-4.
    The paper finds the fit valid at k = 1e-3 h/Mpc and failing on smaller scales by
    growing amounts; at k = 0.1 and 1 h/Mpc the T1 solution lies 4 % below the fit today
    (the paper's 3-4 % at k = 0.01 h/Mpc is not reproduced: see the design notes)."""
    c = W.COSMO.replace(fr0_abs=1e-4)
    k = np.array([1e-3, 1e-2, 0.1, 1.0])
    rows = []
    for a in (0.2, 0.5, 1.0):
        t = gr.growth_tables(c, a, k=k, n_steps=512)
        rows.append(t["D2"] / (-3.0 / 7.0 * t["D1"] ** 2) / cm.omega_m_a(c, a) ** (-1.0 / 143.0))
    rows = np.array(rows)
    assert np.abs(rows[:, 0] - 1.0).max() < 2e-3            # largest scales: the fit holds
    assert np.all(np.abs(rows[-1, 2:] - 1.0) > 0.03)        # k >= 0.1 today: > 3 % off
    assert np.all(np.abs(rows[-1] - 1.0)[1:] > np.abs(rows[-1] - 1.0)[0])
