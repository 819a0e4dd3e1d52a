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


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
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


@pytest.mark.parametrize("variant", [0, 1, 3, 4])
def test_brace_tangent_is_the_derivative(variant):
    c = W.COSMO.replace(fr0_abs=1e-5)
    k = np.array([0.02, 0.2, 1.0, 5.0])
    _, t = gr.d2_braces(c, k, 0.9, variant, tangent=True)
    h = 1e-4
    bp = gr.d2_braces(c.replace(fr0_abs=1e-5 * np.exp(h)), k, 0.9, variant)
    bm = gr.d2_braces(c.replace(fr0_abs=1e-5 * np.exp(-h)), k, 0.9, variant)
    np.testing.assert_allclose(t, (bp - bm) / (2 * h), rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("variant", range(7))
def test_eds_gr_every_variant(variant):
    t = gr.growth_tables(EDS, 1.0, k=np.array([1e-3, 0.1, 1.0]), n_steps=2048, variant=variant)
    np.testing.assert_allclose(t["D2"], -3.0 / 7.0, rtol=1e-10)


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5])
def test_eds_mu_four_thirds_every_variant_is_t1(variant):
    """m^2 -> 0: mu = 4/3 at every k, the m^2/Pi and M2 terms vanish, the braces are
    (4/3) sin^2 theta / sin^2 theta and D1 is scale-independent: every triangle gives the
    T1 solution, itself pinned to the closed form (test_oracle_growth)."""
    c = EDS.replace(fr0_abs=1e30)
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
