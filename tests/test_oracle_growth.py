"""Pins of the oracle's background, f(R) functions, P(k) and growth tables."""
import numpy as np
import pytest
from scipy import integrate

import workloads as W
from oracle import cosmology as cm
from oracle import growth as gr

EDS = W.COSMO.replace(omega_m=1.0, omega_l=0.0, fr0_abs=0.0)


def test_mu_limits():
    c = W.COSMO
    a = 1.0
    m = np.sqrt(cm.m2(c, a))
    assert abs(cm.mu(c, 1e-6 * m, a) - 1.0) < 1e-10          # k << m: GR
    assert abs(cm.mu(c, 1e6 * m, a) - 4.0 / 3.0) < 1e-10     # k >> m: 4/3 enhancement
    assert abs(cm.mu(c, m, a) - 7.0 / 6.0) < 1e-12           # k/a = m: 1 + 1/6
    assert np.all(cm.mu(c.replace(fr0_abs=0.0), np.logspace(-4, 1, 9), a) == 1.0)
    # M1 = 3 m^2 and M2 relation: M2 * |fR0|^2 (Om+4OL)^4 / x^5 == 3/2 * M1 * |fR0| (Om+4OL)^2 / x^3
    x = c.omega_m + 4 * c.omega_l
    lhs = cm.M2(c, a) * c.fr0_abs ** 2 * x ** 4 / x ** 5
    rhs = 1.5 * 3 * cm.m2(c, a) * c.fr0_abs * x ** 2 / x ** 3
    assert abs(lhs / rhs - 1) < 1e-14
    # Compton wavelength for |fR0| = 1e-5 today: 1/m ~ 7.6 Mpc/h
    assert 5.0 < 1.0 / m < 10.0


def test_eh_transfer_limits():
    c = W.COSMO
    assert abs(cm.eh_nowiggle_T(c, 1e-7) - 1.0) < 1e-5
    k = np.logspace(-4, 2, 200)
    T = cm.eh_nowiggle_T(c, k)
    assert np.all(np.diff(T) < 0)
    # large-k asymptote T -> ln(1.8 q)/(14.2 q^2)*... decays close to k^-2 ln k
    slope = np.log(T[-1] / T[-11]) / np.log(k[-1] / k[-11])
    assert -2.0 < slope < -1.7


def test_sigma8_normalisation_independent_quadrature():
    c = W.COSMO
    amp = cm.pk_amplitude(c)

    def integrand(lnk):
        k = np.exp(lnk)
        return k ** 3 * cm.pk_linear(c, k, amp) * cm.tophat_W(8.0 * k) ** 2 / (2 * np.pi ** 2)

    val, _ = integrate.quad(integrand, np.log(1e-5), np.log(1e3), limit=2000, epsabs=0, epsrel=1e-10)
    assert abs(np.sqrt(val) - c.sigma8) < 1e-6


def test_eds_gr_growth_exact():
    t = gr.growth_tables(EDS, 1.0, k=np.array([1e-3, 0.1, 1.0]), n_steps=2048)
    np.testing.assert_allclose(t["D1"], 1.0, rtol=1e-10)
    np.testing.assert_allclose(t["D2"], -3.0 / 7.0, rtol=1e-10)
    t = gr.growth_tables(EDS, 0.5, k=np.array([0.1]), n_steps=2048)
    np.testing.assert_allclose(t["D1"], 0.5, rtol=1e-10)
    np.testing.assert_allclose(t["D2"], -3.0 / 7.0 * 0.25, rtol=1e-10)
    assert np.all(t["dD1"] == 0) and np.all(t["dD2"] == 0)


def test_eds_mu_four_thirds_closed_form():
    """EdS with m^2 -> 0 (|fR0| huge): mu = 4/3 for every k > 0 and D1 = A a^p + B a^q,
    p, q = (-1 +- sqrt 33)/4; D2 solves D2'' + D2'/2 - 2 D2 = -2 D1^2 in s = ln a."""
    c = EDS.replace(fr0_abs=1e30)
    ai = c.a_init
    p, q = (-1 + np.sqrt(33)) / 4, (-1 - np.sqrt(33)) / 4
    # D1(ai) = ai, dD1/ds(ai) = ai
    M = np.array([[ai ** p, ai ** q], [p * ai ** p, q * ai ** q]])
    A, B = np.linalg.solve(M, [ai, ai])
    t = gr.growth_tables(c, 1.0, k=np.array([0.05, 1.0]), n_steps=4096)
    # normalisation: GR EdS D1(a=1) = 1, so the table is unnormalised
    np.testing.assert_allclose(t["D1"], A + B, rtol=1e-9)
    # particular solution of L[D2] = -2 (A a^p + B a^q)^2, L[a^r] = (r^2 + r/2 - 2) a^r
    L = lambda r: r * r + 0.5 * r - 2.0
    terms = {2 * p: A * A, p + q: 2 * A * B, 2 * q: B * B}
    cp = {r: -2.0 * cf / L(r) for r, cf in terms.items()}
    part = lambda a: sum(v * a ** r for r, v in cp.items())
    dpart = lambda a: sum(r * v * a ** r for r, v in cp.items())
    # homogeneous part fixed by D2(ai) = -3/7 ai^2, dD2/ds(ai) = -6/7 ai^2
    C, D = np.linalg.solve(M, [-3 / 7 * ai ** 2 - part(ai), -6 / 7 * ai ** 2 - dpart(ai)])
    np.testing.assert_allclose(t["D2"], part(1.0) + C + D, rtol=1e-9)


def test_lcdm_gr_heath_integral_and_bouchet_fit():
    c = W.COSMO.replace(fr0_abs=0.0)
    E = lambda a: np.sqrt(c.omega_m / a ** 3 + c.omega_l)
    heath = lambda a: 2.5 * c.omega_m * E(a) * integrate.quad(lambda x: 1 / (x * E(x)) ** 3, 0, a,
                                                              epsabs=0, epsrel=1e-12)[0]
    for a in (0.5, 1.0):
        t = gr.growth_tables(c, a, k=np.array([0.1]))
        want = heath(a) / heath(1.0)
        assert abs(t["D1"][0] / want - 1) < 2e-6
        om = c.omega_m / a ** 3 / E(a) ** 2
        ratio = t["D2"][0] / (-3 / 7 * t["D1"][0] ** 2)
        assert abs(ratio / om ** (-1 / 143) - 1) < 1.5e-3


@pytest.mark.parametrize("variant", [0, 3, 5])
def test_rk4_against_scipy_dop853(variant):
    """Pins the RK4 stepping: the same right-hand side integrated by an adaptive
    8th-order method agrees to 1e-10 (T1, a k1 = 2 k2 triangle, Winther)."""
    c = W.COSMO
    k = np.array([1e-3, 0.05, 0.3, 3.0])
    t = gr.growth_tables(c, 1.0, k=k, variant=variant)
    y0 = np.zeros((16, k.size))
    y0[0:6] = c.a_init
    y0[6] = -3 / 7 * c.a_init ** 2
    y0[7] = -6 / 7 * c.a_init ** 2
    f = lambda s, y: gr._rhs(c, k, s, y.reshape(16, -1), variant).ravel()
    sol = integrate.solve_ivp(f, (np.log(c.a_init), 0.0), y0.ravel(), method="DOP853",
                              rtol=1e-13, atol=1e-16)
    y = sol.y[:, -1].reshape(16, -1)
    n1 = gr.d1_gr(c)
    np.testing.assert_allclose(t["D1"], y[0] / n1, rtol=1e-10)
    np.testing.assert_allclose(t["D2"], y[6] / n1 ** 2, rtol=1e-10)
    np.testing.assert_allclose(t["dD1"], y[8] / n1, rtol=1e-8, atol=1e-14)
    np.testing.assert_allclose(t["dD2"], y[14] / n1 ** 2, rtol=1e-8, atol=1e-14)


def test_mg_limits_of_tables():
    c = W.COSMO
    t = gr.growth_tables(c)
    g = gr.growth_tables(c.replace(fr0_abs=0.0))
    # k -> 0: GR; |fR0| -> 0: GR
    assert abs(t["D1"][0] / g["D1"][0] - 1) < 1e-6
    tiny = gr.growth_tables(c.replace(fr0_abs=1e-16))
    np.testing.assert_allclose(tiny["D1"], g["D1"], rtol=1e-6)
    np.testing.assert_allclose(tiny["D2"], g["D2"], rtol=1e-6)
    # MG enhances growth and grows monotonically with k
    assert np.all(np.diff(t["D1"]) >= -1e-15) and t["D1"][-1] > 1.2
    assert np.all(t["D1"] >= g["D1"] * (1 - 1e-12))


def test_tangent_matches_finite_difference():
    c = W.COSMO
    k = np.array([0.01, 0.1, 1.0])
    t = gr.growth_tables(c, 1.0, k=k)
    h = 1e-4
    up = gr.growth_tables(c.replace(fr0_abs=c.fr0_abs * np.exp(h)), 1.0, k=k)
    dn = gr.growth_tables(c.replace(fr0_abs=c.fr0_abs * np.exp(-h)), 1.0, k=k)
    np.testing.assert_allclose(t["dD1"], (up["D1"] - dn["D1"]) / (2 * h), rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(t["dD2"], (up["D2"] - dn["D2"]) / (2 * h), rtol=1e-6, atol=1e-12)


def test_interp_lnk_is_linear_in_lnk_and_clamped():
    kt = gr.k_table(8, 1e-2, 1.0)
    v = np.log(kt) * 3 + 1
    kq = np.array([1e-3, 1e-2, 0.0317, 0.5, 1.0, 5.0])
    got = gr.interp_lnk(kt, v, kq)
    want = np.clip(np.log(kq), np.log(1e-2), 0.0) * 3 + 1
    np.testing.assert_allclose(got, want, rtol=1e-13)
