"""Pins of the oracle's linear transfer function (Eisenstein & Hu 1998, the no-wiggle
fit of their Eqs. 26 and 28-31) against values fixed outside it.

- Sound horizon, Eq. 26: against the sound horizon at the drag epoch that EH98 derive
  before fitting it (their Eqs. 2-6: z_eq, k_eq, the z_d fit, R(z) and the closed-form
  integral), against the fit of Aubourg et al. (2015, Eq. 16; calibrated on CAMB to 0.02 %)
  and against the value the Planck 2018 analysis reports (r_drag = 147.09 Mpc for
  omega_b = 0.02237, omega_c = 0.1200).  A wrong exponent, coefficient or a little-h
  slip (Omega instead of omega) moves s by far more than the few per cent allowed.
- alpha_Gamma, Eq. 31: against the effective shape of Sugiyama (1995),
  Gamma = Omega_m h exp(-Omega_b - sqrt(2h) Omega_b / Omega_m), an independent fit of the
  same small-scale baryon suppression: agreement within 1.5 % over a range of
  cosmologies (measured 0.35-1.05 %).
- Gamma_eff(k), Eq. 30: the limits Omega_m h (k -> 0) and alpha_Gamma Omega_m h
  (k -> infinity), and the transition at the sound-horizon scale: Gamma_eff is halfway
  between its limits where 0.43 k s = 1 with k in Mpc^-1 and s the physical sound
  horizon (Aubourg et al.), i.e. at k = 1 / (0.43 r_d h) in h/Mpc.  Writing k in h/Mpc
  into Eq. 30 without the factor h moves that point by 1/h and Gamma_eff there by 7 %.
- T0(q), Eq. 29 at q of Eq. 28: with no baryons the shape is the CDM transfer function,
  which the fit of Bardeen, Bond, Kaiser & Szalay (1986, Eq. G3) also describes; the two
  agree within 5 % for k in [1e-3, 10] h/Mpc (measured within 4 %).  A k unit off by h in q
  changes T by ~30 % there.
"""
import numpy as np
import pytest

import workloads as W
from oracle import cosmology as cm


def eh98_sound_horizon_exact(omega_m_h2, omega_b_h2, t_cmb):
    """Sound horizon at the drag epoch, Eisenstein & Hu (1998) Eqs. 2-6 (Mpc)."""
    th = t_cmb / 2.7
    wm, wb = omega_m_h2, omega_b_h2
    z_eq = 2.50e4 * wm * th ** -4                                             # Eq. 2
    k_eq = 7.46e-2 * wm * th ** -2                                            # Eq. 3, Mpc^-1
    b1 = 0.313 * wm ** -0.419 * (1.0 + 0.607 * wm ** 0.674)                   # Eq. 4
    b2 = 0.238 * wm ** 0.223
    z_d = 1291.0 * wm ** 0.251 / (1.0 + 0.659 * wm ** 0.828) * (1.0 + b1 * wb ** b2)
    R = lambda z: 31.5 * wb * th ** -4 * (z / 1.0e3) ** -1                   # Eq. 5
    r_d, r_eq = R(z_d), R(z_eq)
    return (2.0 / (3.0 * k_eq) * np.sqrt(6.0 / r_eq)                          # Eq. 6
            * np.log((np.sqrt(1.0 + r_d) + np.sqrt(r_d + r_eq)) / (1.0 + np.sqrt(r_eq))))


def aubourg_r_drag(omega_cb_h2, omega_b_h2, omega_nu_h2=0.0):
    """r_d fit of Aubourg et al. (2015), Eq. 16 (Mpc)."""
    return (55.154 * np.exp(-72.3 * (omega_nu_h2 + 0.0006) ** 2)
            / (omega_cb_h2 ** 0.25351 * omega_b_h2 ** 0.12807))


def sugiyama_gamma(om, ob, h):
    return om * h * np.exp(-ob - np.sqrt(2.0 * h) * ob / om)


def bbks_T(q):
    """Bardeen, Bond, Kaiser & Szalay (1986) Eq. G3."""
    return (np.log(1.0 + 2.34 * q) / (2.34 * q)
            * (1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4) ** -0.25)


def test_sound_horizon_against_exact_eh98_integral():
    for om, ob, h in [(0.3, 0.0481, 0.7), (0.25, 0.045, 0.72), (0.35, 0.05, 0.65), (0.3, 0.03, 0.7)]:
        c = W.COSMO.replace(omega_m=om, omega_l=1 - om, omega_b=ob, h=h)
        exact = eh98_sound_horizon_exact(om * h * h, ob * h * h, c.t_cmb)
        assert abs(cm.eh_sound_horizon(c) / exact - 1.0) < 0.02, (om, ob, h, cm.eh_sound_horizon(c), exact)


def test_sound_horizon_against_aubourg_and_planck():
    c = W.COSMO
    wm, wb = c.omega_m * c.h ** 2, c.omega_b * c.h ** 2
    s = cm.eh_sound_horizon(c)
    assert abs(s / aubourg_r_drag(wm, wb) - 1.0) < 0.03, (s, aubourg_r_drag(wm, wb))
    # Planck 2018 base LCDM: omega_b = 0.02237, omega_c = 0.1200, h = 0.6736, r_drag = 147.09 Mpc
    h = 0.6736
    p18 = W.COSMO.replace(omega_m=(0.02237 + 0.1200) / h ** 2, omega_l=1 - (0.02237 + 0.1200) / h ** 2,
                          omega_b=0.02237 / h ** 2, h=h)
    assert abs(cm.eh_sound_horizon(p18) / 147.09 - 1.0) < 0.03, cm.eh_sound_horizon(p18)
    assert abs(aubourg_r_drag(0.02237 + 0.1200, 0.02237, 0.0006) / 147.09 - 1.0) < 0.003


@pytest.mark.parametrize("om,ob,h", [(0.3, 0.0481, 0.7), (0.3, 0.02, 0.7), (0.25, 0.045, 0.72),
                                     (0.35, 0.05, 0.65), (0.3, 0.06, 0.7), (0.3, 0.01, 0.7),
                                     (0.2, 0.04, 0.7), (0.4, 0.05, 0.7)])
def test_alpha_gamma_against_sugiyama_shape(om, ob, h):
    c = W.COSMO.replace(omega_m=om, omega_l=1 - om, omega_b=ob, h=h)
    got = cm.eh_alpha_gamma(c) * om * h
    assert abs(got / sugiyama_gamma(om, ob, h) - 1.0) < 0.015, (got, sugiyama_gamma(om, ob, h))


def test_gamma_eff_limits_and_sound_horizon_transition():
    c = W.COSMO
    omh = c.omega_m * c.h
    alpha = cm.eh_alpha_gamma(c)
    assert abs(cm.eh_gamma_eff(c, 1e-6) / omh - 1.0) < 1e-9
    assert abs(cm.eh_gamma_eff(c, 1e3) / (alpha * omh) - 1.0) < 1e-9
    r_d = aubourg_r_drag(c.omega_m * c.h ** 2, c.omega_b * c.h ** 2)        # Mpc
    k_half = 1.0 / (0.43 * r_d * c.h)                                        # h/Mpc
    mid = 0.5 * (1.0 + alpha)
    assert abs(cm.eh_gamma_eff(c, k_half) / omh / mid - 1.0) < 0.01
    # the transition is monotone between the limits
    g = cm.eh_gamma_eff(c, np.logspace(-4, 1, 200))
    assert np.all(np.diff(g) < 0)


def test_zero_baryon_shape_against_bbks():
    c = W.COSMO.replace(omega_b=1e-9)
    k = np.logspace(-3, 1, 41)
    q = k * (c.t_cmb / 2.7) ** 2 / (c.omega_m * c.h)
    ratio = cm.eh_nowiggle_T(c, k) / bbks_T(q)
    assert np.all(np.abs(ratio - 1.0) < 0.05), ratio
    # baryons suppress small scales relative to the zero-baryon shape (alpha_Gamma < 1)
    assert np.all(cm.eh_nowiggle_T(W.COSMO, k[k > 0.1]) < cm.eh_nowiggle_T(c, k[k > 0.1]))
