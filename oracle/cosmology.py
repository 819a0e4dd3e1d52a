"""Background, Hu-Sawicki f(R) functions and the linear power spectrum (oracle, float64).

Units: lengths Mpc/h, k in h/Mpc, H0/c = 1/2997.92458 h/Mpc.  Flat background
E^2(a) = Omega_m a^-3 + Omega_L (no radiation, Omega_m + Omega_L = 1, Sec. 4).

  4 pi G rho(a) = 1.5 Omega_m a^-3 (H0/c)^2                      (Poisson, Sec. 2.2)
  M1(a) = 3/2 (H0/c)^2 (Om a^-3 + 4 OL)^3 / (|fR0| (Om + 4 OL)^2)   Eq. mihusawicki
  M2(a) = 9/4 (H0/c)^2 (Om a^-3 + 4 OL)^5 / (|fR0|^2 (Om + 4 OL)^4) Eq. mihusawicki
  m^2(a) = M1(a) / 3                                                Sec. 2.4
  Pi(k,a) = k^2/a^2 + m^2(a)                                        Sec. 3
  mu(k,a) = 1 + (1/3) (k^2/a^2) / Pi(k,a)                           Sec. 2.4
|fR0| = 0 selects GR: mu = 1 and no M2 term.

Linear P(k) (z = 0): Eisenstein & Hu (1998) zero-baryon ("no-wiggle") transfer
function, their Eqs. 26 and 28-31, written from that paper, times k^n_s, with the
amplitude fixed by sigma_8 (top-hat of radius 8 Mpc/h, Simpson rule in ln k).
"""
from __future__ import annotations

import numpy as np

H0_OVER_C = 1.0 / 2997.92458

__all__ = ["H0_OVER_C", "E2", "omega_m_a", "four_pi_g_rho", "m2", "M2", "Pi", "mu",
           "eh_sound_horizon", "eh_alpha_gamma", "eh_gamma_eff", "eh_T0", "eh_nowiggle_T", "pk_shape",
           "sigma_r_sq", "pk_amplitude", "pk_linear"]


def E2(c, a):
    return c.omega_m * a ** -3 + c.omega_l


def omega_m_a(c, a):
    return c.omega_m * a ** -3 / E2(c, a)


def four_pi_g_rho(c, a):
    return 1.5 * c.omega_m * a ** -3 * H0_OVER_C ** 2


def _x(c, a):
    return c.omega_m * a ** -3 + 4.0 * c.omega_l


def m2(c, a):
    """Scalar-field mass squared m^2 = M1/3, (h/Mpc)^2 (Eq. mihusawicki, n = 1)."""
    x0 = c.omega_m + 4.0 * c.omega_l
    return 0.5 * H0_OVER_C ** 2 * _x(c, a) ** 3 / (c.fr0_abs * x0 ** 2)


def M2(c, a):
    """Second-order self-interaction coefficient M2(a), (h/Mpc)^2 (Eq. mihusawicki)."""
    x0 = c.omega_m + 4.0 * c.omega_l
    return 2.25 * H0_OVER_C ** 2 * _x(c, a) ** 5 / (c.fr0_abs ** 2 * x0 ** 4)


def Pi(c, k, a):
    return (k / a) ** 2 + m2(c, a)


def mu(c, k, a):
    """mu(k,a) of Sec. 2.4; exactly 1 in GR (|fR0| = 0)."""
    if c.fr0_abs == 0.0:
        return np.ones_like(np.asarray(k, dtype=np.float64))
    q = (k / a) ** 2
    return 1.0 + q / (3.0 * (q + m2(c, a)))


def eh_sound_horizon(c):
    """Sound horizon fit s (Mpc, not Mpc/h) of Eisenstein & Hu (1998) Eq. 26."""
    wm = c.omega_m * c.h * c.h
    wb = c.omega_b * c.h * c.h
    return 44.5 * np.log(9.83 / wm) / np.sqrt(1.0 + 10.0 * wb ** 0.75)


def eh_alpha_gamma(c):
    """Small-scale baryon suppression alpha_Gamma of Eisenstein & Hu (1998) Eq. 31."""
    wm = c.omega_m * c.h * c.h
    fb = c.omega_b / c.omega_m
    return 1.0 - 0.328 * np.log(431.0 * wm) * fb + 0.38 * np.log(22.3 * wm) * fb * fb


def eh_gamma_eff(c, k):
    """Effective shape Gamma_eff(k) of Eisenstein & Hu (1998) Eq. 30, k in h/Mpc.

    The equation is written for k in Mpc^-1 (s is in Mpc): k_mpc = k h."""
    k = np.asarray(k, dtype=np.float64)
    alpha = eh_alpha_gamma(c)
    k_mpc = k * c.h
    return c.omega_m * c.h * (alpha + (1.0 - alpha) / (1.0 + (0.43 * k_mpc * eh_sound_horizon(c)) ** 4))


def eh_T0(q):
    """Zero-baryon transfer function of Eisenstein & Hu (1998) Eq. 29 at their q (Eq. 28)."""
    q = np.asarray(q, dtype=np.float64)
    L0 = np.log(2.0 * np.e + 1.8 * q)
    C0 = 14.2 + 731.0 / (1.0 + 62.5 * q)
    return L0 / (L0 + C0 * q * q)


def eh_nowiggle_T(c, k):
    """Eisenstein & Hu (1998) no-wiggle transfer function T0(k), k in h/Mpc (Eqs. 26, 28-31)."""
    k = np.asarray(k, dtype=np.float64)
    theta = c.t_cmb / 2.7
    q = k * theta * theta / eh_gamma_eff(c, k)                                # Eq. 28
    return eh_T0(q)


def pk_shape(c, k):
    return np.asarray(k, dtype=np.float64) ** c.n_s * eh_nowiggle_T(c, k) ** 2


def tophat_W(x):
    x = np.asarray(x, dtype=np.float64)
    return 3.0 * (np.sin(x) - x * np.cos(x)) / x ** 3


def sigma_r_sq(pk_fn, r=8.0, lnk_lo=np.log(1e-5), lnk_hi=np.log(1e3), n=20001):
    """sigma^2(R) = 1/(2 pi^2) int k^3 P(k) W(kR)^2 dln k, composite Simpson (n odd)."""
    lnk = np.linspace(lnk_lo, lnk_hi, n)
    k = np.exp(lnk)
    f = k ** 3 * pk_fn(k) * tophat_W(k * r) ** 2 / (2.0 * np.pi ** 2)
    h = (lnk_hi - lnk_lo) / (n - 1)
    w = np.ones(n)
    w[1:-1:2] = 4.0
    w[2:-1:2] = 2.0
    return h / 3.0 * np.dot(w, f)


def pk_amplitude(c):
    """A such that A k^n_s T(k)^2 has sigma_8 = c.sigma8."""
    return c.sigma8 ** 2 / sigma_r_sq(lambda k: pk_shape(c, k))


def pk_linear(c, k, amp=None):
    """Linear LCDM P(k) at z = 0, (Mpc/h)^3."""
    amp = pk_amplitude(c) if amp is None else amp
    return amp * pk_shape(c, k)
