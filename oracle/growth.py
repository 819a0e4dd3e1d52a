"""Scale-dependent growth factors D1(k,a) and D2(k,a) by classical RK4 (oracle, float64).

D1 (Eq. d1, read as (a^2 H^2 T - 4 pi G rho mu) D1 = 0; the printed a^2 H^2
also multiplying the mu term is dimensionally inconsistent).  With s = ln a and
E' = dE/da this is
    D1_ss + (2 + dlnE/ds) D1_s = 1.5 Omega_m(a) mu(k,a) D1 ,
with the Einstein-de Sitter growing mode at a_in as initial condition
(D1 = a_in, dD1/da = 1, Sec. 2.4) and the table normalised so that
D1(k -> 0, a = 1) = 1, i.e. divided by the GR solution at a = 1.

D2 for the orthogonal isosceles triangle T1 (k1 = k2 = k/sqrt2, theta = 90 deg,
the configuration the paper selects in Sec. 3).  At theta = 90 deg every
k1.k2 term of Eq. full-d2 vanishes and the braces reduce to
    mu(k) - (2/27) 4 pi G rho (k^2/a^2) M2(a) / (Pi(k) Pi(k/sqrt2)^2).
Sign reading: Eq. full-d2 with a + source gives +3/7 D1^2 in GR, while the LCDM
equation of Sec. 2.1 and the fit Eq. lcdm-fit use -3/7 D1^2; the oracle returns
D2 = -D2^(full-d2), so that GR gives -3/7 D1^2 (exact in Einstein-de Sitter) and
Psi2 = D2 * grad phi2 with laplacian(phi2) = second-order source.  Hence
    D2_ss + (2 + dlnE/ds) D2_s - 1.5 Om(a) mu(k) D2
        = -1.5 Om(a) D1(k/sqrt2)^2 [mu(k) - B(k,a)].
Initial condition (not given in the paper): the EdS growing mode
D2 = -(3/7) a_in^2, dD2/ds = -(6/7) a_in^2.  D2 is divided by the square of the
D1 normalisation.

Tangents: d/dtheta of every state, theta = ln|f_R0|, by forward sensitivity
(dm^2/dtheta = -m^2, dM2/dtheta = -2 M2), integrated by the same RK4.

The k table is k_t = k_min (k_max/k_min)^(t/(n_k-1)); lookups interpolate
linearly in ln k between nodes and clamp outside the table (a reading: the
paper only says the solution is interpolated in k, Sec. 2.4).
"""
from __future__ import annotations

import numpy as np

from . import cosmology as cm

__all__ = ["k_table", "growth_tables", "interp_lnk", "d1_gr", "DEFAULT_STEPS"]

DEFAULT_STEPS = 2048


def k_table(n_k=512, k_min=1e-4, k_max=10.0):
    t = np.arange(n_k, dtype=np.float64)
    return k_min * (k_max / k_min) ** (t / (n_k - 1))


def _background(c, s):
    a = np.exp(s)
    om = cm.omega_m_a(c, a)
    damp = 2.0 - 1.5 * om        # 2 + dlnE/ds for E^2 = Om a^-3 + OL
    return a, om, damp


def _rhs(c, k, s, y):
    """y: (12, n_k) = [D1, D1_s, D1h, D1h_s, D2, D2_s] and their theta-tangents."""
    a, om, damp = _background(c, s)
    kh = k / np.sqrt(2.0)
    D1, D1s, D1h, D1hs, D2, D2s, Z1, Z1s, Z1h, Z1hs, Z2, Z2s = y
    cc = 1.5 * om
    if c.fr0_abs == 0.0:
        mu_k = np.ones_like(k)
        mu_h = np.ones_like(k)
        mu_kt = mu_ht = B = Bt = np.zeros_like(k)
    else:
        q, qh = (k / a) ** 2, (kh / a) ** 2
        msq = cm.m2(c, a)
        Pk, Ph = q + msq, qh + msq
        mu_k = 1.0 + q / (3.0 * Pk)
        mu_h = 1.0 + qh / (3.0 * Ph)
        mu_kt = q * msq / (3.0 * Pk * Pk)
        mu_ht = qh * msq / (3.0 * Ph * Ph)
        B = (2.0 / 27.0) * cm.four_pi_g_rho(c, a) * q * cm.M2(c, a) / (Pk * Ph * Ph)
        Bt = B * (-2.0 + msq / Pk + 2.0 * msq / Ph)
    src = mu_k - B
    dy = np.empty_like(y)
    dy[0] = D1s
    dy[1] = -damp * D1s + cc * mu_k * D1
    dy[2] = D1hs
    dy[3] = -damp * D1hs + cc * mu_h * D1h
    dy[4] = D2s
    dy[5] = -damp * D2s + cc * mu_k * D2 - cc * D1h * D1h * src
    dy[6] = Z1s
    dy[7] = -damp * Z1s + cc * (mu_k * Z1 + mu_kt * D1)
    dy[8] = Z1hs
    dy[9] = -damp * Z1hs + cc * (mu_h * Z1h + mu_ht * D1h)
    dy[10] = Z2s
    dy[11] = (-damp * Z2s + cc * (mu_k * Z2 + mu_kt * D2)
              - cc * (2.0 * D1h * Z1h * src + D1h * D1h * (mu_kt - Bt)))
    return dy


def _rk4(c, k, a_in, a_out, n_steps):
    s0, s1 = np.log(a_in), np.log(a_out)
    h = (s1 - s0) / n_steps
    y = np.zeros((12, k.size))
    y[0] = y[1] = y[2] = y[3] = a_in
    y[4] = -3.0 / 7.0 * a_in ** 2
    y[5] = -6.0 / 7.0 * a_in ** 2
    for i in range(n_steps):
        s = s0 + i * h
        k1 = _rhs(c, k, s, y)
        k2 = _rhs(c, k, s + 0.5 * h, y + 0.5 * h * k1)
        k3 = _rhs(c, k, s + 0.5 * h, y + 0.5 * h * k2)
        k4 = _rhs(c, k, s + h, y + h * k3)
        y = y + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return y


def d1_gr(c, a_out=1.0, n_steps=DEFAULT_STEPS):
    """Unnormalised GR D1 at a_out from the EdS initial condition at c.a_init."""
    y = _rk4(c.replace(fr0_abs=0.0), np.array([1.0]), c.a_init, a_out, n_steps)
    return float(y[0, 0])


def growth_tables(c, a_out=1.0, k=None, n_steps=DEFAULT_STEPS):
    """Returns dict with k, D1, D2 and dD1/dln|fR0|, dD2/dln|fR0| (all (n_k,))."""
    k = k_table() if k is None else np.asarray(k, dtype=np.float64)
    y = _rk4(c, k, c.a_init, a_out, n_steps)
    n1 = d1_gr(c, 1.0, n_steps)
    return dict(k=k, D1=y[0] / n1, D2=y[4] / n1 ** 2,
                dD1=y[6] / n1, dD2=y[10] / n1 ** 2, norm=n1)


def interp_lnk(table_k, table_v, kq):
    """Piecewise-linear interpolation in ln k, clamped to the end values."""
    lk = np.log(table_k)
    x = np.log(np.maximum(np.asarray(kq, dtype=np.float64), 1e-300))
    return np.interp(x, lk, table_v)
