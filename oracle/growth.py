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

Other triangle configurations (Sec. 3, the comparison of the full source term with
triangles): k1 = r k2 at angle theta between the vectors k1 and k2, k = |k1 + k2|, so
k2 = k / sqrt(r^2 + 1 + 2 r cos theta).  The D2 source is D1(k1) D1(k2) times the braces
of Eq. full-d2 for that triangle divided by sin^2 theta (the GR braces), so that every
configuration keeps the GR limit -3/7 D1^2 (a reading: the factorisation Psi2 = D2 grad phi2
takes the geometric sin^2 theta of each mode pair from the GR source S).  Variants:
  0 T1 (r = 1, 90 deg)   1 T2 (r = 1, 80 deg)   2 isosceles 70 deg
  3 r = 2, 80 deg        4 r = 2, 70 deg
  5 Winther: the T1 braces with D1(k)^2 in place of D1(k1) D1(k2)
  6 GR: the D2 equation with mu = 1 and the GR braces (scale-independent D2)
  7 isosceles 60 deg, the text's "equilateral" (k1 = k2, theta = 60 deg as printed)
  8 squeezed, k1 = 1e-3 k2 at 90 deg (the text's k1 ~ 0, k2 = k; k1 = 0 exactly leaves
    the k1.k2 terms 0/0, and at r = 1e-3 they are below 1e-6 of the braces)
  9 the LCDM fit Eq. lcdm-fit, D2 = -(3/7) D1(k,a)^2 Omega_m(a)^(-1/143) with the D1 of
    Eq. d1 (no D2 equation; tangent -(6/7) D1 dD1/dtheta Omega_m(a)^(-1/143)).

The k table is k_t = k_min (k_max/k_min)^(t/(n_k-1)); lookups interpolate
linearly in ln k between nodes and clamp outside the table (a reading: the
paper only says the solution is interpolated in k, Sec. 2.4).
"""
from __future__ import annotations

import numpy as np

from . import cosmology as cm

__all__ = ["k_table", "growth_tables", "interp_lnk", "d1_gr", "DEFAULT_STEPS", "VARIANTS", "BOUCHET",
           "triangle", "d2_braces"]

DEFAULT_STEPS = 2048


def k_table(n_k=512, k_min=1e-4, k_max=10.0):
    t = np.arange(n_k, dtype=np.float64)
    return k_min * (k_max / k_min) ** (t / (n_k - 1))


def _background(c, s):
    a = np.exp(s)
    om = cm.omega_m_a(c, a)
    damp = 2.0 - 1.5 * om        # 2 + dlnE/ds for E^2 = Om a^-3 + OL
    return a, om, damp


# (r = k1 / k2, angle between k1 and k2 in degrees); 5 Winther and 6 GR use the T1 geometry
VARIANTS = {0: (1.0, 90.0), 1: (1.0, 80.0), 2: (1.0, 70.0), 3: (2.0, 80.0), 4: (2.0, 70.0),
            5: (1.0, 90.0), 6: (1.0, 90.0), 7: (1.0, 60.0), 8: (1e-3, 90.0), 9: (1.0, 90.0)}
WINTHER, GR_D2, BOUCHET = 5, 6, 9


def triangle(k, variant):
    """(k1, k2, cos theta) of the variant's triangle with |k1 + k2| = k."""
    r, th = VARIANTS[variant]
    ct = np.cos(np.deg2rad(th)) if th != 90.0 else 0.0
    k2 = k / np.sqrt(r * r + 1.0 + 2.0 * r * ct)
    return r * k2, k2, ct


def d2_braces(c, k, a, variant, tangent=False):
    """Braces of Eq. full-d2 for the variant's triangle at |k1 + k2| = k, divided by
    sin^2 theta (and, with tangent, their d/dln|fR0|)."""
    k1, k2, ct = triangle(k, variant)
    r = VARIANTS[variant][0]
    c2 = ct * ct
    s2 = 1.0 - c2
    if c.fr0_abs == 0.0 or variant == GR_D2:
        one = np.ones_like(np.asarray(k, dtype=np.float64))
        return (one, 0.0 * one) if tangent else one
    q, q1, q2 = (k / a) ** 2, (k1 / a) ** 2, (k2 / a) ** 2
    msq = cm.m2(c, a)
    P, P1, P2 = q + msq, q1 + msq, q2 + msq
    mu, mu1, mu2 = 1.0 + q / (3.0 * P), 1.0 + q1 / (3.0 * P1), 1.0 + q2 / (3.0 * P2)
    G = msq / P
    lin = 2.0 * c2 * (mu1 + mu2 - 2.0) + (ct / r) * (mu1 - 1.0) + r * ct * (mu2 - 1.0)
    B = (2.0 / 27.0) * cm.four_pi_g_rho(c, a) * q * cm.M2(c, a) / (P * P1 * P2)
    br = mu - c2 * (mu1 + mu2 - mu) + G * lin - B
    if not tangent:
        return br / s2
    mut, mu1t, mu2t = q * msq / (3 * P * P), q1 * msq / (3 * P1 * P1), q2 * msq / (3 * P2 * P2)
    Gt = -G * q / P
    lint = 2.0 * c2 * (mu1t + mu2t) + (ct / r) * mu1t + r * ct * mu2t
    Bt = B * (-2.0 + msq / P + msq / P1 + msq / P2)
    brt = mut - c2 * (mu1t + mu2t - mut) + Gt * lin + G * lint - Bt
    return br / s2, brt / s2


def _rhs(c, k, s, y, variant=0):
    """y: (16, n_k) = [D1, D1_s, Da, Da_s, Db, Db_s, D2, D2_s] (Da = D1(k1), Db = D1(k2))
    and their theta-tangents, theta = ln|f_R0|."""
    a, om, damp = _background(c, s)
    k1, k2, _ = triangle(k, variant)
    D1, D1s, Da, Das, Db, Dbs, D2, D2s, Z1, Z1s, Za, Zas, Zb, Zbs, Z2, Z2s = y
    cc = 1.5 * om
    if c.fr0_abs == 0.0:
        mu_k = mu_a = mu_b = np.ones_like(k)
        mu_kt = mu_at = mu_bt = np.zeros_like(k)
    else:
        msq = cm.m2(c, a)
        def mus(kk):
            qq = (kk / a) ** 2
            pp = qq + msq
            return 1.0 + qq / (3.0 * pp), qq * msq / (3.0 * pp * pp)
        mu_k, mu_kt = mus(k)
        mu_a, mu_at = mus(k1)
        mu_b, mu_bt = mus(k2)
    if variant == GR_D2:       # D2 of GR: GR chains a, b and mu = 1 in its equation
        mu_a = mu_b = mu_2 = np.ones_like(k)
        mu_at = mu_bt = mu_2t = np.zeros_like(k)
    else:
        mu_2, mu_2t = mu_k, mu_kt
    src, srct = d2_braces(c, k, a, variant, tangent=True)
    if variant == WINTHER:     # D1(k)^2 in place of D1(k1) D1(k2)
        Pa, Pb, Pat, Pbt = D1, D1, Z1, Z1
    else:
        Pa, Pb, Pat, Pbt = Da, Db, Za, Zb
    dy = np.empty_like(y)
    dy[0] = D1s
    dy[1] = -damp * D1s + cc * mu_k * D1
    dy[2] = Das
    dy[3] = -damp * Das + cc * mu_a * Da
    dy[4] = Dbs
    dy[5] = -damp * Dbs + cc * mu_b * Db
    dy[6] = D2s
    dy[7] = -damp * D2s + cc * mu_2 * D2 - cc * Pa * Pb * src
    dy[8] = Z1s
    dy[9] = -damp * Z1s + cc * (mu_k * Z1 + mu_kt * D1)
    dy[10] = Zas
    dy[11] = -damp * Zas + cc * (mu_a * Za + mu_at * Da)
    dy[12] = Zbs
    dy[13] = -damp * Zbs + cc * (mu_b * Zb + mu_bt * Db)
    dy[14] = Z2s
    dy[15] = (-damp * Z2s + cc * (mu_2 * Z2 + mu_2t * D2)
              - cc * ((Pat * Pb + Pa * Pbt) * src + Pa * Pb * srct))
    return dy


def _rk4(c, k, a_in, a_out, n_steps, variant=0):
    s0, s1 = np.log(a_in), np.log(a_out)
    h = (s1 - s0) / n_steps
    y = np.zeros((16, k.size))
    y[0:6] = a_in
    y[6] = -3.0 / 7.0 * a_in ** 2
    y[7] = -6.0 / 7.0 * a_in ** 2
    for i in range(n_steps):
        s = s0 + i * h
        k1 = _rhs(c, k, s, y, variant)
        k2 = _rhs(c, k, s + 0.5 * h, y + 0.5 * h * k1, variant)
        k3 = _rhs(c, k, s + 0.5 * h, y + 0.5 * h * k2, variant)
        k4 = _rhs(c, k, s + h, y + h * k3, variant)
        y = y + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return y


def d1_gr(c, a_out=1.0, n_steps=DEFAULT_STEPS):
    """Unnormalised GR D1 at a_out from the EdS initial condition at c.a_init."""
    y = _rk4(c.replace(fr0_abs=0.0), np.array([1.0]), c.a_init, a_out, n_steps)
    return float(y[0, 0])


def growth_tables(c, a_out=1.0, k=None, n_steps=DEFAULT_STEPS, variant=None):
    """Returns dict with k, D1, D2 and dD1/dln|fR0|, dD2/dln|fR0| (all (n_k,)); D2 for
    the triangle variant (default: the cosmology's d2_variant, else T1)."""
    k = k_table() if k is None else np.asarray(k, dtype=np.float64)
    if variant is None:
        variant = int(getattr(c, "d2_variant", 0))
    y = _rk4(c, k, c.a_init, a_out, n_steps, variant)
    n1 = d1_gr(c, 1.0, n_steps)
    D1, dD1 = y[0] / n1, y[8] / n1
    if variant == BOUCHET:     # Eq. lcdm-fit with the scale-dependent D1 of Eq. d1
        f = cm.omega_m_a(c, a_out) ** (-1.0 / 143.0)
        return dict(k=k, D1=D1, D2=-3.0 / 7.0 * D1 * D1 * f, dD1=dD1, dD2=-6.0 / 7.0 * D1 * dD1 * f, norm=n1)
    return dict(k=k, D1=D1, D2=y[6] / n1 ** 2, dD1=dD1, dD2=y[14] / n1 ** 2, norm=n1)


def interp_lnk(table_k, table_v, kq):
    """Piecewise-linear interpolation in ln k, clamped to the end values."""
    lk = np.log(table_k)
    x = np.log(np.maximum(np.asarray(kq, dtype=np.float64), 1e-300))
    return np.interp(x, lk, table_v)
