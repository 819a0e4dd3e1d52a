"""Pins of the oracle's scalar-field coefficients m^2(a) (M1 = 3 m^2) and M2(a) against
their definition rather than their printed closed form.

Sec. 2.2 defines M_k = d^k R / d f_R^k at the background f_R (Eq. mg-pot-exp) for the
Hu-Sawicki model f(R) = -beta^2 c1 (R/beta^2)^n / (c2 (R/beta^2)^n + 1) with beta^2 =
H0^2 Omega_m, c1/c2 = 6 Omega_L / Omega_m and n = 1 (Eq. husawicki), and prints M1, M2 in
the large-curvature limit (Eq. mihusawicki).  Here f(R) is differentiated symbolically,
c2 is fixed by f_R(R0) = -|f_R0| at the LCDM background curvature R = 3 H0^2 (Omega_m a^-3 +
4 Omega_L), and the inverse-function derivatives
    dR/df_R = 1 / f_RR,    d^2R/df_R^2 = -f_RRR / f_RR^3
are evaluated at the background curvature of each a.  They differ from the limit forms
only by terms of relative order 1/(c2 R/beta^2), a few |f_R0|, so a wrong coefficient or
exponent in the oracle fails by far more than the tolerance."""
import numpy as np
import pytest

import workloads as W
from oracle import cosmology as cm

sympy = pytest.importorskip("sympy")


def _model_derivatives(c, a_values):
    H0 = cm.H0_OVER_C
    om, ol = c.omega_m, c.omega_l
    beta2 = H0 * H0 * om
    R, c2s = sympy.symbols("R c2", positive=True)
    c1s = 6.0 * ol / om * c2s
    f = -beta2 * c1s * (R / beta2) / (c2s * (R / beta2) + 1)
    fR = sympy.diff(f, R)
    fRR = sympy.diff(fR, R)
    fRRR = sympy.diff(fRR, R)
    R0 = 3.0 * H0 * H0 * (om + 4.0 * ol)
    # c2 on the large-curvature branch: f_R(R0) = -|f_R0|, bracketed between the limit
    # estimate / 2 and * 2 (f_R(R0) is monotone in c2 there)
    g = sympy.lambdify(c2s, fR.subs(R, R0) + c.fr0_abs, "mpmath")
    y0 = R0 / beta2
    est = 6.0 * ol / om / (c.fr0_abs * y0 * y0)
    import mpmath
    mpmath.mp.dps = 40
    c2 = float(mpmath.findroot(g, (0.5 * est, 2.0 * est), solver="bisect"))
    d2 = sympy.lambdify(R, fRR.subs(c2s, c2), "mpmath")
    d3 = sympy.lambdify(R, fRRR.subs(c2s, c2), "mpmath")
    out = []
    for a in a_values:
        Rb = 3.0 * H0 * H0 * (om * a ** -3 + 4.0 * ol)
        frr, frrr = d2(Rb), d3(Rb)
        out.append((float(1 / frr), float(-frrr / frr ** 3)))
    return np.array(out)


@pytest.mark.parametrize("fr0", [1e-4, 1e-5, 1e-6])
def test_m1_m2_are_the_model_derivatives(fr0):
    c = W.COSMO.replace(fr0_abs=fr0)
    a = np.array([0.1, 0.3, 0.6, 1.0])
    mk = _model_derivatives(c, a)
    m1 = np.array([3.0 * cm.m2(c, x) for x in a])
    m2 = np.array([cm.M2(c, x) for x in a])
    tol = 30.0 * fr0
    np.testing.assert_allclose(m1, mk[:, 0], rtol=tol)
    np.testing.assert_allclose(m2, mk[:, 1], rtol=tol)
    # the large-curvature forms are approached from one side as |f_R0| -> 0
    assert np.all(mk[:, 0] > 0) and np.all(mk[:, 1] > 0)
