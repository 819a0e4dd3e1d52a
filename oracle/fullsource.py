"""The full second-order source term of Sec. 3 (Eqs. full, s1-s4) and its ratio to GR
(oracle, float64; test infrastructure only).

Fields at scale factor a are evolved with the linear growth D1(k, a) (the paper's
prescription for this diagnostic):
  delta1(k) = D1(k,a) delta0(k),  phi(k) = delta1 / k^2   (phi_,ii = -delta1),
  phi_,ij(k) = -k_i k_j phi(k),   psi(k) = delta1(k) / Pi(k,a).
Real-space sources (sums over i, j = x, y, z):
  s1 = phi_,ij (mu * phi_,ij)            mu * f = IDFT[mu(k) DFT[f]]
  s2 = phi_,ii phi_,jj + phi_,ij phi_,ij  (a reading: the paper prints "-" between the two
                                           products; with "-" the sum S1 + S2 does not reduce
                                           to the GR source at mu = 1, with "+" it does and it
                                           reproduces the first bracket of Eq. full-d2)
  s3 = psi^2
  s4 = 2 phi_,ij psi_,ij + phi_,iij psi_,j,  phi_,iij = -delta1_,j
and in k space, with 4 pi G rho = 1.5 Om a^-3 (H0/c)^2 and 8 pi G rho / 3 = (2/3) 4 pi G rho:
  S1 = 4 pi G rho DFT[s1]
  S2 = -2 pi G rho mu(k) DFT[s2]
  S3 = (8 pi G rho / 3)^2 (M2 / 12) (k^2/a^2) / Pi(k) DFT[s3]
  S4 = -(8 pi G rho / 3) m^2 / (2 a^2) / Pi(k) DFT[s4]
The GR source (same delta0, fields evolved with D1_GR(a)) is S1 + S2 at mu = 1:
  S_GR = 2 pi G rho DFT[phi_,ij phi_,ij - (phi_,ii)^2].
Sec. 3 divides the MG source by the GR one mode by mode and bins the ratio in k
(mean and scatter per bin).  The ratio of two complex numbers is read as its real part,
modes with |S_GR| < 1e-8 of its rms are skipped (a reading: the paper says neither).

The T1 analytic curve (k1 = k2 = k/sqrt(2), theta = 90 deg) is the ratio of the braces
of Eq. full-d2 (times D1 D1) in MG and in GR for that triangle.
"""
from __future__ import annotations

import numpy as np

from . import cosmology as cm
from . import fft as offt
from . import growth as gr
from . import lpt2

__all__ = ["PAIRS", "source_terms", "source_ratio", "full_d2_kernel", "t1_ratio", "d1_gr_norm"]

PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def d1_gr_norm(c, a, n_steps=gr.DEFAULT_STEPS):
    """GR growth D1_GR(a) / D1_GR(1) (the normalisation of the growth tables)."""
    return gr.d1_gr(c, a, n_steps) / gr.d1_gr(c, 1.0, n_steps)


def source_terms(n, box, c, a, dk0, tables, d1gr):
    """S1, S2, S3, S4 and S_GR on the full complex grid for delta0(k) = dk0 (full spectrum,
    DC and Nyquist already zero), MG growth tables at a, and the GR growth d1gr = D1_GR(a)."""
    kv, k2, zero = lpt2.kvectors(n, box)
    kmag = np.sqrt(k2)
    safe = np.where(zero, 1.0, k2)
    kq = np.where(zero, 1.0, kmag)
    D1 = gr.interp_lnk(tables["k"], tables["D1"], kq)
    mu = cm.mu(c, kq, a)
    Pi = cm.Pi(c, kq, a)
    d1k = np.where(zero, 0.0, D1 * dk0)
    pot = np.where(zero, 0.0, d1k / safe)
    psi = np.where(zero, 0.0, d1k / Pi)
    pot0 = np.where(zero, 0.0, d1gr * dk0 / safe)

    def inv(f):
        return offt.ifftn(f).real

    s1 = np.zeros((n, n, n))
    s2b = np.zeros((n, n, n))
    s4 = np.zeros((n, n, n))
    tr = np.zeros((n, n, n))
    sgb = np.zeros((n, n, n))
    tr0 = np.zeros((n, n, n))
    for i, j in PAIRS:
        w = 1.0 if i == j else 2.0
        kk = -kv[i] * kv[j]
        phi = inv(kk * pot)
        s1 += w * phi * inv(kk * pot * mu)
        s2b += w * phi * phi
        s4 += 2.0 * w * phi * inv(kk * psi)
        phi0 = inv(kk * pot0)
        sgb += w * phi0 * phi0
        if i == j:
            tr += phi
            tr0 += phi0
    for j in range(3):
        s4 += -inv(1j * kv[j] * d1k) * inv(1j * kv[j] * psi)
    s2 = tr * tr + s2b
    s3 = inv(psi) ** 2
    fpg = cm.four_pi_g_rho(c, a)
    e = 2.0 / 3.0 * fpg
    if c.fr0_abs == 0.0:
        c3 = np.zeros_like(k2)
        c4 = np.zeros_like(k2)
    else:
        c3 = e * e * cm.M2(c, a) / 12.0 * (k2 / a ** 2) / Pi
        c4 = -e * cm.m2(c, a) / (2.0 * a ** 2) / Pi
    S1 = fpg * offt.fftn(s1)
    S2 = -0.5 * fpg * mu * offt.fftn(s2)
    S3 = c3 * offt.fftn(s3)
    S4 = c4 * offt.fftn(s4)
    SG = 0.5 * fpg * offt.fftn(sgb - tr0 * tr0)
    out = [np.where(zero, 0.0, X) for X in (S1, S2, S3, S4, SG)]
    return tuple(out)


def source_ratio(n, box, c, a, dk0, tables, d1gr, n_bins=32, rel_floor=1e-8):
    """Per-mode Re(S_MG / S_GR) binned in the P(k) shells: (mean, sigma, count) per bin."""
    S1, S2, S3, S4, SG = source_terms(n, box, c, a, dk0, tables, d1gr)
    smg = S1 + S2 + S3 + S4
    b = lpt2.shell_index(n, n_bins)
    absg = np.abs(SG)
    rms = np.sqrt(np.mean(absg[b >= 0] ** 2))
    ok = (b >= 0) & (absg >= rel_floor * rms)
    r = np.real(smg[ok] / SG[ok])
    bb = b[ok]
    cnt = np.bincount(bb, minlength=n_bins).astype(np.int64)
    s = np.bincount(bb, weights=r, minlength=n_bins)
    s2 = np.bincount(bb, weights=r * r, minlength=n_bins)
    with np.errstate(invalid="ignore", divide="ignore"):
        mean = np.where(cnt > 0, s / np.maximum(cnt, 1), 0.0)
        var = np.where(cnt > 0, s2 / np.maximum(cnt, 1) - mean * mean, 0.0)
    return mean, np.sqrt(np.maximum(var, 0.0)), cnt


def full_d2_kernel(c, a, k1, k2, D1a, D1b):
    """The right-hand side of Eq. full-d2 per unit delta(k1) delta(k2): 4 pi G rho D1(k1) D1(k2)
    times its braces, for wave vectors k1, k2 (3-vectors, h/Mpc) and growth values D1a, D1b."""
    k1 = np.asarray(k1, dtype=np.float64)
    k2 = np.asarray(k2, dtype=np.float64)
    k = k1 + k2
    q1, q2, q = k1 @ k1, k2 @ k2, k @ k
    dot = k1 @ k2
    cos2 = dot * dot / (q1 * q2)
    fpg = cm.four_pi_g_rho(c, a)
    m1, m2_, mk = (float(cm.mu(c, np.sqrt(x), a)) for x in (q1, q2, q))
    br = mk - cos2 * (m1 + m2_ - mk)
    if c.fr0_abs != 0.0:
        pk, p1, p2 = (float(cm.Pi(c, np.sqrt(x), a)) for x in (q, q1, q2))
        br += cm.m2(c, a) / pk * (2.0 * cos2 * (m1 + m2_ - 2.0) + dot / q1 * (m1 - 1.0) + dot / q2 * (m2_ - 1.0))
        br -= 2.0 / 27.0 * fpg * (q / a ** 2) * cm.M2(c, a) / (pk * p1 * p2)
    return fpg * D1a * D1b * br


def t1_ratio(c, a, k, tables, d1gr):
    """T1 triangle (k1 = k2 = k / sqrt 2, theta = 90 deg): ratio of the Eq. full-d2 source in MG
    to the one in GR, = (D1(k/sqrt2) / D1_GR)^2 [mu(k) - (2/27) 4 pi G rho (k^2/a^2) M2 /
    (Pi(k) Pi(k/sqrt2)^2)]."""
    k = np.asarray(k, dtype=np.float64)
    kh = k / np.sqrt(2.0)
    d1h = gr.interp_lnk(tables["k"], tables["D1"], kh)
    br = cm.mu(c, k, a)
    if c.fr0_abs != 0.0:
        br = br - 2.0 / 27.0 * cm.four_pi_g_rho(c, a) * (k / a) ** 2 * cm.M2(c, a) / (
            cm.Pi(c, k, a) * cm.Pi(c, kh, a) ** 2)
    return (d1h / d1gr) ** 2 * br
