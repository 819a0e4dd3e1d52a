"""Hand adjoint (vector-Jacobian product) of the forward 2LPT map (oracle, float64).

The paper has no gradients; this is the transpose of the forward steps of
`oracle.lpt2` taken in reverse order, written out plainly on full spectra:

  outputs  : CIC density contrast delta_rho(x) and shell P_b
  cotangent: g_density(x) = dL/d delta_rho(x), g_pk[b] = dL/dP_b
  inputs   : white noise w(x) and theta = ln|f_R0|

Convention: for real fields, a step y = IDFT[m(k) DFT[x]] has the transpose
x_bar = IDFT[conj(m(k)) DFT[y_bar]].  Spectral gradients h(k) are defined by
dL = sum_k Re[d(field_hat)(k) conj(h(k))].

  1. g_rho = g_density + N^3 IDFT[ w_b delta_rho_hat ],  w_b = 2 V g_pk[b] / (N^6 c_b)
     (dP_b / d delta_rho(x) = 2V/(N^6 c_b) Re sum_{k in b} conj(delta_hat) e^{-ikx})
  2. CIC transpose: dL/dx_p = sum over the 8 cells of g_rho(cell) dW/dx_p
  3. x = q + Psi  ->  g_Psi_c = dL/dx_c (plus any cotangent given for the positions)
  4. g_u(k) = sum_c conj(i k_c) DFT[g_Psi_c],  u = (D1 delta - D2 S_hat)/(k^2 N^3)
  5. h_Psi = D1 g_u /(k^2 N^3),  h_S = -D2 g_u /(k^2 N^3)
  6. dL/dtheta = sum_k Re[(dD1 delta - dD2 S_hat) conj(g_u)] /(k^2 N^3)
  7. g_S = N^3 IDFT[h_S];  g_phi_ij = g_S dS/dphi_ij  (S of Eq. second-ini)
  8. h_phi = sum_{i<=j} conj((i k_i)(i k_j)) DFT[g_phi_ij] /(k^2 N^3)
  9. g_w = N^3 IDFT[ s(k) (h_Psi + h_phi) ],  s = sqrt(P_lin N^3 / V)
"""
from __future__ import annotations

import numpy as np

from . import cosmology as cm
from . import fft as offt
from . import growth as gr
from . import lpt2

__all__ = ["forward_state", "vjp", "loss_and_cotangents"]


def forward_state(n, box, cosmo, noise, tables, n_shells=32):
    """Forward map keeping what the adjoint needs."""
    kv, k2, zero = lpt2.kvectors(n, box)
    kmag = np.sqrt(k2)
    amp = cm.pk_amplitude(cosmo)
    with np.errstate(divide="ignore", invalid="ignore"):
        pk = np.where(zero, 0.0, cm.pk_linear(cosmo, np.where(zero, 1.0, kmag), amp))
    s = np.sqrt(pk * n ** 3 / box ** 3)
    dk = offt.fftn(np.asarray(noise, dtype=np.float64)) * s
    dk[zero] = 0.0
    psi1, psi2, S, phi = lpt2.displacements(n, box, dk, tables)
    Sk = offt.fftn(S)
    pos = lpt2.positions(n, box, psi1 + psi2)
    dens = lpt2.cic_density(n, box, pos)
    P, kmean, cnt = lpt2.power_spectrum(n, box, dens, n_shells)
    return dict(s=s, dk=dk, S=S, Sk=Sk, phi=phi, pos=pos, density=dens, pk=P, n_modes=cnt,
                psi1=psi1, psi2=psi2)


def _cic_transpose(n, box, pos, g_rho):
    """dL/dx for each particle given dL/drho_contrast per cell (one particle per cell)."""
    u = pos * (n / box)
    i0 = np.floor(u)
    d = u - i0
    i0 = i0.astype(np.int64) % n
    g = g_rho.ravel() * (n ** 3 / pos.shape[1])
    out = np.zeros_like(pos)
    for ox in (0, 1):
        wx, dwx = (d[0], 1.0) if ox else (1.0 - d[0], -1.0)
        ix = (i0[0] + ox) % n
        for oy in (0, 1):
            wy, dwy = (d[1], 1.0) if oy else (1.0 - d[1], -1.0)
            iy = (i0[1] + oy) % n
            for oz in (0, 1):
                wz, dwz = (d[2], 1.0) if oz else (1.0 - d[2], -1.0)
                iz = (i0[2] + oz) % n
                gc = g[(ix * n + iy) * n + iz]
                out[0] += gc * dwx * wy * wz
                out[1] += gc * wx * dwy * wz
                out[2] += gc * wx * wy * dwz
    return out * (n / box)


def vjp(n, box, st, tables, g_density, g_pk, n_shells=32, g_pos=None):
    """Returns (g_noise (N,N,N), g_theta) for cotangents of (density, P(k)) and,
    optionally, of the positions (3, N^3)."""
    kv, k2, zero = lpt2.kvectors(n, box)
    kmag = np.sqrt(k2)
    safe = np.where(zero, 1.0, k2)
    n3 = float(n) ** 3
    # 1. density cotangent including the P(k) term
    b = lpt2.shell_index(n, n_shells)
    cnt = st["n_modes"]
    wb = np.zeros(n_shells)
    ok = cnt > 0
    wb[ok] = 2.0 * box ** 3 * np.asarray(g_pk)[ok] / (n3 * n3 * cnt[ok])
    wk = np.where(b >= 0, wb[np.maximum(b, 0)], 0.0)
    dhat = offt.fftn(st["density"])
    g_rho = np.asarray(g_density, dtype=np.float64) + n3 * offt.ifftn(wk * dhat).real
    # 2-3. CIC transpose -> g_Psi
    g_psi = _cic_transpose(n, box, st["pos"], g_rho)
    if g_pos is not None:
        g_psi = g_psi + np.asarray(g_pos, dtype=np.float64).reshape(3, -1)
    g_psi = g_psi.reshape(3, n, n, n)
    # 4. g_u
    G = [offt.fftn(g_psi[c]) for c in range(3)]
    g_u = sum(-1j * kv[c] * G[c] for c in range(3))
    g_u = np.where(zero, 0.0, g_u)
    d1 = gr.interp_lnk(tables["k"], tables["D1"], np.where(zero, 1.0, kmag))
    d2 = gr.interp_lnk(tables["k"], tables["D2"], np.where(zero, 1.0, kmag))
    t1 = gr.interp_lnk(tables["k"], tables["dD1"], np.where(zero, 1.0, kmag))
    t2 = gr.interp_lnk(tables["k"], tables["dD2"], np.where(zero, 1.0, kmag))
    # 5-6.
    h_psi = np.where(zero, 0.0, d1 * g_u / (safe * n3))
    h_S = np.where(zero, 0.0, -d2 * g_u / (safe * n3))
    g_theta = float(np.sum(np.where(zero, 0.0, ((t1 * st["dk"] - t2 * st["Sk"]) * np.conj(g_u)).real
                                    / (safe * n3))))
    # 7. source transpose
    g_S = n3 * offt.ifftn(h_S).real
    ph = st["phi"]
    dS = {"xx": ph["yy"] + ph["zz"], "yy": ph["xx"] + ph["zz"], "zz": ph["xx"] + ph["yy"],
          "xy": -2.0 * ph["xy"], "xz": -2.0 * ph["xz"], "yz": -2.0 * ph["yz"]}
    # 8. phi_ij transpose: conj((i k_i)(i k_j)) = -k_i k_j
    idx = {"x": 0, "y": 1, "z": 2}
    h_phi = np.zeros((n, n, n), dtype=np.complex128)
    for key, dsv in dS.items():
        m = -kv[idx[key[0]]] * kv[idx[key[1]]]
        h_phi += m * offt.fftn(g_S * dsv)
    h_phi = np.where(zero, 0.0, h_phi / (safe * n3))
    # 9. noise
    g_w = n3 * offt.ifftn(st["s"] * (h_psi + h_phi)).real
    return g_w, g_theta


def loss_and_cotangents(density, pk, target_density, target_pk, lam=1.0):
    """L = sum (delta - delta_t)^2 / N^3 + lam sum_b (ln P_b - ln P_t,b)^2 over non-empty shells,
    and its cotangents (g_density, g_pk)."""
    n3 = density.size
    diff = density - target_density
    ok = (pk > 0) & (target_pk > 0)
    lr = np.where(ok, np.log(np.where(ok, pk, 1.0)) - np.log(np.where(ok, target_pk, 1.0)), 0.0)
    L = float(np.sum(diff * diff) / n3 + lam * np.sum(lr * lr))
    g_density = 2.0 * diff / n3
    g_pk = np.where(ok, 2.0 * lam * lr / np.where(ok, pk, 1.0), 0.0)
    return L, g_density, g_pk
