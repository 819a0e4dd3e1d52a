"""The 2LPT f(R) displacement pipeline, step by step, in float64 (oracle).

Steps, in the paper's order (Sec. 3 method paragraph and Sec. 2):
  1. noise w(x) -> delta(k) = DFT[w] * sqrt(P_lin(k) N^3 / V), DC and every
     Nyquist plane (|n_i| = N/2) set to 0 (a reading: the paper fixes no
     discretisation).                                  "linear density field", Sec. 3
  2. Psi1(k) = i k D1(k,a) delta(k) / k^2                 phi1_,ii = -delta, Sec. 2.1; Eq. d1
  3. phi_ij(k) = -k_i k_j delta(k) / k^2 (six fields, taken at the initial
     time: the space part is the GR one, Sec. 2.4 factorisation)
  4. S(x) = sum_{i<j} (phi_ii phi_jj - phi_ij^2)          Eq. second-ini
  5. phi2(k) = -S(k) D2(k,a) / k^2, DC and Nyquist planes set to 0;
     Psi2(k) = i k phi2(k)                                 Sec. 2.4 factorisation
  6. x = q + Psi1 + Psi2, q the cell corner, periodic     Eq. position; Sec. 4
  7. CIC density contrast and P(k) in linear shells       (halo P(k) analogue, Sec. 4)

Grid conventions: index i in [0, N) is the mode n = i for i < N/2, i - N
otherwise; k = 2 pi n / L; arrays are (x, y, z) with z fastest.
"""
from __future__ import annotations

import numpy as np

from . import cosmology as cm
from . import fft as offt
from . import growth as gr
from . import philox

__all__ = ["mode_numbers", "kvectors", "delta_k", "displacements", "source_term",
           "positions", "cic_density", "power_spectrum", "run", "shell_index"]


def mode_numbers(n: int) -> np.ndarray:
    i = np.arange(n)
    return np.where(i < n // 2, i, i - n)


def kvectors(n: int, box: float):
    """(kx, ky, kz) broadcastable arrays, k^2, and the Nyquist/DC mask (True = zeroed)."""
    m = mode_numbers(n)
    kf = 2.0 * np.pi / box
    kx = (kf * m)[:, None, None]
    ky = (kf * m)[None, :, None]
    kz = (kf * m)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    nyq = (np.abs(m) == n // 2)
    zero = nyq[:, None, None] | nyq[None, :, None] | nyq[None, None, :]
    zero = zero | (k2 == 0.0)
    return (kx, ky, kz), k2, zero


def delta_k(n: int, box: float, cosmo, noise: np.ndarray) -> np.ndarray:
    """Step 1: Gaussian delta(k) from unit white noise (full complex spectrum)."""
    _, k2, zero = kvectors(n, box)
    kmag = np.sqrt(k2)
    amp = cm.pk_amplitude(cosmo)
    with np.errstate(divide="ignore", invalid="ignore"):
        pk = np.where(zero, 0.0, cm.pk_linear(cosmo, np.where(zero, 1.0, kmag), amp))
    scale = np.sqrt(pk * n ** 3 / box ** 3)
    d = offt.fftn(np.asarray(noise, dtype=np.float64)) * scale
    d[zero] = 0.0
    return d


def source_term(phi: dict) -> np.ndarray:
    """Eq. second-ini: S = sum_{i<j} (phi_ii phi_jj - phi_ij^2)."""
    return (phi["xx"] * phi["yy"] + phi["xx"] * phi["zz"] + phi["yy"] * phi["zz"]
            - phi["xy"] ** 2 - phi["xz"] ** 2 - phi["yz"] ** 2)


def displacements(n: int, box: float, dk: np.ndarray, tables: dict):
    """Steps 2-5. Returns Psi1 (3,N,N,N), Psi2 (3,N,N,N), S (N,N,N), phi dict."""
    kv, k2, zero = kvectors(n, box)
    kmag = np.sqrt(k2)
    safe = np.where(zero, 1.0, k2)
    d1 = gr.interp_lnk(tables["k"], tables["D1"], np.where(zero, 1.0, kmag))
    d2 = gr.interp_lnk(tables["k"], tables["D2"], np.where(zero, 1.0, kmag))
    pot1 = np.where(zero, 0.0, dk / safe)                      # phi1(k) = delta/k^2
    psi1 = np.stack([offt.ifftn(1j * kc * d1 * pot1).real for kc in kv])
    names = {"x": 0, "y": 1, "z": 2}
    phi = {}
    for a, b in ("xx", "yy", "zz", "xy", "xz", "yz"):
        phi[a + b] = offt.ifftn(-kv[names[a]] * kv[names[b]] * pot1).real
    S = source_term(phi)
    Sk = offt.fftn(S)
    phi2 = np.where(zero, 0.0, -Sk * d2 / safe)
    psi2 = np.stack([offt.ifftn(1j * kc * phi2).real for kc in kv])
    return psi1, psi2, S, phi


def positions(n: int, box: float, psi: np.ndarray) -> np.ndarray:
    """Eq. position: x = q + Psi, q = cell corner, wrapped into [0, L). Shape (3, N^3)."""
    q = np.indices((n, n, n)).reshape(3, -1).astype(np.float64) * (box / n)
    return np.mod(q + psi.reshape(3, -1), box)


def cic_density(n: int, box: float, pos: np.ndarray) -> np.ndarray:
    """Cloud-in-cell deposit of unit-mass particles; returns delta = rho N^3/N_p - 1."""
    u = np.asarray(pos, dtype=np.float64) * (n / box)
    i0 = np.floor(u)
    d = u - i0
    i0 = i0.astype(np.int64) % n
    rho = np.zeros(n ** 3)
    for ox in (0, 1):
        wx = d[0] if ox else 1.0 - d[0]
        ix = (i0[0] + ox) % n
        for oy in (0, 1):
            wy = d[1] if oy else 1.0 - d[1]
            iy = (i0[1] + oy) % n
            for oz in (0, 1):
                wz = d[2] if oz else 1.0 - d[2]
                iz = (i0[2] + oz) % n
                rho += np.bincount((ix * n + iy) * n + iz, weights=wx * wy * wz, minlength=n ** 3)
    npart = pos.shape[1]
    return (rho * (n ** 3 / npart) - 1.0).reshape(n, n, n)


def shell_index(n: int, n_shells: int) -> np.ndarray:
    """Exact integer shell of every full-grid mode: b = floor(2 n_shells |n| / N)
    for 0 < |n| < N/2, else -1.  Shell width k_Ny / n_shells (linear, [0, k_Ny))."""
    m = mode_numbers(n).astype(np.int64)
    n2 = m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2
    M = 4 * n_shells * n_shells * n2
    r = np.floor(np.sqrt(M.astype(np.float64))).astype(np.int64)
    r = np.where((r + 1) ** 2 <= M, r + 1, r)
    r = np.where(r * r > M, r - 1, r)                          # r = isqrt(M)
    b = r // n
    ok = (n2 > 0) & (4 * n2 < n * n)
    return np.where(ok, b, -1)


def power_spectrum(n: int, box: float, delta: np.ndarray, n_shells: int = 32):
    """P_b = mean over shell b of V |delta(k)|^2 / N^6; also mean |k| and mode count."""
    dk = offt.fftn(delta)
    p = box ** 3 * np.abs(dk) ** 2 / float(n) ** 6
    b = shell_index(n, n_shells).ravel()
    _, k2, _ = kvectors(n, box)
    kmag = np.sqrt(k2).ravel()
    sel = b >= 0
    cnt = np.bincount(b[sel], minlength=n_shells).astype(np.int64)
    psum = np.bincount(b[sel], weights=p.ravel()[sel], minlength=n_shells)
    ksum = np.bincount(b[sel], weights=kmag[sel], minlength=n_shells)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(cnt > 0, psum / np.maximum(cnt, 1), 0.0), \
            np.where(cnt > 0, ksum / np.maximum(cnt, 1), 0.0), cnt


def run(n: int, box: float, cosmo, seed: int | None = None, noise=None, a_out: float = 1.0,
        n_shells: int = 32, tables: dict | None = None, n_steps: int = gr.DEFAULT_STEPS):
    """The whole forward path for one instance. Returns a dict of every output."""
    if noise is None:
        noise = philox.gaussian_noise(n, seed).reshape(n, n, n)
    if tables is None:
        tables = gr.growth_tables(cosmo, a_out, n_steps=n_steps)
    dk = delta_k(n, box, cosmo, noise)
    psi1, psi2, S, _ = displacements(n, box, dk, tables)
    pos = positions(n, box, psi1 + psi2)
    dens = cic_density(n, box, pos)
    pk, kmean, cnt = power_spectrum(n, box, dens, n_shells)
    return dict(noise=noise, delta_k=dk, psi1=psi1, psi2=psi2, S=S, pos=pos,
                density=dens, pk=pk, k_mean=kmean, n_modes=cnt, tables=tables)
