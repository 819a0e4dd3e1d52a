"""A float64 forward map for finite differences of the adjoint (test infrastructure only).

The oracle (`oracle/lpt2.py`) runs the method step by step on the CPU with its own FFT;
at 512^3 the 130 forward evaluations that central differences on 64 noise cells need
would take hours there.  This module restates the same steps, in float64 and in the
oracle's conventions, with torch tensors on the GPU and library FFTs as steps:

  delta(k) = DFT[w] sqrt(P N^3 / V) (DC and every Nyquist plane zero)
  Psi(k)   = i k (D1 delta / k^2 - D2 S(k) / k^2),  S = sum_{i<j} (phi_ii phi_jj - phi_ij^2),
             phi_ij(k) = -k_i k_j delta / k^2          (Sec. 2.1 Eq. second-ini, Sec. 2.4)
  x        = q + Psi, CIC density contrast, shell P(k), and the loss of the
             differentiable configuration L = sum (delta - delta_t)^2 / N^3 + sum_b (ln P_b -
             ln P_t,b)^2.

P_lin and the growth tables D1, D2 come from the oracle (evaluated once per distinct
|n|^2).  The CIC deposit can be given the lower-corner cells of every particle
(`base`): then the weights are the linear functions 1 - d, d of d = u - base even
where u has left that cell, so that the loss is smooth in the noise around the point
where `base` was taken and central differences measure the derivative of that
branch of the piecewise-linear deposit, the one the adjoint differentiates.
It is pinned against the oracle's forward state, adjoint and CIC transpose in
tests/test_fd64_cpu.py.
"""
from __future__ import annotations

import numpy as np
import torch

from oracle import cosmology as cm
from oracle import growth as gr


def _isqrt(M: torch.Tensor) -> torch.Tensor:
    r = torch.floor(torch.sqrt(M.double())).long()
    r = torch.where((r + 1) ** 2 <= M, r + 1, r)
    return torch.where(r * r > M, r - 1, r)


class Forward64:
    def __init__(self, n: int, box: float, cosmo, tables: dict, n_shells: int = 32, device="cuda"):
        self.n, self.box, self.ns, self.dev = n, float(box), n_shells, device
        i = torch.arange(n, device=device)
        m = torch.where(i < n // 2, i, i - n)
        mz = torch.arange(n // 2 + 1, device=device)
        n2 = m[:, None, None] ** 2 + m[None, :, None] ** 2 + mz[None, None, :] ** 2
        zero = ((m.abs() == n // 2)[:, None, None] | (m.abs() == n // 2)[None, :, None]
                | (mz == n // 2)[None, None, :] | (n2 == 0))
        kf = 2.0 * np.pi / box
        self.kx = (kf * m.double())[:, None, None]
        self.ky = (kf * m.double())[None, :, None]
        self.kz = (kf * mz.double())[None, None, :]
        # radial factors per distinct |n|^2 (float64, oracle formulas)
        j = np.arange(3 * (n // 2) ** 2 + 1, dtype=np.float64)
        k = kf * np.sqrt(np.maximum(j, 1.0))
        amp = cm.pk_amplitude(cosmo)
        s = np.sqrt(cm.pk_linear(cosmo, k, amp) * n ** 3 / box ** 3)
        inv_k2 = 1.0 / (k * k)
        self.set_tables(tables, k, inv_k2)
        self.s = torch.where(zero, 0.0, torch.from_numpy(s).to(device)[n2])
        self.n2, self.zero = n2, zero
        # P(k) shells of the half spectrum: kz = 0 counts once, 0 < kz < N/2 twice
        M = 4 * n_shells * n_shells * n2
        b = torch.where((n2 > 0) & (4 * n2 < n * n), _isqrt(M) // n, -1)
        w = torch.where(mz == 0, 1.0, 2.0).double()[None, None, :].expand_as(b)
        self.sel = b >= 0
        self.b = b[self.sel]
        self.w = w[self.sel]
        self.count = torch.bincount(self.b, weights=self.w, minlength=n_shells)
        q = torch.stack(torch.meshgrid(i, i, i, indexing="ij")).double()
        self.q = q.reshape(3, -1)

    def set_tables(self, tables: dict, k=None, inv_k2=None):
        """Growth tables (oracle.growth.growth_tables output) of the forward map."""
        n, kf = self.n, 2.0 * np.pi / self.box
        if k is None:
            j = np.arange(3 * (n // 2) ** 2 + 1, dtype=np.float64)
            k = kf * np.sqrt(np.maximum(j, 1.0))
            inv_k2 = 1.0 / (k * k)
        d1 = gr.interp_lnk(tables["k"], tables["D1"], k)
        d2 = gr.interp_lnk(tables["k"], tables["D2"], k)
        self._g1 = torch.from_numpy(d1 * inv_k2).to(self.dev)
        self._g2 = torch.from_numpy(d2 * inv_k2).to(self.dev)
        self._ik2 = torch.from_numpy(inv_k2).to(self.dev)
        if hasattr(self, "n2"):
            self._apply_tables()

    def _apply_tables(self):
        self.g1 = torch.where(self.zero, 0.0, self._g1[self.n2])   # D1 / k^2
        self.g2 = torch.where(self.zero, 0.0, self._g2[self.n2])   # D2 / k^2
        self.ik2 = torch.where(self.zero, 0.0, self._ik2[self.n2])

    def displacement_cells(self, noise: torch.Tensor) -> torch.Tensor:
        """Psi1 + Psi2 in cell units, shape (3, N^3)."""
        if not hasattr(self, "g1"):
            self._apply_tables()
        n = self.n
        sh = (n, n, n)
        dk = torch.fft.rfftn(noise.double().reshape(sh)) * self.s
        pot = dk * self.ik2                                           # phi1 = delta / k^2
        kv = (self.kx, self.ky, self.kz)

        def phi(a, b):
            return torch.fft.irfftn(-kv[a] * kv[b] * pot, s=sh)
        S = phi(0, 0)
        T = S.clone()
        f = phi(1, 1)
        S *= f
        T += f
        f = phi(2, 2)
        S += T * f
        del T
        for a, b in ((0, 1), (0, 2), (1, 2)):
            f = phi(a, b)
            S -= f * f
        del f
        Sk = torch.fft.rfftn(S)
        del S
        u = dk * self.g1 - Sk * self.g2                               # D1 delta/k^2 - D2 S/k^2
        cell = self.box / n
        return torch.stack([torch.fft.irfftn(1j * kc * u, s=sh).reshape(-1) for kc in kv]) / cell

    def lattice_coords(self, noise: torch.Tensor) -> torch.Tensor:
        """u = q + Psi / cell (cells, not wrapped), shape (3, N^3)."""
        return self.q + self.displacement_cells(noise)

    def density(self, u: torch.Tensor, base: torch.Tensor | None = None) -> torch.Tensor:
        """CIC density contrast of particles at u (cells); base = lower-corner cells (int64,
        same shape) to deposit with, default floor(u)."""
        n = self.n
        if base is None:
            base = torch.floor(u).long()
        d = u - base
        i0 = torch.remainder(base, n)
        rho = torch.zeros(n ** 3, dtype=torch.float64, device=self.dev)
        for ox in (0, 1):
            wx = d[0] if ox else 1.0 - d[0]
            ix = (i0[0] + ox) % n
            for oy in (0, 1):
                wy = d[1] if oy else 1.0 - d[1]
                iy = (i0[1] + oy) % n
                for oz in (0, 1):
                    wz = d[2] if oz else 1.0 - d[2]
                    iz = (i0[2] + oz) % n
                    rho.index_add_(0, (ix * n + iy) * n + iz, wx * wy * wz)
        return (rho * (n ** 3 / u.shape[1]) - 1.0).reshape(n, n, n)

    def power(self, density: torch.Tensor) -> torch.Tensor:
        n = self.n
        dk = torch.fft.rfftn(density)
        p = (self.box ** 3 / float(n) ** 6) * (dk.real ** 2 + dk.imag ** 2)
        psum = torch.bincount(self.b, weights=self.w * p[self.sel], minlength=self.ns)
        return torch.where(self.count > 0, psum / self.count.clamp_min(1), 0.0)

    def loss(self, density, pk, target_density, target_pk) -> float:
        ok = (pk > 0) & (target_pk > 0)
        lr = torch.where(ok, torch.log(torch.where(ok, pk, 1.0)) - torch.log(torch.where(ok, target_pk, 1.0)), 0.0)
        return float(((density - target_density) ** 2).sum() / density.numel() + (lr * lr).sum())

    def density_cotangent(self, density, g_density, g_pk):
        """dL/d(density) of a loss with cotangents g_density (per cell) and g_pk (per shell):
        g_density + N^3 IDFT[w_b delta(k)], w_b = 2 V g_pk[b] / (N^6 c_b)."""
        n = self.n
        wb = torch.where(self.count > 0, 2.0 * self.box ** 3 * g_pk / (float(n) ** 6 * self.count.clamp_min(1)), 0.0)
        m = torch.zeros_like(self.s)
        m[self.sel] = wb[self.b]
        return g_density + float(n) ** 3 * torch.fft.irfftn(m * torch.fft.rfftn(density), s=(n, n, n))

    def cic_transpose(self, u: torch.Tensor, base: torch.Tensor, g_rho: torch.Tensor) -> torch.Tensor:
        """dL/dx (per unit length, shape (3, M)) of particles at u (cells) deposited with
        lower-corner cells `base`, for the density cotangent g_rho (one particle per cell)."""
        n = self.n
        d = u - base
        i0 = torch.remainder(base, n)
        g = g_rho.reshape(-1)
        out = torch.zeros_like(u)
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
        return out * (n / self.box)

    def cotangents(self, density, pk, target_density, target_pk):
        """(dL/d density, dL/dP_b) of the loss above."""
        ok = (pk > 0) & (target_pk > 0)
        lr = torch.where(ok, torch.log(torch.where(ok, pk, 1.0)) - torch.log(torch.where(ok, target_pk, 1.0)), 0.0)
        gd = 2.0 * (density - target_density) / density.numel()
        gp = torch.where(ok, 2.0 * lr / torch.where(ok, pk, 1.0), 0.0)
        return gd, gp
