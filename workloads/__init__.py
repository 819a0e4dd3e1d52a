"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds workload descriptions (grid size, box, cosmology, seeds,
|f_R0| draws) and seeded random arrays only.  It contains none of the method's
arithmetic: no FFT, no growth factor, no power spectrum, no displacement.

Cosmology: the flat LCDM background the paper uses for its f(R) runs
(Omega_m + Omega_Lambda = 1, Sec. 4), with h, n_s, sigma_8 of the synthetic
workloads, Omega_b = 0.0481 and T_CMB = 2.7255 K (needed by the
Eisenstein-Hu no-wiggle transfer function, not given for these runs).
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "Cosmology", "Instance", "COSMO", "oracle_64", "plain_256", "fwd_512",
    "large_1024", "batched_96", "differentiable_512", "white_noise",
    "random_positions", "random_field",
]


@dataclasses.dataclass(frozen=True)
class Cosmology:
    omega_m: float = 0.3
    omega_l: float = 0.7
    omega_b: float = 0.0481
    h: float = 0.7
    n_s: float = 0.96
    sigma8: float = 0.8
    t_cmb: float = 2.7255
    fr0_abs: float = 1e-5     # |f_R0|; 0 means GR (mu = 1)
    hs_n: int = 1             # Hu-Sawicki n; only n = 1 is defined (Sec. 2.3)
    a_init: float = 1e-3      # start of the growth integration
    d2_variant: int = 0       # triangle configuration of D2: 0 = T1 (the paper's choice)

    def replace(self, **kw) -> "Cosmology":
        return dataclasses.replace(self, **kw)


@dataclasses.dataclass(frozen=True)
class Instance:
    n: int            # grid points per side = particles per side
    box: float        # side of the periodic cube, Mpc/h
    seed: int         # Philox key
    cosmo: Cosmology
    a_out: float = 1.0

    @property
    def n_particles(self) -> int:
        return self.n ** 3


COSMO = Cosmology()

# growth-table grid: 512 log-spaced k in [1e-4, 10] h/Mpc
N_K = 512
K_MIN = 1e-4
K_MAX = 10.0
N_SHELLS = 32


def oracle_64() -> Instance:
    """64^3 grid, 256 Mpc/h, |f_R0| = 1e-5, seed 1, z = 0."""
    return Instance(64, 256.0, 1, COSMO)


def plain_256() -> Instance:
    """256^3 grid, 1024 Mpc/h, |f_R0| = 1e-5, seed 1, z = 0."""
    return Instance(256, 1024.0, 1, COSMO)


def fwd_512() -> Instance:
    """512^3 grid, 1024 Mpc/h, |f_R0| = 1e-5, seed 1, z = 0 (the throughput workload)."""
    return Instance(512, 1024.0, 1, COSMO)


def differentiable_512(seed: int = 1) -> Instance:
    """512^3 grid, 1024 Mpc/h, |f_R0| = 1e-5; the target field uses seed 7."""
    return Instance(512, 1024.0, seed, COSMO)


def large_1024(fr0_abs: float = 1e-5) -> Instance:
    """1024^3 grid, 2048 Mpc/h, |f_R0| in {1e-4, 1e-5, 1e-6}."""
    return Instance(1024, 2048.0, 1, COSMO.replace(fr0_abs=fr0_abs))


def batched_96(host_seed: int = 12345) -> list[Instance]:
    """96 instances: 32 each of 96^3/384, 128^3/512, 192^3/768 Mpc/h, seeds 1..96,
    |f_R0| log-uniform in [1e-6, 1e-4] drawn from a fixed host RNG."""
    rng = np.random.default_rng(host_seed)
    logf = rng.uniform(np.log(1e-6), np.log(1e-4), size=96)
    out = []
    for i in range(96):
        n, box = [(96, 384.0), (128, 512.0), (192, 768.0)][i // 32]
        out.append(Instance(n, box, i + 1, COSMO.replace(fr0_abs=float(np.exp(logf[i])))))
    return out


def white_noise(n: int, seed: int, dtype=np.float32) -> np.ndarray:
    """Explicit unit-variance Gaussian noise (numpy PCG64), shape (n, n, n), z fastest.
    Used where a test passes noise in rather than drawing it from Philox."""
    return np.random.default_rng(seed).standard_normal((n, n, n)).astype(dtype)


def random_field(shape, seed: int, dtype=np.float32) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(shape).astype(dtype)


def random_positions(n: int, box: float, seed: int, spread_cells: float = 3.0) -> np.ndarray:
    """Particle positions SoA (3, n^3) in [0, box): the cell-corner lattice plus a
    Gaussian jitter of `spread_cells` cells, wrapped into the box (FP32)."""
    rng = np.random.default_rng(seed)
    cell = box / n
    g = np.indices((n, n, n)).reshape(3, -1).astype(np.float64) * cell
    g += rng.standard_normal(g.shape) * spread_cells * cell
    return np.mod(g, box).astype(np.float32) % np.float32(box)
