"""Philox4x32-10 and Box-Muller white noise (oracle, float64).

The paper starts from "a linear density field on a regular grid" (Sec. 3); the
white noise behind it is drawn here with the counter-based Philox4x32 generator
of Salmon, Moraes, Dror & Shaw (2011), 10 rounds, written from that paper's
definition: each round multiplies words 0 and 2 by the two published 32-bit
multipliers, takes the high/low halves, xors the high halves with words 1 / 3
and the two key words, and the key is bumped by the two Weyl constants between
rounds.

Stream layout (a reading; the paper has no RNG):
  key     = (seed mod 2^32, seed div 2^32)
  counter = (c mod 2^32, c div 2^32, 0, 0) with c = (ix*N + iy)*N + iz (z fastest) of the
            cell with even iy; the cells (ix, iy, iz) and (ix, iy+1, iz) share that draw
  u_j     = ((x_j >> 8) + 1) * 2^-24 for output words x_0, x_1  (exact in FP32, in (0, 1])
  g       = sqrt(-2 ln u_0) * (cos, sin)(2 pi u_1) for (even iy, odd iy): both outputs of
            one Box-Muller transform, evaluated in float64, stored as float32.
"""
from __future__ import annotations

import numpy as np

__all__ = ["philox4x32_10", "uniforms", "box_muller", "gaussian_noise", "MULT", "WEYL"]

MULT = (0xD2511F53, 0xCD9E8D57)   # round multipliers (Salmon et al. 2011)
WEYL = (0x9E3779B9, 0xBB67AE85)   # key schedule increments (Salmon et al. 2011)
_M32 = np.uint64(0xFFFFFFFF)


def _mulhilo(a: int, b: np.ndarray):
    p = np.uint64(a) * b.astype(np.uint64)
    return (p >> np.uint64(32)) & _M32, p & _M32


def philox4x32_10(ctr, key):
    """ctr: 4 uint arrays (broadcastable), key: 2 ints or arrays. Returns 4 uint32 arrays."""
    c = [np.asarray(x, dtype=np.uint64) & _M32 for x in ctr]
    k0 = np.asarray(key[0], dtype=np.uint64) & _M32
    k1 = np.asarray(key[1], dtype=np.uint64) & _M32
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(WEYL[0])) & _M32
            k1 = (k1 + np.uint64(WEYL[1])) & _M32
        hi0, lo0 = _mulhilo(MULT[0], c[0])
        hi1, lo1 = _mulhilo(MULT[1], c[2])
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return [x.astype(np.uint32) for x in c]


def _words(n: int, seed: int, first: int = 0, count: int | None = None):
    total = n ** 3
    count = total - first if count is None else count
    cell = np.arange(first, first + count, dtype=np.uint64)
    ctr = (cell & _M32, cell >> np.uint64(32), np.zeros_like(cell), np.zeros_like(cell))
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return philox4x32_10(ctr, key)


def uniforms(x: np.ndarray) -> np.ndarray:
    """u = ((x >> 8) + 1) * 2^-24 in float64 (exactly representable in float32)."""
    return ((x.astype(np.uint64) >> np.uint64(8)) + np.uint64(1)).astype(np.float64) * 2.0 ** -24


def box_muller(x0: np.ndarray, x1: np.ndarray):
    """(g_even, g_odd) = sqrt(-2 ln u0) (cos, sin)(2 pi u1) in float64 for words x0, x1."""
    u0, u1 = uniforms(x0), uniforms(x1)
    r = np.sqrt(-2.0 * np.log(u0))
    return r * np.cos(2.0 * np.pi * u1), r * np.sin(2.0 * np.pi * u1)


def gaussian_noise(n: int, seed: int, first: int = 0, count: int | None = None,
                   as_float64: bool = False) -> np.ndarray:
    """Unit-variance Gaussian per cell via Box-Muller on Philox words 0 and 1 of the
    draw of its even-iy cell.  Returns the flat cells [first, first+count) (all N^3
    cells by default)."""
    total = n ** 3
    count = total - first if count is None else count
    cell = np.arange(first, first + count, dtype=np.int64)
    iy = (cell // n) % n
    base = np.where(iy % 2 == 0, cell, cell - n).astype(np.uint64)      # counter of the pair
    ctr = (base & _M32, base >> np.uint64(32), np.zeros_like(base), np.zeros_like(base))
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    x0, x1, _, _ = philox4x32_10(ctr, key)
    ge, go = box_muller(x0, x1)
    g = np.where(iy % 2 == 0, ge, go)
    return g if as_float64 else g.astype(np.float32)
