"""Pins of the oracle's FFT and Philox noise against facts outside the oracle."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import fft as of
from oracle import philox

HERE = os.path.dirname(os.path.abspath(__file__))


def brute_dft3(a, sign):
    """O(N^6) direct sum over every (n, x) pair."""
    n = a.shape[0]
    idx = np.arange(n)
    x = np.stack(np.meshgrid(idx, idx, idx, indexing="ij"), -1).reshape(-1, 3)
    ph = (x @ x.T) % n                       # n.x for every pair (mode list = position list)
    return (np.exp(sign * 2j * np.pi * ph / n) @ a.reshape(-1)).reshape(a.shape)


@pytest.mark.parametrize("n", [4, 8])
def test_fft_matches_brute_force_dft(n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    np.testing.assert_allclose(of.fftn(a), brute_dft3(a, -1), atol=1e-11 * n ** 3)
    np.testing.assert_allclose(of.ifftn(a), brute_dft3(a, +1) / n ** 3, atol=1e-12)


@pytest.mark.parametrize("shape", [(16, 16, 16), (32, 8, 64), (6, 96, 4), (3, 5, 192)])
def test_fft_axis_matches_numpy(shape):
    rng = np.random.default_rng(1)
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    for ax in range(3):
        np.testing.assert_allclose(of.fft_axis(a, ax), np.fft.fft(a, axis=ax), atol=1e-10)
        np.testing.assert_allclose(of.fft_axis(a, ax, inverse=True), np.fft.ifft(a, axis=ax),
                                   atol=1e-13)


def test_fft_roundtrip_and_parseval():
    rng = np.random.default_rng(2)
    a = rng.standard_normal((32, 32, 32))
    f = of.fftn(a)
    np.testing.assert_allclose(of.ifftn(f).real, a, atol=1e-13)
    assert abs(np.sum(np.abs(f) ** 2) / a.size - np.sum(a * a)) < 1e-9 * np.sum(a * a)


def _kat():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(v, 16) for v in line.split()])
    return rows


def test_philox_known_answers():
    for r in _kat():
        out = philox.philox4x32_10([np.array([v]) for v in r[:4]], (r[4], r[5]))
        assert [int(o[0]) for o in out] == r[6:10]


TORCH_PHILOX_SRC = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdlib>
int main(int argc, char** argv) {
  unsigned long long seed = strtoull(argv[1], 0, 10);
  unsigned long long first = strtoull(argv[2], 0, 10), count = strtoull(argv[3], 0, 10);
  for (unsigned long long c = first; c < first + count; ++c) {
    at::philox_engine e(seed, 0, c);       // key = seed, counter = (c, 0) as (lo, hi, 0, 0)
    unsigned a = e(), b = e(), d = e(), f = e();
    printf("%u %u %u %u\n", a, b, d, f);
  }
  return 0;
}
"""


def test_philox_matches_torch_engine():
    """Cross-run against the Philox4x32-10 engine that ships as a header with PyTorch."""
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "p.cpp")
        exe = os.path.join(d, "p")
        with open(src, "w") as fh:
            fh.write(TORCH_PHILOX_SRC)
        r = subprocess.run(["g++", "-O1", "-std=c++17", "-I", inc, src, "-o", exe],
                           capture_output=True, text=True)
        if r.returncode != 0:
            pytest.skip("torch Philox header does not compile here: " + r.stderr[-300:])
        for seed, first, count in [(1, 0, 300), (0x123456789ABCDEF, (1 << 32) - 5, 10),
                                   (7, 134217700, 20)]:
            out = subprocess.run([exe, str(seed), str(first), str(count)], capture_output=True,
                                 text=True, check=True).stdout.split()
            ref = np.array(out, dtype=np.uint64).reshape(-1, 4).T
            n_big = 1 << 12   # any N with N^3 > first + count; the counter is the flat index
            got = philox._words(n_big, seed, first, count)
            for j in range(4):
                np.testing.assert_array_equal(got[j].astype(np.uint64), ref[j])


def test_gaussian_noise_statistics():
    g = philox.gaussian_noise(128, 3, as_float64=True)
    assert g.size == 128 ** 3
    assert abs(g.mean()) < 5 / np.sqrt(g.size)
    assert abs(g.var() - 1.0) < 5 * np.sqrt(2.0 / g.size)
    from scipy import stats
    assert stats.kstest(g[:200000], "norm").pvalue > 1e-4
    # the uniforms are exact in float32 and lie in (0, 1]
    x0, _, _, _ = philox._words(16, 3)
    u = philox.uniforms(x0)
    assert np.all(u > 0) and np.all(u <= 1)
    np.testing.assert_array_equal(u.astype(np.float32).astype(np.float64), u)


def test_noise_is_counter_addressed():
    a = philox.gaussian_noise(32, 9)
    b = philox.gaussian_noise(32, 9, first=1000, count=77)
    np.testing.assert_array_equal(a[1000:1077], b)
    assert not np.array_equal(a, philox.gaussian_noise(32, 10))


def test_noise_pairs_are_one_box_muller_draw():
    """Cells (x, 2j, z) and (x, 2j+1, z) are the cosine and sine outputs of the draw at
    the even cell: their squares sum to -2 ln u0 and their angle is 2 pi u1."""
    n, seed = 8, 4
    g = philox.gaussian_noise(n, seed, as_float64=True).reshape(n, n, n)
    x0, x1, _, _ = philox._words(n, seed)
    u0 = philox.uniforms(x0).reshape(n, n, n)[:, 0::2, :]
    u1 = philox.uniforms(x1).reshape(n, n, n)[:, 0::2, :]
    ge, go = g[:, 0::2, :], g[:, 1::2, :]
    np.testing.assert_allclose(ge ** 2 + go ** 2, -2 * np.log(u0), rtol=1e-12, atol=1e-15)
    ang = np.mod(np.arctan2(go, ge), 2 * np.pi)
    np.testing.assert_allclose(np.cos(ang - 2 * np.pi * u1), 1.0, atol=1e-9)
    big = philox.gaussian_noise(64, 5, as_float64=True).reshape(64, 64, 64)
    assert abs(np.corrcoef(big[:, 0::2, :].ravel(), big[:, 1::2, :].ravel())[0, 1]) < 0.01
