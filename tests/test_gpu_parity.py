"""GPU parity: every entry point of the C ABI against the FP64 oracle on the same
seeded inputs.  Tolerances (FP32 CUDA path vs FP64 oracle):
  Philox words             bit-exact
  white noise (FP32)       the FP64 transform rounded once: equal in >= 99.999 % of cells,
                           within 1 ulp everywhere (the GPU evaluates it in float-float)
  growth tables (FP64)     1e-10 relative (same RK4 step count on both sides)
  Psi1, Psi2, Psi          relative L2 <= 2e-5 and max |delta Psi| <= 1e-4 cell
  P(k)                     <= 1e-4 relative per non-empty shell
"""
import functools

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STEPS = 1024
REL_L2 = 2e-5
MAX_CELL = 1e-4
PK_REL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_06282_gb300 import build as B
    B.build()


def lp():
    import paper_1909_06282_gb300 as L
    return L


@functools.lru_cache(maxsize=None)
def oracle_run(n, box, seed, fr0, noise_seed=None):
    from oracle import lpt2
    inst = W.Instance(n, box, seed, W.COSMO.replace(fr0_abs=fr0))
    noise = None if noise_seed is None else W.white_noise(n, noise_seed)
    return lpt2.run(n, box, inst.cosmo, seed=seed, noise=noise, n_steps=STEPS)


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def periodic_diff(a, b, box):
    d = a - b
    return d - box * np.round(d / box)


def check_psi(got, want, cell, what):
    r = rel_l2(got, want)
    m = float(np.max(np.abs(got - want))) / cell
    assert r <= REL_L2, f"{what}: rel L2 {r:.3e}"
    assert m <= MAX_CELL, f"{what}: max |d| {m:.3e} cell"
    return r, m


def test_philox_words_bit_exact():
    from oracle import philox
    for seed, first, count in [(1, 0, 4096), (0xDEADBEEF12345, (1 << 32) - 100, 300), (7, 10 ** 9, 1000)]:
        got = lp().lpt2_philox_words(seed, first, count).cpu().numpy().view(np.uint32)
        want = np.stack(philox._words(1 << 12, seed, first, count), axis=1)
        np.testing.assert_array_equal(got, want)


def ulp_distance(a32, b32):
    """Distance in units in the last place between float32 arrays (+0 and -0 coincide)."""
    def ordered(x):
        i = x.view(np.int32).astype(np.int64)
        return np.where(i < 0, -(i & 0x7FFFFFFF), i)
    return np.abs(ordered(a32) - ordered(b32))


def check_gaussians(got, want64, r64):
    """C8: equal to the FP64 value rounded once in >= 99.999 % of the values, within 1 ulp
    everywhere.  Where the FP64 reference is one of the exact zeros of cos / sin (2 pi u1 a
    multiple of pi/2, rounded in FP64: |value| ~ 1e-16 r instead of 0) the bound is the
    reference's own absolute error, 1e-15 r."""
    want = want64.astype(np.float32)
    ulp = ulp_distance(got, want)
    zero_case = np.abs(want64) < 1e-12 * np.maximum(r64, 1.0)
    assert np.all(np.abs(got[zero_case].astype(np.float64) - want64[zero_case]) <= 1e-15 * np.maximum(r64[zero_case], 1)), \
        (got[zero_case], want64[zero_case])
    ulp = np.where(zero_case, 0, ulp)
    equal = float(np.mean(ulp == 0))
    assert ulp.max() <= 1, (int(ulp.max()), np.argmax(ulp))
    assert equal >= 0.99999, equal
    return equal, int(np.sum(ulp != 0)), int(np.sum(zero_case))


@pytest.mark.parametrize("n,seed", [(64, 1), (32, 123456789012), (128, 5)])
def test_white_noise_against_oracle(n, seed):
    from oracle import philox
    plan = lp().Plan(W.Instance(n, 100.0, seed, W.COSMO), n_steps=16)
    got = lp().lpt2_white_noise(plan).cpu().numpy().ravel()
    want64 = philox.gaussian_noise(n, seed, as_float64=True)
    # radius of each cell's draw, for the absolute bound at exact zeros of cos / sin
    r64 = np.abs(want64).reshape(n, n // 2, 2, n)
    r64 = np.repeat(np.sqrt(r64[:, :, 0, :] ** 2 + r64[:, :, 1, :] ** 2)[:, :, None, :], 2, axis=2).ravel()
    equal, n_off, n_zero = check_gaussians(got, want64, r64)
    print(f"noise {n}^3: {equal:.7f} equal after rounding, {n_off} cells 1 ulp off, {n_zero} exact zeros")


def test_box_muller_edge_words():
    """The transform on chosen words: u0 = 1 (radius 0), u0 = 2^-24 (largest radius), the
    values of u0 around the sqrt(2) and table boundaries of the logarithm, every quadrant and
    octant boundary of the angle and its neighbours, the sine/cosine table boundaries, and
    2^20 random words."""
    from oracle import philox
    rng = np.random.default_rng(2024)
    m0 = [1, 2, 3, 255, 256, (1 << 23), (1 << 23) + 1, (1 << 24) - 1, 1 << 24]
    m0 += [int(round(2 ** 23 * np.sqrt(2))) + d for d in (-2, -1, 0, 1, 2)]
    m0 += [int((1 << 23) * (1 + j / 128)) + d for j in range(-37, 54, 3) for d in (-1, 0, 1)]
    m1 = [1, 2, 1 << 24, (1 << 24) - 1]
    m1 += [q * (1 << 21) + d for q in range(1, 8) for d in (-2, -1, 0, 1, 2)]
    m1 += [j * (1 << 12) + d for j in range(0, 2048, 37) for d in (-1, 0, 1)]
    m0 = np.array([m for m in m0 if 1 <= m <= 1 << 24], dtype=np.uint64)
    m1 = np.array([m for m in m1 if 1 <= m <= 1 << 24], dtype=np.uint64)
    M0, M1 = np.meshgrid(m0, m1, indexing="ij")
    x0 = ((M0.ravel() - 1) << np.uint64(8)) | np.uint64(0x5A)     # low 8 bits do not matter
    x1 = ((M1.ravel() - 1) << np.uint64(8)) | np.uint64(0xA5)
    rx = rng.integers(0, 2 ** 32, size=(2, 1 << 20), dtype=np.uint64)
    x0 = np.concatenate([x0, rx[0]]).astype(np.uint32)
    x1 = np.concatenate([x1, rx[1]]).astype(np.uint32)
    words = torch.from_numpy(np.stack([x0, x1], axis=1).view(np.int32)).cuda()
    plan = lp().Plan(W.Instance(16, 100.0, 1, W.COSMO), n_steps=16)
    got = lp().lpt2_box_muller(plan, words).cpu().numpy()
    ge, go = philox.box_muller(x0, x1)
    r64 = np.sqrt(-2.0 * np.log(philox.uniforms(x0)))
    for j, want64 in enumerate((ge, go)):
        equal, n_off, n_zero = check_gaussians(got[:, j].copy(), want64, r64)
        print(f"box-muller output {j}: {equal:.7f} equal, {n_off} off by 1 ulp, {n_zero} exact zeros")
    # u0 = 1: both outputs are zero
    one = (x0 >> 8) == 0xFFFFFF
    assert np.all(got[one] == 0)


@pytest.mark.parametrize("n", [16, 32, 64, 96, 128, 192])
def test_fft_r2c_c2r_against_oracle(n):
    from oracle import fft as of
    plan = lp().Plan(W.Instance(n, 100.0, 1, W.COSMO), n_steps=16)
    x = W.random_field((n, n, n), 40 + n)
    X = lp().lpt2_fft_r2c(plan, torch.from_numpy(x).cuda()).cpu().numpy()
    ref = of.fftn(x.astype(np.float64))
    half = ref[:, :, : n // 2]
    assert rel_l2(X, half) < 2e-6
    # inverse of the half spectrum (kz = N/2 plane implicitly zero)
    full = ref.copy()
    full[:, :, n // 2] = 0
    want = of.ifftn(full).real * n ** 3
    got = lp().lpt2_fft_c2r(plan, torch.from_numpy(half.astype(np.complex64)).cuda()).cpu().numpy()
    assert rel_l2(got, want) < 2e-6


@pytest.mark.parametrize("fr0,a_out", [(1e-5, 1.0), (1e-4, 0.5), (0.0, 1.0), (1e-6, 0.8)])
def test_growth_tables_against_oracle(fr0, a_out):
    from oracle import growth as gr
    c = W.COSMO.replace(fr0_abs=fr0)
    plan = lp().Plan(W.Instance(32, 100.0, 1, c, a_out=a_out), n_steps=STEPS)
    d1, d2, dd1, dd2 = [t.cpu().numpy() for t in lp().lpt2_growth_tables(plan)]
    ref = gr.growth_tables(c, a_out, n_steps=STEPS)
    np.testing.assert_allclose(d1, ref["D1"], rtol=1e-10)
    np.testing.assert_allclose(d2, ref["D2"], rtol=1e-10)
    scale1 = np.max(np.abs(ref["dD1"])) + 1e-300
    scale2 = np.max(np.abs(ref["dD2"])) + 1e-300
    assert np.max(np.abs(dd1 - ref["dD1"])) <= 1e-10 * scale1
    assert np.max(np.abs(dd2 - ref["dD2"])) <= 1e-10 * scale2


@pytest.mark.parametrize("n,box,fr0", [(64, 256.0, 1e-5), (32, 200.0, 1e-4), (16, 64.0, 0.0),
                                       (128, 512.0, 1e-6), (96, 384.0, 3e-5)])
def test_displace_split_against_oracle(n, box, fr0):
    inst = W.Instance(n, box, 1, W.COSMO.replace(fr0_abs=fr0))
    plan = lp().Plan(inst, n_steps=STEPS)
    out = lp().lpt2_displace(plan, psi1=True, psi2=True, pos=True, dk=True)
    ref = oracle_run(n, box, 1, fr0)
    cell = box / n
    check_psi(out["psi1"].cpu().numpy(), ref["psi1"], cell, "psi1")
    check_psi(out["psi2"].cpu().numpy(), ref["psi2"], cell, "psi2")
    dk = out["dk"].cpu().numpy()
    assert rel_l2(dk, ref["delta_k"][:, :, : n // 2]) < 2e-6
    pos = out["pos"].cpu().numpy().reshape(3, -1).astype(np.float64)
    d = periodic_diff(pos, ref["pos"], box)
    assert np.max(np.abs(d)) / cell <= MAX_CELL


def test_displace_total_mode_equals_split_and_oracle():
    n, box = 64, 256.0
    inst = W.Instance(n, box, 1, W.COSMO)
    plan = lp().Plan(inst, n_steps=STEPS)
    tot = lp().lpt2_displace(plan, psi1=False, psi2=False, pos=True)["pos"].cpu().numpy()
    ref = oracle_run(n, box, 1, 1e-5)
    d = periodic_diff(tot.reshape(3, -1).astype(np.float64), ref["pos"], box)
    psi = (ref["psi1"] + ref["psi2"]).reshape(3, -1)
    assert np.linalg.norm(d) / np.linalg.norm(psi) <= REL_L2
    assert np.max(np.abs(d)) / (box / n) <= MAX_CELL


def test_displace_with_explicit_noise():
    n, box = 32, 128.0
    inst = W.Instance(n, box, 5, W.COSMO)
    plan = lp().Plan(inst, n_steps=STEPS)
    noise = torch.from_numpy(W.white_noise(n, 77)).cuda()
    out = lp().lpt2_displace(plan, noise=noise, psi1=True, psi2=True, pos=False)
    ref = oracle_run(n, box, 5, 1e-5, noise_seed=77)
    check_psi(out["psi1"].cpu().numpy(), ref["psi1"], box / n, "psi1")
    check_psi(out["psi2"].cpu().numpy(), ref["psi2"], box / n, "psi2")


@pytest.mark.parametrize("n,box", [(64, 256.0), (32, 100.0)])
def test_cic_pk_on_seeded_positions(n, box):
    from oracle import lpt2
    plan = lp().Plan(W.Instance(n, box, 1, W.COSMO), n_steps=16)
    pos = W.random_positions(n, box, 11)
    res = lp().lpt2_cic_pk(plan, pos=torch.from_numpy(pos).cuda(), density=True, n_shells=32)
    want = lpt2.cic_density(n, box, pos.astype(np.float64))
    got = res["density"].cpu().numpy()
    assert np.max(np.abs(got - want)) < 2e-5 * max(1.0, np.max(np.abs(want)))
    pk, km, cnt = lpt2.power_spectrum(n, box, want, 32)
    np.testing.assert_array_equal(res["n_modes"].cpu().numpy(), cnt)
    ok = cnt > 0
    np.testing.assert_allclose(res["pk"].cpu().numpy()[ok], pk[ok], rtol=PK_REL)
    np.testing.assert_allclose(res["k_mean"].cpu().numpy()[ok], km[ok], rtol=1e-6)
    assert np.all(res["pk"].cpu().numpy()[~ok] == 0)


@pytest.mark.parametrize("n_shells", [1, 7, 32, 100])
def test_pk_shell_counts_any_shell_number(n_shells):
    from oracle import lpt2
    n, box = 32, 100.0
    plan = lp().Plan(W.Instance(n, box, 1, W.COSMO), n_steps=16)
    pos = W.random_positions(n, box, 12)
    res = lp().lpt2_cic_pk(plan, pos=torch.from_numpy(pos).cuda(), n_shells=n_shells)
    want = lpt2.cic_density(n, box, pos.astype(np.float64))
    pk, km, cnt = lpt2.power_spectrum(n, box, want, n_shells)
    np.testing.assert_array_equal(res["n_modes"].cpu().numpy(), cnt)
    ok = cnt > 0
    np.testing.assert_allclose(res["pk"].cpu().numpy()[ok], pk[ok], rtol=PK_REL)


def test_end_to_end_pk_64():
    n, box = 64, 256.0
    plan = lp().Plan(W.Instance(n, box, 1, W.COSMO), n_steps=STEPS)
    lp().lpt2_displace(plan, psi1=False, psi2=False, pos=False)
    res = lp().lpt2_cic_pk(plan, pos=None, n_shells=32)
    ref = oracle_run(n, box, 1, 1e-5)
    ok = ref["n_modes"] > 0
    np.testing.assert_array_equal(res["n_modes"].cpu().numpy(), ref["n_modes"])
    np.testing.assert_allclose(res["pk"].cpu().numpy()[ok], ref["pk"][ok], rtol=PK_REL)


def test_repeat_calls_are_deterministic_and_launch_counted():
    n, box = 32, 128.0
    plan = lp().Plan(W.Instance(n, box, 3, W.COSMO), n_steps=64)
    a = lp().lpt2_displace(plan, psi1=True, psi2=True, pos=True)
    c0 = lp().lpt2_launch_count(plan)
    b = lp().lpt2_displace(plan, psi1=True, psi2=True, pos=True)
    assert lp().lpt2_launch_count(plan) > c0
    for k in a:
        assert torch.equal(a[k], b[k])
    lp().lpt2_device_status(plan)   # no bounded device-side wait ran out


def test_192_full_against_oracle():
    """192^3, L = 768 Mpc/h (the largest grid of the batched workload; radix 4-12-4 FFTs):
    displacements, positions and the P(k) of the displaced particles against the FP64
    oracle on the full grid."""
    n, box = 192, 768.0
    plan = lp().Plan(W.Instance(n, box, 1, W.COSMO), n_steps=STEPS)
    out = lp().lpt2_displace(plan, psi1=True, psi2=True, pos=True)
    res = lp().lpt2_cic_pk(plan, pos=None, density=True, n_shells=32)
    ref = oracle_run(n, box, 1, 1e-5)
    cell = box / n
    check_psi(out["psi1"].cpu().numpy(), ref["psi1"], cell, "psi1 192")
    check_psi(out["psi2"].cpu().numpy(), ref["psi2"], cell, "psi2 192")
    pos = out["pos"].cpu().numpy().reshape(3, -1).astype(np.float64)
    assert np.max(np.abs(periodic_diff(pos, ref["pos"], box))) / cell <= MAX_CELL
    ok = ref["n_modes"] > 0
    np.testing.assert_array_equal(res["n_modes"].cpu().numpy(), ref["n_modes"])
    np.testing.assert_allclose(res["pk"].cpu().numpy()[ok], ref["pk"][ok], rtol=PK_REL)
    d = res["density"].cpu().numpy().ravel()
    assert np.max(np.abs(d - ref["density"].ravel())) < 1e-3


def test_256_full_against_oracle():
    n, box = 256, 1024.0
    plan = lp().Plan(W.Instance(n, box, 1, W.COSMO), n_steps=STEPS)
    out = lp().lpt2_displace(plan, psi1=True, psi2=True, pos=False)
    res = lp().lpt2_cic_pk(plan, pos=None, n_shells=32)
    ref = oracle_run(n, box, 1, 1e-5)
    check_psi(out["psi1"].cpu().numpy(), ref["psi1"], box / n, "psi1 256")
    check_psi(out["psi2"].cpu().numpy(), ref["psi2"], box / n, "psi2 256")
    ok = ref["n_modes"] > 0
    np.testing.assert_allclose(res["pk"].cpu().numpy()[ok], ref["pk"][ok], rtol=PK_REL)
