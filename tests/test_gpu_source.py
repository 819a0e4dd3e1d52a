"""GPU full-source diagnostic (lpt2_source_ratio, Sec. 3 Eqs. full, s1-s4) against the
FP64 oracle (oracle/fullsource.py) on the same Philox noise.

Tolerances (FP32, about 36 three-pass transforms, against FP64):
  S_MG, S_GR half spectra      relative L2 <= 2e-5
  shell mean of Re(S_MG/S_GR)  <= 1e-4 absolute (the ratios are O(1))
  shell scatter                <= 2e-3 absolute: modes whose S_GR nearly vanishes carry
                                 ratio errors of eps_32 |S| / |S_GR| and dominate the variance
  mode counts                  exact; T1 curve at the shell mean |k| <= 1e-6 relative
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
STEPS = 256


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_06282_gb300 import build as B
    B.build()
    import paper_1909_06282_gb300 as L
    return L


def oracle(n, box, c, a, seed, nb):
    from oracle import fullsource as fs
    from oracle import growth, lpt2, philox
    noise = philox.gaussian_noise(n, seed, as_float64=True).reshape(n, n, n)
    dk0 = lpt2.delta_k(n, box, c, noise)
    tab = growth.growth_tables(c, a, n_steps=STEPS)
    d1gr = fs.d1_gr_norm(c, a, n_steps=STEPS)
    S = fs.source_terms(n, box, c, a, dk0, tab, d1gr)
    mean, sig, cnt = fs.source_ratio(n, box, c, a, dk0, tab, d1gr, n_bins=nb)
    return S, mean, sig, cnt, tab, d1gr


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("n,box,fr0,a_out", [(32, 128.0, 1e-4, 1.0), (32, 200.0, 1e-5, 0.6667),
                                             (32, 64.0, 1e-6, 0.5), (64, 256.0, 1e-4, 1.0)])
def test_source_ratio_against_oracle(lib, n, box, fr0, a_out):
    from oracle import fullsource as fs
    c = W.COSMO.replace(fr0_abs=fr0)
    nb = 16
    plan = lib.Plan(W.Instance(n, box, 3, c, a_out), n_steps=STEPS)
    res = lib.lpt2_source_ratio(plan, n_bins=nb, spectra=True)
    torch.cuda.synchronize()
    lib.lpt2_device_status(plan)
    S, mean, sig, cnt, tab, d1gr = oracle(n, box, c, a_out, 3, nb)
    smg = (S[0] + S[1] + S[2] + S[3])[:, :, : n // 2]
    sgr = S[4][:, :, : n // 2]
    assert rel_l2(res["s_mg"].cpu().numpy(), smg) <= 2e-5
    assert rel_l2(res["s_gr"].cpu().numpy(), sgr) <= 2e-5
    np.testing.assert_array_equal(res["count"].cpu().numpy(), cnt)
    ok = cnt > 0
    gm = res["mean"].cpu().numpy()
    assert np.abs(gm[ok] - mean[ok]).max() <= 1e-4, (gm, mean)
    assert np.abs(res["sigma"].cpu().numpy()[ok] - sig[ok]).max() <= 2e-3
    km = res["k_mean"].cpu().numpy()
    np.testing.assert_allclose(res["t1"].cpu().numpy()[ok], fs.t1_ratio(c, a_out, km[ok], tab, d1gr), rtol=1e-6)
    assert gm[ok][-1] > 1.0           # the MG source is enhanced over GR on the smallest scales


def test_source_ratio_gr_limit(lib):
    n, box = 32, 128.0
    c = W.COSMO.replace(fr0_abs=1e-16)
    plan = lib.Plan(W.Instance(n, box, 4, c), n_steps=STEPS)
    res = lib.lpt2_source_ratio(plan, n_bins=8)
    ok = res["count"].cpu().numpy() > 0
    assert np.abs(res["mean"].cpu().numpy()[ok] - 1.0).max() <= 1e-4
    np.testing.assert_allclose(res["t1"].cpu().numpy()[ok], 1.0, atol=1e-6)


def test_source_ratio_after_set_fr0_equals_a_fresh_plan(lib):
    """The diagnostic reads the plan's current tables: after lpt2_set_fr0 it equals a plan
    made at that |fR0| (the GR reference is recomputed per call)."""
    n, box, a = 32, 64.0, 0.5
    plan = lib.Plan(W.Instance(n, box, 5, W.COSMO.replace(fr0_abs=1e-5), a), n_steps=STEPS)
    lib.lpt2_set_fr0(plan, 1e-4)
    got = lib.lpt2_source_ratio(plan, n_bins=16)
    fresh = lib.Plan(W.Instance(n, box, 5, W.COSMO.replace(fr0_abs=1e-4), a), n_steps=STEPS)
    want = lib.lpt2_source_ratio(fresh, n_bins=16)
    for k in ("mean", "sigma", "t1", "k_mean"):
        np.testing.assert_allclose(got[k].cpu().numpy(), want[k].cpu().numpy(), rtol=1e-6, atol=1e-12)
    assert torch.equal(got["count"], want["count"])
