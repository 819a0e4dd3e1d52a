"""Batched plans: several instances of mixed grid sizes, seeds and |f_R0| in one
plan (each grid size one batch), with and without CUDA-graph replay.  Every
instance must reproduce its single-instance plan exactly (the kernels are the
same; only the batch offsets differ) and the FP64 oracle within the parity
tolerances."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
STEPS = 256


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_06282_gb300 import build as B
    B.build()


def lp():
    import paper_1909_06282_gb300 as L
    return L


def instances():
    out = []
    fr0s = [1e-6, 3e-5, 1e-4, 2e-5, 5e-6, 7e-5, 1e-5]
    sizes = [(32, 128.0)] * 2 + [(64, 256.0)] * 3 + [(96, 384.0)] * 2
    for i, ((n, box), f) in enumerate(zip(sizes, fr0s)):
        out.append(W.Instance(n, box, 11 + i, W.COSMO.replace(fr0_abs=f)))
    return out


@pytest.mark.parametrize("graph", [False, True])
def test_batched_matches_single_instance_plans(graph):
    L = lp()
    insts = instances()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plan = L.Plan(insts, n_steps=STEPS, stream=stream, graph=graph)
        for rep in range(2):   # second call replays the captured graph
            out = L.lpt2_displace(plan, psi1=True, psi2=True, pos=True)
            pk = L.lpt2_cic_pk(plan, pos=None, n_shells=16)
        stream.synchronize()
        d1, d2, _, _ = L.lpt2_growth_tables(plan)
        for j, it in enumerate(insts):
            single = L.Plan(it, n_steps=STEPS, stream=stream)
            ref = L.lpt2_displace(single, psi1=True, psi2=True, pos=True)
            rpk = L.lpt2_cic_pk(single, pos=None, n_shells=16)
            sd1, sd2, _, _ = L.lpt2_growth_tables(single)
            stream.synchronize()
            for key in ("psi1", "psi2", "pos"):
                got = plan.split(out[key], 3)[j].reshape(ref[key].shape)
                assert torch.equal(got, ref[key]), (j, key)
            torch.testing.assert_close(pk["pk"][j], rpk["pk"], rtol=1e-6, atol=0)
            assert torch.equal(pk["n_modes"][j], rpk["n_modes"])
            assert torch.equal(d1[j], sd1) and torch.equal(d2[j], sd2)


def test_batched_instance_against_oracle():
    from oracle import lpt2
    L = lp()
    insts = instances()
    plan = L.Plan(insts, n_steps=STEPS)
    out = L.lpt2_displace(plan, psi1=True, psi2=True, pos=False)
    j = 3   # second 64^3 instance
    it = insts[j]
    ref = lpt2.run(it.n, it.box, it.cosmo, seed=it.seed, n_steps=STEPS)
    for key in ("psi1", "psi2"):
        got = plan.split(out[key], 3)[j].reshape(3, it.n, it.n, it.n).cpu().numpy()
        rel = np.linalg.norm(got - ref[key]) / np.linalg.norm(ref[key])
        assert rel <= 2e-5, (key, rel)


def test_batched_rejects_bad_orderings():
    L = lp()
    a, b = W.Instance(32, 128.0, 1, W.COSMO), W.Instance(64, 256.0, 2, W.COSMO)
    with pytest.raises(L.LPT2Error):
        L.Plan([a, b, a])                                   # grid sizes not contiguous
    with pytest.raises(L.LPT2Error):
        L.Plan([a, W.Instance(32, 100.0, 3, W.COSMO)])      # same size, different box
    with pytest.raises(L.LPT2Error):
        L.Plan([a, W.Instance(32, 128.0, 3, W.COSMO.replace(sigma8=0.9))])
    p = L.Plan([a, b])
    with pytest.raises(L.LPT2Error):
        L.lpt2_displace_vjp(p)


def test_batched_96_workload_one_instance_per_size_against_oracle():
    """The real 96-instance batched workload (32 x 96^3/384, 128^3/512, 192^3/768 Mpc/h,
    seeds 1-96, |fR0| log-uniform in [1e-6, 1e-4]) as one plan, in the launch configuration
    the benchmark times (one CUDA graph): one instance of every grid size against the FP64
    oracle (Psi1, Psi2 within the parity tolerances, P(k) of its density per shell)."""
    from oracle import lpt2
    L = lp()
    insts = W.batched_96()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plan = L.Plan(insts, n_steps=1024, stream=stream, graph=True)
        out = L.lpt2_displace(plan, psi1=True, psi2=True, pos=False)
        pk = L.lpt2_cic_pk(plan, pos=None, n_shells=32)
        stream.synchronize()
    L.lpt2_device_status(plan)
    for j in (5, 32 + 17, 64 + 30):     # one 96^3, one 128^3, one 192^3 instance
        it = insts[j]
        ref = lpt2.run(it.n, it.box, it.cosmo, seed=it.seed, n_steps=1024)
        cell = it.box / it.n
        for key in ("psi1", "psi2"):
            got = plan.split(out[key], 3)[j].reshape(3, it.n, it.n, it.n).cpu().numpy()
            rel = np.linalg.norm(got - ref[key]) / np.linalg.norm(ref[key])
            mx = np.abs(got - ref[key]).max() / cell
            assert rel <= 2e-5 and mx <= 1e-4, (j, key, rel, mx)
        ok = ref["n_modes"] > 0
        np.testing.assert_array_equal(pk["n_modes"][j].cpu().numpy(), ref["n_modes"])
        np.testing.assert_allclose(pk["pk"][j].cpu().numpy()[ok], ref["pk"][ok], rtol=1e-4)


def test_tile_choices_are_bit_identical_and_autotuned():
    """The y-pass pencils per CTA (8, 16) and the x-pass tile path of the phi potentials
    (bulk-tensor tiles, global loads) change only how the same arithmetic is laid out on
    the GPU: Psi1, Psi2 and positions of a mixed batched plan, and the adjoint of a
    single-instance plan, are equal bit for bit under every choice; P(k) to 1e-6 (the
    particles that leave their CIC tile's halo are deposited with float atomics, whose
    order varies from run to run whatever the tiles).  Invalid choices are refused, and
    the autotuner leaves a valid one per group."""
    L = lp()
    insts = instances()   # groups 32^3, 64^3, 96^3
    plan = L.Plan(insts, n_steps=STEPS)
    assert L.lpt2_tiles(plan) == ([0, 0, 0], [0, 0, 0])

    def run():
        out = L.lpt2_displace(plan, psi1=True, psi2=True, pos=True)
        pk = L.lpt2_cic_pk(plan, pos=None, n_shells=16)
        torch.cuda.synchronize()
        return {k: v.clone() for k, v in out.items()}, pk["pk"].clone()

    ref, ref_pk = run()
    for yt in (8, 16):
        for xt in (1, 2):
            L.lpt2_set_tiles(plan, [yt] * 3, [xt] * 3)
            assert L.lpt2_tiles(plan) == ([yt] * 3, [xt] * 3)
            got, got_pk = run()
            for key in ("psi1", "psi2", "pos"):
                assert torch.equal(got[key], ref[key]), (yt, xt, key)
            torch.testing.assert_close(got_pk, ref_pk, rtol=1e-6, atol=0)
    for bad_y, bad_x in (([12, 8, 8], [0, 0, 0]), ([8, 8, 8], [0, 3, 0]), ([8, 8, 8], [-1, 0, 0])):
        with pytest.raises(L.LPT2Error):
            L.lpt2_set_tiles(plan, bad_y, bad_x)
    with pytest.raises(L.LPT2Error):
        L.lpt2_set_tiles(plan, [8, 8], [0, 0])                # one entry per group
    small = L.Plan(W.Instance(16, 64.0, 3, W.COSMO), n_steps=STEPS)
    with pytest.raises(L.LPT2Error):
        L.lpt2_set_tiles(small, [16], [0])                     # 16 pencils need N >= 32
    L.lpt2_set_tiles(small, [8], [2])
    L.lpt2_set_tiles(plan, [0, 0, 0], [0, 0, 0])
    L.lpt2_autotune(plan, n_shells=16, reps=1)
    yt, xt = L.lpt2_tiles(plan)
    assert all(v in (0, 8, 16) for v in yt) and all(v in (0, 1, 2) for v in xt)
    got, got_pk = run()
    for key in ("psi1", "psi2", "pos"):
        assert torch.equal(got[key], ref[key]), key

    single = L.Plan(W.Instance(64, 256.0, 5, W.COSMO), n_steps=STEPS)
    vjps = []
    for yt, xt in ((0, 0), (16, 2), (8, 1)):
        L.lpt2_set_tiles(single, [yt], [xt])
        g_noise, g_t = L.lpt2_displace_vjp(single, g_density=torch.full((64 ** 3,), 1e-3, device="cuda"))
        torch.cuda.synchronize()
        vjps.append((g_noise.clone(), g_t.clone()))
    for g_noise, g_t in vjps[1:]:
        assert torch.equal(g_noise, vjps[0][0]) and torch.equal(g_t, vjps[0][1])
