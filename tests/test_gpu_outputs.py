"""GPU tests of several output times from one realisation (lpt2_set_outputs,
lpt2_displace_outputs).

The prefix noise -> delta(k) -> phi_ij -> S(k) does not depend on the output scale
factor; after it, each a_j runs the same kernels as a plan made with a_out = a_j.  So
each a_j's positions must equal that plan's bit for bit and its P(k) agree to 1e-6
relative (the CIC flush adds floats in a run-dependent order).  The FP64 oracle run at
a_out = 0.5 pins an a != 1 output directly (the parity tolerances of the one-a path)."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NS = 32


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_06282_gb300 import build as B
    B.build()
    import paper_1909_06282_gb300 as lib
    return lib


def single_a(L, n, box, seed, cosmo, a, n_steps, noise=None):
    plan = L.Plan(W.Instance(n, box, seed, cosmo, a_out=a), n_steps=n_steps)
    pos = torch.empty((3, n, n, n), dtype=torch.float32, device="cuda")
    L.lpt2_displace(plan, noise=noise, psi1=False, psi2=False, pos=pos)
    res = L.lpt2_cic_pk(plan, pos=None, n_shells=NS)
    torch.cuda.synchronize()
    return pos, res


@pytest.mark.parametrize("noise_seed", [None, 21])
def test_each_output_equals_a_plan_at_that_a(L, noise_seed):
    n, box, seed, steps = 64, 128.0, 4, 512
    a_list = [0.5, 0.8, 1.0, 0.25]
    noise = None if noise_seed is None else torch.from_numpy(W.white_noise(n, noise_seed)).cuda()
    plan = L.Plan(W.Instance(n, box, seed, W.COSMO), n_steps=steps, max_outputs=4)
    L.lpt2_set_outputs(plan, a_list)
    out = L.lpt2_displace_outputs(plan, noise=noise, pos=True, n_shells=NS)
    torch.cuda.synchronize()
    for j, a in enumerate(a_list):
        pos, res = single_a(L, n, box, seed, W.COSMO, a, steps, noise)
        assert torch.equal(out["pos"][j], pos), a
        np.testing.assert_allclose(out["pk"][j].cpu().numpy(), res["pk"].cpu().numpy(), rtol=1e-6, atol=0)
    assert torch.equal(out["n_modes"].cpu(), res["n_modes"].cpu())
    np.testing.assert_allclose(out["k_mean"].cpu().numpy(), res["k_mean"].cpu().numpy(), rtol=1e-12)
    # growth: the earlier output has smaller displacements and less power on large scales
    assert float(out["pk"][0, 1]) < float(out["pk"][2, 1])


def test_output_at_half_against_oracle(L):
    from oracle import lpt2
    n, box, seed = 32, 64.0, 2
    plan = L.Plan(W.Instance(n, box, seed, W.COSMO), n_steps=1024, max_outputs=2)
    L.lpt2_set_outputs(plan, [1.0, 0.5])
    out = L.lpt2_displace_outputs(plan, pos=True, n_shells=NS)
    ref = lpt2.run(n, box, W.COSMO, seed=seed, a_out=0.5, n_steps=1024)
    p64 = out["pos"][1].double().cpu().numpy().reshape(3, -1)
    d = p64 - ref["pos"]
    d -= box * np.round(d / box)
    assert np.abs(d).max() <= 1e-4 * box / n
    pk_o = lpt2.power_spectrum(n, box, lpt2.cic_density(n, box, p64), NS)[0]
    ok = pk_o > 0
    np.testing.assert_allclose(out["pk"][1].cpu().numpy()[ok], pk_o[ok], rtol=1e-4)


def test_set_fr0_refreshes_the_output_tables(L):
    n, box, seed, steps = 32, 64.0, 3, 256
    plan = L.Plan(W.Instance(n, box, seed, W.COSMO), n_steps=steps, max_outputs=2)
    L.lpt2_set_outputs(plan, [0.6, 1.0])
    L.lpt2_set_fr0(plan, 1e-6)
    out = L.lpt2_displace_outputs(plan, pos=True, n_shells=NS)
    cosmo6 = W.COSMO.replace(fr0_abs=1e-6)
    for j, a in enumerate([0.6, 1.0]):
        pos, _ = single_a(L, n, box, seed, cosmo6, a, steps)
        assert torch.equal(out["pos"][j], pos), a


def test_full_size_two_outputs(L):
    """512^3, L = 1024 Mpc/h, |fR0| = 1e-5 (the throughput configuration), outputs at
    z = 1 and z = 0: each equals a one-output plan at that a."""
    n, box, steps = 512, 1024.0, 1024
    plan = L.Plan(W.Instance(n, box, 1, W.COSMO), n_steps=steps, max_outputs=2)
    L.lpt2_set_outputs(plan, [0.5, 1.0])
    out = L.lpt2_displace_outputs(plan, pos=True, n_shells=NS)
    torch.cuda.synchronize()
    L.lpt2_device_status(plan)
    for j, a in enumerate([0.5, 1.0]):
        pos, res = single_a(L, n, box, 1, W.COSMO, a, steps)
        assert torch.equal(out["pos"][j], pos), a
        np.testing.assert_allclose(out["pk"][j].cpu().numpy(), res["pk"].cpu().numpy(), rtol=1e-6, atol=0)
        del pos, res


def test_argument_errors(L):
    import ctypes as C
    from paper_1909_06282_gb300._lib import load_library
    n = 32
    plan = L.Plan(W.Instance(n, 64.0, 1, W.COSMO), n_steps=64, max_outputs=4)
    pk = torch.empty(NS, dtype=torch.float64, device="cuda")
    # no output list yet
    rc = load_library().lpt2_displace_outputs(plan.handle, None, None, C.c_void_p(pk.data_ptr()), None, None, NS)
    assert rc != 0 and "lpt2_set_outputs" in L.lpt2_last_error()
    for bad in ([], [0.0], [1e-4], [1.5], [0.5, float("nan")]):
        with pytest.raises(L.LPT2Error):
            L.lpt2_set_outputs(plan, bad)
    batched = L.Plan([W.Instance(32, 64.0, s, W.COSMO) for s in (1, 2)], n_steps=64)
    with pytest.raises(L.LPT2Error):
        L.lpt2_set_outputs(batched, [0.5])
    # more output times than the plan reserved room for in its workspace
    with pytest.raises(L.LPT2Error, match="LPT2_MAX_OUTPUTS"):
        L.lpt2_set_outputs(plan, [0.2, 0.4, 0.6, 0.8, 1.0])
    small = L.Plan(W.Instance(n, 64.0, 1, W.COSMO), n_steps=64)
    with pytest.raises(L.LPT2Error, match="LPT2_MAX_OUTPUTS"):
        L.lpt2_set_outputs(small, [0.5])


def test_output_tables_follow_a_new_workspace(L):
    """The output tables live in the workspace: after lpt2_set_workspace with another
    buffer they are recomputed there and the outputs are unchanged."""
    n, box, seed, steps = 32, 64.0, 3, 256
    plan = L.Plan(W.Instance(n, box, seed, W.COSMO), n_steps=steps, max_outputs=2)
    L.lpt2_set_outputs(plan, [0.6, 1.0])
    first = L.lpt2_displace_outputs(plan, pos=True, n_shells=NS)["pos"].clone()
    import ctypes as C
    from paper_1909_06282_gb300._lib import load_library
    ws2 = torch.full_like(plan.workspace, 0x7F)
    assert load_library().lpt2_set_workspace(plan.handle, C.c_void_p(ws2.data_ptr()), ws2.numel()) == 0
    plan.workspace = ws2
    second = L.lpt2_displace_outputs(plan, pos=True, n_shells=NS)["pos"]
    assert torch.equal(first, second)
