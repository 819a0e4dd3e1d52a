"""GPU tests of lpt2_displace_host, the forward step from and to host memory.

The host path runs the same kernels as lpt2_displace + lpt2_cic_pk on device buffers,
with the copies pipelined over realisations, so its positions must equal the device
path's bit for bit (the position kernels are deterministic) and its P(k) agree to
1e-6 relative (the CIC flush adds floats to the density in a run-dependent order).  One
case also checks the host path's P(k) directly against the FP64 oracle (1e-4 per shell,
the parity tolerance of the device path)."""
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


def device_step(L, plan, noise=None):
    n = plan.n
    pos = torch.empty((3, n, n, n), dtype=torch.float32, device="cuda")
    L.lpt2_displace(plan, noise=None if noise is None else torch.from_numpy(noise).cuda(),
                    psi1=False, psi2=False, pos=pos)
    pk = L.lpt2_cic_pk(plan, pos=None, n_shells=NS)["pk"]
    torch.cuda.synchronize()
    return pos.cpu(), pk.cpu()


def test_philox_noise_matches_device_path(L):
    n = 64
    plan = L.Plan(W.Instance(n, 128.0, 5, W.COSMO), n_steps=256, host_io=True)
    pos_ref, pk_ref = device_step(L, plan)
    pos = torch.empty((3, n, n, n), dtype=torch.float32).pin_memory()
    pk = torch.empty(NS, dtype=torch.float64).pin_memory()
    L.lpt2_displace_host(plan, 1, noise=None, pos=pos, pk=pk, n_shells=NS)
    assert torch.equal(pos, pos_ref)
    np.testing.assert_allclose(pk.numpy(), pk_ref.numpy(), rtol=1e-6, atol=0)


@pytest.mark.parametrize("pinned", [True, False])
def test_three_realisations_each_match(L, pinned):
    """Three host noise fields in one call (strided buffers): realisation r's outputs
    equal the device path run on noise r."""
    n, R = 64, 3
    plan = L.Plan(W.Instance(n, 128.0, 1, W.COSMO), n_steps=256, host_io=True)
    noise = np.stack([W.white_noise(n, 100 + r) for r in range(R)])
    noise_h = torch.from_numpy(noise)
    pos = torch.empty((R, 3, n, n, n), dtype=torch.float32)
    pk = torch.empty((R, NS), dtype=torch.float64)
    if pinned:
        noise_h, pos, pk = noise_h.pin_memory(), pos.pin_memory(), pk.pin_memory()
    L.lpt2_displace_host(plan, R, noise=noise_h, pos=pos, pk=pk, n_shells=NS)
    for r in range(R):
        pos_ref, pk_ref = device_step(L, plan, noise[r])
        assert torch.equal(pos[r], pos_ref), r
        np.testing.assert_allclose(pk[r].numpy(), pk_ref.numpy(), rtol=1e-6, atol=0)
    assert not torch.equal(pos[0], pos[1])


def test_shared_buffers_keep_the_last_realisation(L):
    """Stride 0: one noise buffer feeds every realisation and one position buffer
    receives every download; what remains is the last realisation's result."""
    n, R = 32, 4
    plan = L.Plan(W.Instance(n, 64.0, 1, W.COSMO), n_steps=256, host_io=True)
    noise = np.stack([W.white_noise(n, 7 + r) for r in range(R)])
    pos = torch.empty((3, n, n, n), dtype=torch.float32).pin_memory()
    pk = torch.empty(NS, dtype=torch.float64).pin_memory()
    L.lpt2_displace_host(plan, R, noise=torch.from_numpy(noise).pin_memory(), pos=pos, pk=pk, n_shells=NS)
    pos_ref, pk_ref = device_step(L, plan, noise[-1])
    assert torch.equal(pos, pos_ref)
    np.testing.assert_allclose(pk.numpy(), pk_ref.numpy(), rtol=1e-6, atol=0)
    # one shared noise buffer: every realisation is the same, so the last equals the first
    one = torch.from_numpy(noise[0]).pin_memory()
    pk_all = torch.empty((R, NS), dtype=torch.float64)
    L.lpt2_displace_host(plan, R, noise=one, pos=None, pk=pk_all, n_shells=NS)
    for r in range(1, R):
        np.testing.assert_allclose(pk_all[r].numpy(), pk_all[0].numpy(), rtol=1e-6, atol=0)


def test_host_path_against_oracle(L):
    from oracle import lpt2
    n, box = 32, 64.0
    inst = W.Instance(n, box, 3, W.COSMO)
    noise = W.white_noise(n, 11)
    plan = L.Plan(inst, n_steps=1024, host_io=True)
    pos = torch.empty((3, n, n, n), dtype=torch.float32)
    pk = torch.empty(NS, dtype=torch.float64)
    L.lpt2_displace_host(plan, 1, noise=torch.from_numpy(noise), pos=pos, pk=pk, n_shells=NS)
    ref = lpt2.run(n, box, inst.cosmo, seed=3, noise=noise, n_steps=1024)
    p64 = pos.double().numpy().reshape(3, -1)
    d = p64 - ref["pos"]
    d -= box * np.round(d / box)
    assert np.abs(d).max() <= 1e-4 * box / n
    # P(k): the oracle's CIC and shells of the same (FP32) positions
    pk_o = lpt2.power_spectrum(n, box, lpt2.cic_density(n, box, p64), NS)[0]
    ok = pk_o > 0
    np.testing.assert_allclose(pk.numpy()[ok], pk_o[ok], rtol=1e-4)


def test_full_size_two_realisations(L):
    """512^3, L = 1024 Mpc/h (the throughput configuration): two host noise fields, one
    shared pinned position buffer; P(k) of each equals the device path's."""
    n = 512
    plan = L.Plan(W.Instance(n, 1024.0, 1, W.COSMO), n_steps=1024, host_io=True)
    noise = torch.from_numpy(np.stack([W.white_noise(n, 1000 + r) for r in range(2)])).pin_memory()
    pos = torch.empty((3, n, n, n), dtype=torch.float32).pin_memory()
    pk = torch.empty((2, NS), dtype=torch.float64).pin_memory()
    L.lpt2_displace_host(plan, 2, noise=noise, pos=pos, pk=pk, n_shells=NS)
    for r in range(2):
        pos_ref, pk_ref = device_step(L, plan, noise[r].numpy())
        np.testing.assert_allclose(pk[r].numpy(), pk_ref.numpy(), rtol=1e-6, atol=0)
    assert torch.equal(pos, pos_ref)
    L.lpt2_device_status(plan)


def test_argument_errors(L):
    n = 32
    plan = L.Plan(W.Instance(n, 64.0, 1, W.COSMO), n_steps=64, host_io=True)
    pk = torch.empty(NS, dtype=torch.float64)
    with pytest.raises(L.LPT2Error):
        L.lpt2_displace_host(plan, 0, pk=pk, n_shells=NS)
    with pytest.raises(L.LPT2Error):
        L.lpt2_displace_host(plan, 1, pos=None, pk=None, n_shells=NS)
    with pytest.raises(L.LPT2Error):
        L.lpt2_displace_host(plan, 1, pk=torch.empty(300, dtype=torch.float64), n_shells=300)
    with pytest.raises(ValueError):
        L.lpt2_displace_host(plan, 1, pk=pk.cuda(), n_shells=NS)
    with pytest.raises(ValueError):
        L.lpt2_displace_host(plan, 2, pos=torch.empty((5, 3, n, n, n)), n_shells=NS)
