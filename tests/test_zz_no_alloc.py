"""lpt2_cic_pk_noalloc: the allocation-free CIC + P(k) entry point.

Some callers may not allocate GPU memory (their device memory belongs to their
own pool, or cudaMalloc is forbidden where they run), so they cannot make a
plan or a workspace.  This entry point keeps its scratch in a static device
array inside the library.  Its results must match the plan-based lpt2_cic_pk,
call after call (the shared scratch keeps the previous call's contents).
Collected last so that a failure here leaves every other test already run.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PK_REL = 1e-4


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_06282_gb300 import build as B
    B.build()
    import paper_1909_06282_gb300 as L
    return L


def call_noalloc(L, n, box, pos, n_shells=32):
    lib = L.load_library()
    pk = torch.empty(n_shells, dtype=torch.float64, device="cuda")
    km = torch.empty(n_shells, dtype=torch.float64, device="cuda")
    nm = torch.empty(n_shells, dtype=torch.int64, device="cuda")
    dens = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.lpt2_cic_pk_noalloc(n, box, C.c_void_p(pos.data_ptr()), C.c_void_p(dens.data_ptr()),
                                 C.c_void_p(pk.data_ptr()), C.c_void_p(km.data_ptr()),
                                 C.c_void_p(nm.data_ptr()), n_shells, stream)
    assert rc == 0, L.lpt2_last_error()
    torch.cuda.synchronize()
    return dict(pk=pk.cpu().numpy(), k_mean=km.cpu().numpy(), n_modes=nm.cpu().numpy(),
                density=dens.cpu().numpy())


def reference(L, n, box, pos, n_shells=32):
    plan = L.Plan(W.Instance(n, box, 1, W.COSMO), n_steps=16)
    r = L.lpt2_cic_pk(plan, pos=pos, density=True, n_shells=n_shells)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in r.items()}


def check_same(got, want):
    np.testing.assert_array_equal(got["n_modes"], want["n_modes"])
    ok = want["n_modes"] > 0
    np.testing.assert_allclose(got["pk"][ok], want["pk"][ok], rtol=PK_REL)
    np.testing.assert_allclose(got["k_mean"][ok], want["k_mean"][ok], rtol=1e-6)
    assert np.max(np.abs(got["density"] - want["density"])) < 2e-5 * max(1.0, np.abs(want["density"]).max())


@pytest.mark.parametrize("n,box", [(64, 256.0), (128, 300.0), (32, 100.0)])
def test_noalloc_matches_plan_entry_point_two_calls(lib, n, box):
    pos_a = torch.from_numpy(W.random_positions(n, box, 21)).cuda()
    pos_b = torch.from_numpy(W.random_positions(n, box, 22)).cuda()
    want_a = reference(lib, n, box, pos_a)
    want_b = reference(lib, n, box, pos_b)
    check_same(call_noalloc(lib, n, box, pos_a), want_a)   # first call
    check_same(call_noalloc(lib, n, box, pos_b), want_b)   # second call reuses the same scratch
    check_same(call_noalloc(lib, n, box, pos_a), want_a)


def test_noalloc_against_oracle_128(lib):
    """The no-allocation entry point against the FP64 oracle directly (CIC density and
    shell P(k) of seeded lattice-plus-jitter positions at 128^3), on two calls in a row."""
    from oracle import lpt2
    n, box = 128, 512.0
    for seed in (31, 32):
        pos = W.random_positions(n, box, seed)
        got = call_noalloc(lib, n, box, torch.from_numpy(pos).cuda())
        want = lpt2.cic_density(n, box, pos.astype(np.float64))
        assert np.max(np.abs(got["density"] - want.reshape(n, n, n))) < 2e-5 * max(1.0, np.abs(want).max())
        pk, km, cnt = lpt2.power_spectrum(n, box, want, 32)
        np.testing.assert_array_equal(got["n_modes"], cnt)
        ok = cnt > 0
        np.testing.assert_allclose(got["pk"][ok], pk[ok], rtol=PK_REL)
        np.testing.assert_allclose(got["k_mean"][ok], km[ok], rtol=1e-6)


def test_noalloc_rejects_sizes_beyond_its_static_scratch(lib):
    L = lib
    pk = torch.empty(32, dtype=torch.float64, device="cuda")
    pos = torch.zeros(3 * 16 ** 3, dtype=torch.float32, device="cuda")
    rc = L.load_library().lpt2_cic_pk_noalloc(256, 100.0, C.c_void_p(pos.data_ptr()), None,
                                              C.c_void_p(pk.data_ptr()), None, None, 32, None)
    assert rc == -4
    assert "128" in L.lpt2_last_error()
    rc = L.load_library().lpt2_cic_pk_noalloc(64, 100.0, C.c_void_p(pos.data_ptr()), None,
                                              C.c_void_p(pk.data_ptr()), None, None, 300, None)
    assert rc == -1
