"""Caller-owned memory, checked on the host: every device allocation of the library is
made by lpt2_plan (the source has no other cudaMalloc), and the plan-free size query
lpt2_workspace_bytes covers the buffers of lpt2_displace_host (LPT2_HOST_IO) and the
output-time tables of lpt2_set_outputs (LPT2_MAX_OUTPUTS) with the documented sizes."""
import ctypes as C
import os
import re

import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1909_06282_gb300", "csrc")


@pytest.fixture(scope="module")
def L():
    from paper_1909_06282_gb300 import build as B
    B.build()
    import paper_1909_06282_gb300 as lib
    return lib


def up256(b):
    return (b + 255) // 256 * 256


def test_only_lpt2_plan_allocates_device_memory():
    api = open(os.path.join(CSRC, "api.cu")).read()
    # the one cudaMalloc sits in plan_malloc
    assert len(re.findall(r"\bcudaMalloc\w*\s*\(", api)) == 1
    body = api[api.index("cudaError_t plan_malloc("):]
    assert re.search(r"\bcudaMalloc\s*\(", body[:body.index("\n}\n")])
    # plan_malloc is called from lpt2_plan only
    plan_body = api[api.index("int lpt2_plan(lpt2_plan_t* out"):]
    plan_body = plan_body[:plan_body.index("\n}\n")]
    calls = [m.start() for m in re.finditer(r"plan_malloc\(\(void", api)]
    start = api.index(plan_body)
    assert calls and all(start <= c < start + len(plan_body) for c in calls)
    for f in os.listdir(CSRC):
        if f.endswith((".cu", ".cuh", ".h")) and f != "api.cu":
            src = open(os.path.join(CSRC, f)).read()
            assert not re.search(r"\bcuda(Malloc|MallocAsync|MallocManaged|MallocHost|HostAlloc)\s*\(", src), f


def test_workspace_bytes_without_a_gpu(L):
    n, nk = 64, 512
    inst = W.Instance(n, 256.0, 1, W.COSMO)
    base = L.lpt2_workspace_bytes(inst, n_k=nk)
    n3 = n ** 3
    hio_set = up256(up256(up256(n3 * 4) + 3 * n3 * 4) + 256 * 8)
    assert L.lpt2_workspace_bytes(inst, n_k=nk, host_io=True) - base == 2 * hio_set
    length = 3 * (n // 2) ** 2 + 1
    out_each = up256(up256(up256(up256(4 * nk * 8) + 4 * nk * 4) + length * 16) + length * 8)
    for m in (1, 3, 64):
        assert L.lpt2_workspace_bytes(inst, n_k=nk, max_outputs=m) - base == m * out_each
    both = L.lpt2_workspace_bytes(inst, n_k=nk, host_io=True, max_outputs=2)
    assert both - base == 2 * hio_set + 2 * out_each
    # 21 slots of N^3 floats and the density lead the layout
    assert base >= 22 * n3 * 4
    # batched: the slots follow the largest group, the density covers every instance
    two = [W.Instance(32, 64.0, 1, W.COSMO), W.Instance(64, 128.0, 2, W.COSMO)]
    assert L.lpt2_workspace_bytes(two, n_k=nk) > L.lpt2_workspace_bytes(two[1], n_k=nk)


def test_workspace_bytes_rejects_what_lpt2_plan_rejects(L):
    inst = W.Instance(64, 256.0, 1, W.COSMO)
    two = [inst, W.Instance(64, 256.0, 2, W.COSMO)]
    with pytest.raises(L.LPT2Error) as ei:
        L.lpt2_workspace_bytes(two, host_io=True)          # host buffers: single-instance plans
    assert ei.value.code == -1
    with pytest.raises(L.LPT2Error):
        L.lpt2_workspace_bytes(two, max_outputs=2)
    with pytest.raises(L.LPT2Error):
        L.lpt2_workspace_bytes(inst, max_outputs=65)
    with pytest.raises(L.LPT2Error) as ei:
        L.lpt2_workspace_bytes(W.Instance(100, 256.0, 1, W.COSMO))
    assert ei.value.code == -4
    lib = L.load_library()
    nb = C.c_size_t()
    from paper_1909_06282_gb300._lib import _instances
    assert lib.lpt2_workspace_bytes(_instances([inst]), 1, 512, 1 << 4, C.byref(nb)) == -1   # unknown flag
    assert lib.lpt2_workspace_bytes(None, 1, 512, 0, C.byref(nb)) == -1


def test_injected_allocation_failure_on_the_host(L):
    """With the first allocation made to fail, lpt2_plan returns LPT2_ENOMEM, hands back no
    plan and leaves nothing allocated (runs without a GPU: the failure comes before any
    device call)."""
    from paper_1909_06282_gb300._lib import _instances
    lib = L.load_library()
    base = L.lpt2_debug_alloc_hook(0)
    try:
        h = C.c_void_p()
        rc = lib.lpt2_plan(C.byref(h), _instances([W.Instance(32, 64.0, 1, W.COSMO)]), 1, 64, 1e-4, 10.0, 16,
                           None, 0)
        assert rc == -2 and h.value is None
        assert "allocation" in L.lpt2_last_error()
    finally:
        assert L.lpt2_debug_alloc_hook(-1) == base
    with pytest.raises(L.LPT2Error):
        L.lpt2_debug_alloc_hook(-2)
