"""Failure detection on the GPU, in forms that fault, trap or hang nothing.

- Bounded waits: with a wait budget of 0 every consumer wait of the bulk-copy rings
  (z_source, z_final) gives up at once without looking at its barrier.  The copies are
  real and land; each CTA waits for its own copies in flight (default budget), sets the
  plan's device error word and returns.  lpt2_device_status must report LPT2_ETIMEOUT
  once, clear the word, and with the budget restored the same call must give the normal
  result.  The workspace is zeroed first, so the passes after a CTA that gave up see
  finite data.
- Allocation failure: every device allocation is made by lpt2_plan; making the k-th one
  fail must return LPT2_ENOMEM, leave no plan and free every allocation already made.
"""
import gc

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_06282_gb300 import build as B
    B.build()
    import paper_1909_06282_gb300 as lib
    return lib


def test_bounded_wait_timeout_is_reported_and_cleared(L):
    n = 32
    plan = L.Plan(W.Instance(n, 128.0, 1, W.COSMO), n_steps=64)
    plan.workspace.zero_()
    pos_ref = L.lpt2_displace(plan, psi1=False, psi2=False, pos=True)["pos"].clone()
    L.lpt2_device_status(plan)                       # clean so far
    L.lpt2_set_wait_budget(plan, 0)
    pos = torch.zeros_like(pos_ref)
    L.lpt2_displace(plan, psi1=False, psi2=False, pos=pos)
    with pytest.raises(L.LPT2Error) as ei:
        L.lpt2_device_status(plan)
    assert ei.value.code == -5 and "bounded device-side wait" in str(ei.value)
    L.lpt2_device_status(plan)                       # the word was cleared
    L.lpt2_set_wait_budget(plan, 2_000_000_000)
    again = L.lpt2_displace(plan, psi1=False, psi2=False, pos=True)["pos"]
    L.lpt2_device_status(plan)
    assert torch.equal(again, pos_ref)


def test_bounded_wait_timeout_in_the_adjoint_source_pass(L):
    n = 32
    plan = L.Plan(W.Instance(n, 128.0, 1, W.COSMO), n_steps=64)
    plan.workspace.zero_()
    gd = torch.zeros((n, n, n), dtype=torch.float32, device="cuda")
    L.lpt2_set_wait_budget(plan, 0)
    L.lpt2_displace_vjp(plan, g_density=gd, n_shells=8)
    with pytest.raises(L.LPT2Error) as ei:
        L.lpt2_device_status(plan)
    assert ei.value.code == -5
    L.lpt2_device_status(plan)


def test_every_plan_allocation_failure_returns_enomem_and_frees(L):
    insts = [W.Instance(32, 64.0, 1, W.COSMO), W.Instance(64, 128.0, 2, W.COSMO)]
    gc.collect()   # plans of earlier tests awaiting collection would free theirs mid-count
    base = L.lpt2_debug_alloc_hook(-1)
    ok = L.Plan(insts, n_steps=16, workspace=False)
    n_alloc = L.lpt2_debug_alloc_hook(-1) - base      # allocations a two-group plan makes
    ok.close()
    assert L.lpt2_debug_alloc_hook(-1) == base and n_alloc >= 10
    try:
        for k in range(n_alloc):
            L.lpt2_debug_alloc_hook(k)
            with pytest.raises(L.LPT2Error) as ei:
                L.Plan(insts, n_steps=16, workspace=False)
            assert ei.value.code == -2, (k, ei.value)
            assert L.lpt2_debug_alloc_hook(-1) == base, k   # nothing leaked
    finally:
        L.lpt2_debug_alloc_hook(-1)
    p = L.Plan(insts, n_steps=16, workspace=False)     # and it works again
    p.close()
    assert L.lpt2_debug_alloc_hook(-1) == base
