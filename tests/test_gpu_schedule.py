"""GPU tests of the launch schedule of batched plans (lpt2_schedule, lpt2_set_schedule,
lpt2_autotune): running a grid-size group in chunks of instances changes only how the
launches are cut, so positions must equal the whole-group run bit for bit and P(k) agree
to 1e-6 (CIC float reductions may add in another order), with and without CUDA graphs."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NS = 16


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_06282_gb300 import build as B
    B.build()
    import paper_1909_06282_gb300 as lib
    return lib


def instances():
    rng = np.random.default_rng(3)
    out = []
    for n, box, cnt in ((32, 64.0, 6), (64, 128.0, 4), (96, 192.0, 3)):
        for _ in range(cnt):
            fr0 = float(10 ** rng.uniform(-6, -4))
            out.append(W.Instance(n, box, len(out) + 1, W.COSMO.replace(fr0_abs=fr0)))
    return out


def run(L, plan, stream):
    pos = torch.empty(3 * plan.cells, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        L.lpt2_displace(plan, psi1=False, psi2=False, pos=pos)
        pk = L.lpt2_cic_pk(plan, pos=None, n_shells=NS)["pk"]
    stream.synchronize()
    return pos.cpu(), pk.cpu().numpy()


@pytest.mark.parametrize("graph", [False, True])
def test_chunked_schedule_gives_the_same_outputs(L, graph):
    st = torch.cuda.Stream()
    plan = L.Plan(instances(), n_steps=128, stream=st, graph=graph)
    assert L.lpt2_schedule(plan) == [6, 4, 3]
    pos0, pk0 = run(L, plan, st)
    for sched in ([1, 3, 2], [4, 1, 1], [100, 2, 3]):
        L.lpt2_set_schedule(plan, sched)
        assert L.lpt2_schedule(plan) == [min(c, m) for c, m in zip(sched, (6, 4, 3))]
        pos, pk = run(L, plan, st)
        assert torch.equal(pos, pos0), sched
        np.testing.assert_allclose(pk, pk0, rtol=1e-6, atol=0)
    L.lpt2_device_status(plan)


def test_autotune_keeps_outputs_and_picks_valid_chunks(L):
    st = torch.cuda.Stream()
    plan = L.Plan(instances(), n_steps=128, stream=st, graph=True)
    pos0, pk0 = run(L, plan, st)
    with torch.cuda.stream(st):
        sched = L.lpt2_autotune(plan, n_shells=NS, reps=2)
    assert len(sched) == 3 and all(1 <= c <= m for c, m in zip(sched, (6, 4, 3)))
    pos, pk = run(L, plan, st)
    assert torch.equal(pos, pos0)
    np.testing.assert_allclose(pk, pk0, rtol=1e-6, atol=0)


def test_schedule_errors(L):
    plan = L.Plan(instances(), n_steps=64)
    with pytest.raises(L.LPT2Error):
        L.lpt2_set_schedule(plan, [1, 1])          # three groups
    with pytest.raises(L.LPT2Error):
        L.lpt2_set_schedule(plan, [1, 0, 1])
    with pytest.raises(L.LPT2Error):
        L.lpt2_autotune(plan, n_shells=NS, reps=0)
    single = L.Plan(W.Instance(32, 64.0, 1, W.COSMO), n_steps=64)
    assert L.lpt2_schedule(single) == [1]
