"""Argument checks of the Python binding that run before any library call, tested on
CPU with a stand-in plan object (no handle is ever passed to the library here)."""
import types

import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    import paper_1909_06282_gb300 as lib
    return lib


def fake_plan(n=16):
    return types.SimpleNamespace(n=n, handle=None, n_inst=1, cells=n ** 3)


def test_displace_host_rejects_device_and_misshaped_buffers(L):
    p = fake_plan()
    n3 = p.n ** 3
    with pytest.raises(ValueError):   # wrong dtype
        L.lpt2_displace_host(p, 1, pos=torch.empty(3 * n3, dtype=torch.float64))
    with pytest.raises(ValueError):   # neither one realisation nor n_real of them
        L.lpt2_displace_host(p, 2, pos=torch.empty(5 * 3 * n3, dtype=torch.float32))
    with pytest.raises(ValueError):
        L.lpt2_displace_host(p, 3, noise=torch.empty(2 * n3, dtype=torch.float32),
                             pk=torch.empty(32, dtype=torch.float64))
    with pytest.raises(ValueError):
        L.lpt2_displace_host(p, 1, pk=torch.empty(31, dtype=torch.float64), n_shells=32)
    with pytest.raises(ValueError):   # host tensors must be contiguous
        L.lpt2_displace_host(p, 1, pk=torch.empty((32, 2), dtype=torch.float64)[:, 0], n_shells=32)


def test_displace_outputs_needs_an_output_list(L):
    with pytest.raises(ValueError):
        L.lpt2_displace_outputs(fake_plan(), pos=False)
