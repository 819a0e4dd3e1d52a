"""GPU P(k) estimator refinements (lpt2_cic_pk_est: CIC window deconvolution and
interlacing) against the FP64 oracle (oracle/pkest.py) on the same seeded positions:
shell P(k) <= 1e-4 relative, mode counts exact, flags = 0 equal to lpt2_cic_pk."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_06282_gb300 import build as B
    B.build()
    import paper_1909_06282_gb300 as L
    return L


@pytest.mark.parametrize("n,box", [(32, 128.0), (64, 200.0), (96, 300.0)])
@pytest.mark.parametrize("deconvolve,interlace", [(True, False), (False, True), (True, True)])
def test_pk_est_against_oracle(lib, n, box, deconvolve, interlace):
    from oracle import pkest
    plan = lib.Plan(W.Instance(n, box, 1, W.COSMO), n_steps=64)
    pos = W.random_positions(n, box, 7)
    res = lib.lpt2_cic_pk_est(plan, pos=torch.from_numpy(pos).cuda(), n_shells=16,
                              deconvolve=deconvolve, interlace=interlace)
    pk, km, cnt = pkest.power_spectrum_est(n, box, pos.astype(np.float64), 16, deconvolve, interlace)
    ok = cnt > 0
    np.testing.assert_array_equal(res["n_modes"].cpu().numpy(), cnt)
    np.testing.assert_allclose(res["pk"].cpu().numpy()[ok], pk[ok], rtol=1e-4)
    np.testing.assert_allclose(res["k_mean"].cpu().numpy()[ok], km[ok], rtol=1e-6)


def test_pk_est_without_flags_is_cic_pk(lib):
    n, box = 32, 128.0
    plan = lib.Plan(W.Instance(n, box, 1, W.COSMO), n_steps=64)
    pos = torch.from_numpy(W.random_positions(n, box, 8)).cuda()
    a = lib.lpt2_cic_pk(plan, pos=pos, n_shells=16)
    b = lib.lpt2_cic_pk_est(plan, pos=pos, n_shells=16)
    # the same kernels; the deposit's cross-CTA atomic adds make the last bits run-dependent
    torch.testing.assert_close(a["pk"], b["pk"], rtol=1e-6, atol=0)
    assert torch.equal(a["n_modes"], b["n_modes"])


def test_pk_est_rejects_interlacing_without_positions(lib):
    plan = lib.Plan(W.Instance(32, 128.0, 1, W.COSMO), n_steps=64)
    lib.lpt2_displace(plan, psi1=False, psi2=False, pos=False)
    with pytest.raises(lib.LPT2Error):
        lib.lpt2_cic_pk_est(plan, pos=None, n_shells=16, interlace=True)
    lib.lpt2_cic_pk_est(plan, pos=None, n_shells=16, deconvolve=True)   # the displaced density
