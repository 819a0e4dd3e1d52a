"""Degenerate and edge inputs of the GPU path against exact answers or the FP64 oracle:
zero noise, every particle at one point (the fixed-point CIC window at its heaviest
load), particles far from their Lagrangian tiles (the direct-deposit fallback), and the
extreme shell counts."""
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


def test_zero_noise_gives_the_lattice(lib):
    n, box = 32, 64.0
    plan = lib.Plan(W.Instance(n, box, 1, W.COSMO), n_steps=64)
    z = torch.zeros((n, n, n), dtype=torch.float32, device="cuda")
    out = lib.lpt2_displace(plan, noise=z, psi1=True, psi2=True, pos=True)
    assert bool((out["psi1"] == 0).all()) and bool((out["psi2"] == 0).all())
    q = torch.from_numpy(np.indices((n, n, n)).astype(np.float32) * np.float32(box / n)).cuda()
    assert torch.equal(out["pos"], q)
    res = lib.lpt2_cic_pk(plan, pos=None, density=True, n_shells=8)
    assert bool((res["density"] == 0).all()) and bool((res["pk"] == 0).all())


@pytest.mark.parametrize("point", [(0.0, 0.0, 0.0), (10.3, 63.99, 31.25)])
def test_all_particles_at_one_point(lib, point):
    """N^3 unit masses in the 8 cells around one point: the window sums of a tile hold up
    to 4096 masses (< 2^13 in units of 2^-19), the total contrast N^3 - 1 per filled cell.
    Particles outside their tile's window add their weights in FP32 into cells that hold
    up to N^3 masses, so a filled cell carries the rounding of summing M = N^3 terms in FP32:
    |error| <= M eps_32 |cell| = 2e-3 relative (exact for the on-corner point: weights 0, 1)."""
    from oracle import lpt2
    n, box = 32, 64.0
    plan = lib.Plan(W.Instance(n, box, 1, W.COSMO), n_steps=64)
    pos = np.empty((3, n ** 3), dtype=np.float32)
    for c in range(3):
        pos[c] = point[c]
    res = lib.lpt2_cic_pk(plan, pos=torch.from_numpy(pos).cuda(), density=True, n_shells=8)
    want = lpt2.cic_density(n, box, pos.astype(np.float64))
    got = res["density"].cpu().numpy()
    assert np.abs(got - want).max() <= n ** 3 * 6e-8 * np.abs(want).max()
    assert abs(float(res["density"].double().sum())) <= n ** 3 * 6e-8 * n ** 3


def test_particles_far_from_their_tiles(lib):
    """Uniform random positions (not near their lattice cells): most particles take the
    direct-deposit path of the tiled CIC kernel."""
    from oracle import lpt2
    n, box = 64, 128.0
    plan = lib.Plan(W.Instance(n, box, 1, W.COSMO), n_steps=64)
    pos = (np.random.default_rng(9).random((3, n ** 3)) * box).astype(np.float32)
    res = lib.lpt2_cic_pk(plan, pos=torch.from_numpy(pos).cuda(), density=True, n_shells=16)
    want = lpt2.cic_density(n, box, pos.astype(np.float64))
    assert np.abs(res["density"].cpu().numpy() - want).max() <= 2e-5 * max(1.0, np.abs(want).max())
    pk, km, cnt = lpt2.power_spectrum(n, box, want, 16)
    ok = cnt > 0
    np.testing.assert_allclose(res["pk"].cpu().numpy()[ok], pk[ok], rtol=1e-4)


@pytest.mark.parametrize("ns", [1, 256])
def test_extreme_shell_counts(lib, ns):
    from oracle import lpt2
    n, box = 32, 100.0
    plan = lib.Plan(W.Instance(n, box, 1, W.COSMO), n_steps=64)
    pos = W.random_positions(n, box, 3)
    res = lib.lpt2_cic_pk(plan, pos=torch.from_numpy(pos).cuda(), n_shells=ns)
    pk, km, cnt = lpt2.power_spectrum(n, box, lpt2.cic_density(n, box, pos.astype(np.float64)), ns)
    np.testing.assert_array_equal(res["n_modes"].cpu().numpy(), cnt)
    ok = cnt > 0
    np.testing.assert_allclose(res["pk"].cpu().numpy()[ok], pk[ok], rtol=1e-4)
    assert bool((res["pk"].cpu()[~torch.from_numpy(ok)] == 0).all())
