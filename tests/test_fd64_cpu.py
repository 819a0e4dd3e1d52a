"""Pins of the float64 finite-difference forward map (tests/fd64.py) on the CPU: it must
reproduce the oracle's forward state (positions, CIC density, shell P(k), loss) and, with
the deposit cells frozen at the central point, central differences of its loss must equal
the oracle's hand adjoint cell by cell."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("n,box,fr0", [(16, 64.0, 1e-4), (32, 128.0, 1e-5)])
def test_fd64_forward_and_differences_match_the_oracle(n, box, fr0):
    from fd64 import Forward64
    from oracle import growth as gr
    from oracle import philox
    from oracle import vjp as ov
    ns = 16
    c = W.COSMO.replace(fr0_abs=fr0)
    tab = gr.growth_tables(c, 1.0, n_steps=128)
    noise = W.white_noise(n, 3).astype(np.float64)
    tn = philox.gaussian_noise(n, 7, as_float64=True).reshape(n, n, n)
    st = ov.forward_state(n, box, c, noise, tab, ns)
    tg = ov.forward_state(n, box, c, tn, tab, ns)
    F = Forward64(n, box, c, tab, ns, device="cpu")
    u = F.lattice_coords(torch.from_numpy(noise))
    d = torch.remainder(u * (box / n), box).numpy() - st["pos"]
    d -= box * np.round(d / box)
    assert np.abs(d).max() < 1e-10 * box
    dens = F.density(u)
    assert np.abs(dens.numpy() - st["density"]).max() < 1e-10
    pk = F.power(dens)
    ok = st["pk"] > 0
    np.testing.assert_allclose(pk.numpy()[ok], st["pk"][ok], rtol=1e-10)
    dt = F.density(F.lattice_coords(torch.from_numpy(tn)))
    pt = F.power(dt)
    L = F.loss(dens, pk, dt, pt)
    Lo, gd, gp = ov.loss_and_cotangents(st["density"], st["pk"], tg["density"], tg["pk"])
    assert abs(L - Lo) <= 1e-12 * abs(Lo)
    gw, _ = ov.vjp(n, box, st, tab, gd, gp, ns)
    base = torch.floor(u).long()
    h = 1e-3
    cells = np.random.default_rng(n).choice(n ** 3, 6, replace=False)
    for cidx in cells:
        ls = []
        for sgn in (1.0, -1.0):
            e = np.zeros(n ** 3)
            e[cidx] = sgn * h
            dp = F.density(F.lattice_coords(torch.from_numpy(noise + e.reshape(n, n, n))), base)
            ls.append(F.loss(dp, F.power(dp), dt, pt))
        fd = (ls[0] - ls[1]) / (2 * h)
        assert abs(fd - gw.ravel()[cidx]) <= 1e-6 * np.abs(gw).max(), (cidx, fd, gw.ravel()[cidx])


def test_fd64_density_cotangent_and_cic_transpose():
    """The density-space cotangent against central differences of the loss in the density
    (one cell at a time), and the CIC transpose against the oracle's."""
    from fd64 import Forward64
    from oracle import growth as gr
    from oracle import vjp as ov
    n, box, ns = 16, 64.0, 8
    c = W.COSMO.replace(fr0_abs=1e-5)
    tab = gr.growth_tables(c, 1.0, n_steps=64)
    F = Forward64(n, box, c, tab, ns, device="cpu")
    rng = np.random.default_rng(5)
    dens = torch.from_numpy(rng.normal(0, 0.5, (n, n, n)))
    dt = torch.from_numpy(rng.normal(0, 0.5, (n, n, n)))
    pt = F.power(dt)
    gd, gp = F.cotangents(dens, F.power(dens), dt, pt)
    g = F.density_cotangent(dens, gd, gp).numpy()
    h = 1e-6
    for cidx in rng.choice(n ** 3, 5, replace=False):
        ls = []
        for sgn in (1.0, -1.0):
            dd = dens.clone().reshape(-1)
            dd[cidx] += sgn * h
            dd = dd.reshape(n, n, n)
            ls.append(F.loss(dd, F.power(dd), dt, pt))
        fd = (ls[0] - ls[1]) / (2 * h)
        assert abs(fd - g.ravel()[cidx]) <= 1e-7 * np.abs(g).max(), (fd, g.ravel()[cidx])
    pos = W.random_positions(n, box, 9).astype(np.float64)
    u = torch.from_numpy(pos * (n / box))
    got = F.cic_transpose(u, torch.floor(u).long(), torch.from_numpy(g)).numpy()
    want = ov._cic_transpose(n, box, pos, g)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
