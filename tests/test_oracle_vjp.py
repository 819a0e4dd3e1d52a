"""Pins of the oracle's hand adjoint: FP64 central finite differences of the loss
L = sum (delta - delta_t)^2 / N^3 + sum_b (ln P_b - ln P_t,b)^2 with respect to
single noise cells and to ln|f_R0|, on a 16^3 grid."""
import numpy as np
import pytest

import workloads as W
from oracle import growth as gr
from oracle import philox
from oracle import vjp as ov

N, BOX, NS = 16, 64.0, 8
STEPS = 256


def loss_of(noise, cosmo, target):
    tab = gr.growth_tables(cosmo, 1.0, n_steps=STEPS)
    st = ov.forward_state(N, BOX, cosmo, noise, tab, NS)
    L, gd, gp = ov.loss_and_cotangents(st["density"], st["pk"], target["density"], target["pk"])
    return L, st, tab, gd, gp


@pytest.fixture(scope="module")
def setup():
    c = W.COSMO.replace(fr0_abs=1e-4)
    tab = gr.growth_tables(c, 1.0, n_steps=STEPS)
    target = ov.forward_state(N, BOX, c, philox.gaussian_noise(N, 7, as_float64=True).reshape(N, N, N),
                              tab, NS)
    noise = philox.gaussian_noise(N, 1, as_float64=True).reshape(N, N, N)
    L, st, tab, gd, gp = loss_of(noise, c, target)
    g_w, g_t = ov.vjp(N, BOX, st, tab, gd, gp, NS)
    return c, target, noise, L, g_w, g_t


def test_vjp_noise_matches_central_differences(setup):
    c, target, noise, L, g_w, _ = setup
    rng = np.random.default_rng(3)
    cells = rng.choice(N ** 3, size=64, replace=False)
    h = 1e-6
    errs = []
    for cidx in cells:
        e = np.zeros(N ** 3)
        e[cidx] = h
        lp = loss_of(noise + e.reshape(N, N, N), c, target)[0]
        lm = loss_of(noise - e.reshape(N, N, N), c, target)[0]
        fd = (lp - lm) / (2 * h)
        errs.append(abs(fd - g_w.ravel()[cidx]) / (np.abs(g_w).max()))
    assert max(errs) < 1e-5, max(errs)


def test_vjp_log_fr0_matches_central_difference(setup):
    c, target, noise, L, _, g_t = setup
    h = 1e-4
    lp = loss_of(noise, c.replace(fr0_abs=c.fr0_abs * np.exp(h)), target)[0]
    lm = loss_of(noise, c.replace(fr0_abs=c.fr0_abs * np.exp(-h)), target)[0]
    fd = (lp - lm) / (2 * h)
    assert abs(fd - g_t) <= 1e-5 * max(abs(fd), 1e-12) + 1e-12, (fd, g_t)
    assert abs(g_t) > 0


def test_vjp_directional_derivative(setup):
    c, target, noise, L, g_w, _ = setup
    v = np.random.default_rng(5).standard_normal(noise.shape)
    h = 1e-6
    lp = loss_of(noise + h * v, c, target)[0]
    lm = loss_of(noise - h * v, c, target)[0]
    fd = (lp - lm) / (2 * h)
    assert abs(fd - np.sum(g_w * v)) < 1e-6 * abs(fd)


def test_vjp_gr_limit_has_no_fr0_gradient():
    c = W.COSMO.replace(fr0_abs=1e-16)
    tab = gr.growth_tables(c, 1.0, n_steps=64)
    noise = philox.gaussian_noise(N, 2, as_float64=True).reshape(N, N, N)
    st = ov.forward_state(N, BOX, c, noise, tab, NS)
    _, gd, gp = ov.loss_and_cotangents(st["density"], st["pk"], np.zeros_like(st["density"]),
                                       np.ones(NS))
    _, g_t = ov.vjp(N, BOX, st, tab, gd, gp, NS)
    assert abs(g_t) < 1e-8


def test_vjp_position_cotangent_matches_central_difference():
    """L = sum_p v_p . Psi_p (a smooth function of the noise): the position cotangent v
    goes straight into the displacement transpose."""
    from oracle import lpt2
    c = W.COSMO.replace(fr0_abs=1e-5)
    tab = gr.growth_tables(c, 1.0, n_steps=STEPS)
    noise = philox.gaussian_noise(N, 4, as_float64=True).reshape(N, N, N)
    v = np.random.default_rng(8).standard_normal((3, N ** 3))

    def L(nz, cc=c):
        t = gr.growth_tables(cc, 1.0, n_steps=STEPS)
        st = ov.forward_state(N, BOX, cc, nz, t, NS)
        return float(np.sum(v * (st["psi1"] + st["psi2"]).reshape(3, -1))), st, t

    _, st, _ = L(noise)
    g_w, g_t = ov.vjp(N, BOX, st, tab, np.zeros((N, N, N)), np.zeros(NS), NS, g_pos=v)
    d = np.random.default_rng(9).standard_normal(noise.shape)
    h = 1e-5
    fd = (L(noise + h * d)[0] - L(noise - h * d)[0]) / (2 * h)
    assert abs(fd - np.sum(g_w * d)) < 1e-7 * abs(fd)
    hf = 1e-4
    fdt = (L(noise, c.replace(fr0_abs=c.fr0_abs * np.exp(hf)))[0]
           - L(noise, c.replace(fr0_abs=c.fr0_abs * np.exp(-hf)))[0]) / (2 * hf)
    assert abs(fdt - g_t) < 1e-5 * abs(fdt), (fdt, g_t)
