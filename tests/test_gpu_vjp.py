"""GPU adjoint (lpt2_displace_vjp) against the FP64 oracle adjoint and against
central finite differences of the GPU forward map.

Loss: L = sum (delta - delta_t)^2 / N^3 + sum_b (ln P_b - ln P_t,b)^2, the target
from seed 7.  Tolerances: gradient vs FP64 oracle gradient (relative L2 of g_noise,
relative dL/dln|fR0|) 1e-5 for position cotangents, 1e-4 (32^3) / 2e-3 (64^3) for the
full loss; directional central differences of the FP32 forward along a random
unit-variance direction: smooth position loss (step 0.05) within 1e-4, density +
P(k) loss (step 1e-4) within 2e-3 on average over four directions, ln|fR0| (step
1e-2) within 1e-3.

CIC face crossings: the transpose of the CIC deposit is discontinuous at cell
faces (one-sided derivatives differ).  A particle whose FP32 and FP64 positions
(about 1e-5 cell apart) fall on opposite sides of a face takes a different, equally
valid, one-sided derivative; at 64^3 a few of the 786k coordinates do, which moves
the density-term gradient by ~1e-3 in relative L2.  The smooth part of the adjoint
(position cotangents, no CIC) is therefore compared at 1e-5 at every size; the
full loss is compared at 1e-4 at 32^3 and 2e-3 at 64^3.
Per-cell differences are checked on the oracle in FP64 (tests/test_oracle_vjp.py):
in FP32 a single cell moves the loss by ~1e-9 of itself, below FP32 resolution.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
STEPS = 512
NS = 32


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_06282_gb300 import build as B
    B.build()


def lp():
    import paper_1909_06282_gb300 as L
    return L


def gpu_forward(plan, noise):
    L = lp()
    L.lpt2_displace(plan, noise=noise, psi1=False, psi2=False, pos=False)
    r = L.lpt2_cic_pk(plan, pos=None, density=True, n_shells=NS)
    return r["density"], r["pk"]


def gpu_loss(plan, noise, tgt_d, tgt_pk):
    d, pk = gpu_forward(plan, noise)
    d64, pk64 = d.double(), pk
    ok = (pk64 > 0) & (tgt_pk > 0)
    lr = torch.where(ok, torch.log(torch.where(ok, pk64, 1.0)) - torch.log(torch.where(ok, tgt_pk, 1.0)), 0.0)
    return float(((d64 - tgt_d) ** 2).sum() / d.numel() + (lr * lr).sum()), d, pk


@pytest.mark.parametrize("n,box,fr0", [(64, 256.0, 1e-5), (128, 512.0, 1e-4)])
def test_vjp_position_cotangent_against_oracle(n, box, fr0):
    from oracle import growth as gr
    from oracle import vjp as ov
    c = W.COSMO.replace(fr0_abs=fr0)
    tab = gr.growth_tables(c, 1.0, n_steps=STEPS)
    noise = W.white_noise(n, 3)
    st = ov.forward_state(n, box, c, noise.astype(np.float64), tab, NS)
    gpos = W.random_field((3, n ** 3), 17)
    want_w, want_t = ov.vjp(n, box, st, tab, np.zeros((n, n, n)), np.zeros(NS), NS, g_pos=gpos)
    plan = lp().Plan(W.Instance(n, box, 1, c), n_steps=STEPS)
    g_noise, g_t = lp().lpt2_displace_vjp(plan, noise=torch.from_numpy(noise).cuda(),
                                          g_pos=torch.from_numpy(gpos).cuda(), n_shells=NS)
    got = g_noise.cpu().numpy()
    rel = np.linalg.norm(got - want_w) / np.linalg.norm(want_w)
    assert rel < 1e-5, rel
    assert abs(float(g_t) - want_t) <= 1e-5 * abs(want_t), (float(g_t), want_t)


@pytest.mark.parametrize("n,box,fr0,tol", [(32, 128.0, 1e-4, 1e-4), (64, 256.0, 1e-5, 2e-3)])
def test_vjp_against_oracle(n, box, fr0, tol):
    from oracle import growth as gr
    from oracle import philox
    from oracle import vjp as ov
    c = W.COSMO.replace(fr0_abs=fr0)
    tab = gr.growth_tables(c, 1.0, n_steps=STEPS)
    tgt = ov.forward_state(n, box, c, philox.gaussian_noise(n, 7, as_float64=True).reshape(n, n, n), tab, NS)
    noise = W.white_noise(n, 3)
    st = ov.forward_state(n, box, c, noise.astype(np.float64), tab, NS)
    _, gd, gp = ov.loss_and_cotangents(st["density"], st["pk"], tgt["density"], tgt["pk"])
    want_w, want_t = ov.vjp(n, box, st, tab, gd, gp, NS)

    plan = lp().Plan(W.Instance(n, box, 1, c), n_steps=STEPS)
    g_noise, g_t = lp().lpt2_displace_vjp(plan, g_density=torch.from_numpy(gd.astype(np.float32)).cuda(),
                                          g_pk=torch.from_numpy(gp).cuda(),
                                          noise=torch.from_numpy(noise).cuda(), n_shells=NS)
    got = g_noise.cpu().numpy()
    rel = np.linalg.norm(got - want_w) / np.linalg.norm(want_w)
    assert rel < tol, rel
    assert abs(float(g_t) - want_t) <= tol * abs(want_t), (float(g_t), want_t)


def _loss_setup(n, box):
    c = W.COSMO.replace(fr0_abs=1e-5)
    plan = lp().Plan(W.Instance(n, box, 1, c), n_steps=STEPS)
    tplan = lp().Plan(W.Instance(n, box, 7, c), n_steps=STEPS)
    tgt_d, tgt_pk = gpu_forward(tplan, None)
    noise = torch.from_numpy(W.white_noise(n, 3)).cuda()
    return plan, tgt_d.double().clone(), tgt_pk.clone(), noise


def _cotangents(d, pk, tgt_d, tgt_pk):
    ok = (pk > 0) & (tgt_pk > 0)
    gd = (2.0 * (d.double() - tgt_d) / d.numel()).float()
    lr = torch.where(ok, torch.log(torch.where(ok, pk, 1.0)) - torch.log(torch.where(ok, tgt_pk, 1.0)), 0.0)
    gp = torch.where(ok, 2.0 * lr / torch.where(ok, pk, 1.0), 0.0)
    return gd.contiguous(), gp.contiguous()


def test_vjp_directional_fd_smooth_position_loss():
    """L = sum v . (Psi1 + Psi2) is a quadratic polynomial of the noise, so the central
    difference is exact for any step; the step (0.05) is chosen large so that the FP32
    rounding of the forward (about 1e-6 of |Psi| per particle) stays far below the
    difference."""
    n, box = 64, 256.0
    plan, _, _, noise = _loss_setup(n, box)
    v = torch.from_numpy(W.random_field((3, n, n, n), 21)).cuda()

    def L(nz):
        o = lp().lpt2_displace(plan, noise=nz.contiguous(), psi1=True, psi2=True, pos=False)
        return float(((o["psi1"].double() + o["psi2"].double()) * v.double()).sum())

    g_noise, _ = lp().lpt2_displace_vjp(plan, noise=noise, g_pos=v.reshape(3, -1).contiguous(), n_shells=NS)
    d = torch.from_numpy(W.white_noise(n, 11)).cuda()
    h = 0.05
    fd = (L(noise + h * d) - L(noise - h * d)) / (2 * h)
    an = float((g_noise.double() * d.double()).sum())
    assert abs(fd - an) <= 1e-4 * abs(fd), (fd, an)


def test_vjp_directional_fd_density_pk_loss():
    """Density + P(k) loss. CIC is piecewise linear, so the step is kept small (1e-4)
    to limit the cell-face crossings inside the difference.  Particles that cross a
    face within +-h (about 0.2 % of them at this step) still make each central
    difference uncertain at the 1e-3 level, with a sign that varies from direction to
    direction, so the check averages the relative error over four random directions
    (mean <= 2e-3, each <= 5e-3); the smooth loss above checks the same adjoint at
    1e-4 and the oracle comparison checks the CIC transpose itself."""
    n, box = 64, 256.0
    plan, tgt_d, tgt_pk, noise = _loss_setup(n, box)
    L0, d, pk = gpu_loss(plan, noise, tgt_d, tgt_pk)
    gd, gp = _cotangents(d, pk, tgt_d, tgt_pk)
    g_noise, g_t = lp().lpt2_displace_vjp(plan, g_density=gd, g_pk=gp, noise=noise, n_shells=NS)
    h = 1e-4
    errs = []
    for dseed in (11, 12, 13, 14):
        v = torch.from_numpy(W.white_noise(n, dseed)).cuda()
        lp_, _, _ = gpu_loss(plan, (noise + h * v).contiguous(), tgt_d, tgt_pk)
        lm_, _, _ = gpu_loss(plan, (noise - h * v).contiguous(), tgt_d, tgt_pk)
        fd = (lp_ - lm_) / (2 * h)
        an = float((g_noise.double() * v.double()).sum())
        errs.append(abs(fd - an) / abs(fd))
    assert np.mean(errs) <= 2e-3 and max(errs) <= 5e-3, errs
    # d/dln|fR0| by central differences of the GPU forward (tables recomputed).  Step 1e-2:
    # the multiplier tables are FP32, whose rounding (6e-8 of D1) is 1e-3 of the change a
    # 1e-3 step makes; the O(h^2) truncation of a 1e-2 step is ~1e-5.
    hf = 1e-2
    lp().lpt2_set_fr0(plan, 1e-5 * np.exp(hf))
    lpf, _, _ = gpu_loss(plan, noise, tgt_d, tgt_pk)
    lp().lpt2_set_fr0(plan, 1e-5 * np.exp(-hf))
    lmf, _, _ = gpu_loss(plan, noise, tgt_d, tgt_pk)
    fdt = (lpf - lmf) / (2 * hf)
    assert abs(fdt - float(g_t)) <= 1e-3 * abs(fdt), (fdt, float(g_t))


def test_autograd_function_matches_vjp():
    n, box = 32, 128.0
    c = W.COSMO.replace(fr0_abs=1e-5)
    plan = lp().Plan(W.Instance(n, box, 1, c), n_steps=STEPS)
    noise = torch.from_numpy(W.white_noise(n, 4)).cuda().requires_grad_(True)
    logf = torch.tensor(np.log(1e-5), dtype=torch.float64, device="cuda", requires_grad=True)
    d, pk = lp().Displace.apply(noise, logf, plan, NS)
    loss = (d.double() ** 2).sum() / d.numel() + (torch.log(pk[pk > 0]) ** 2).sum()
    loss.backward()
    gd = (2.0 * d.detach().double() / d.numel()).float()
    gp = torch.where(pk > 0, 2.0 * torch.log(torch.where(pk > 0, pk, 1.0)) / torch.where(pk > 0, pk, 1.0), 0.0)
    g_noise, g_t = lp().lpt2_displace_vjp(plan, g_density=gd.contiguous(), g_pk=gp.detach().contiguous(),
                                          noise=noise.detach(), n_shells=NS)
    # same adjoint; only the order of the float atomics of the CIC deposit differs
    rel = float((noise.grad.double() - g_noise.double()).norm() / g_noise.double().norm())
    assert rel < 1e-5, rel
    assert abs(float(logf.grad) - float(g_t)) <= 1e-5 * abs(float(g_t)), (float(logf.grad), float(g_t))
