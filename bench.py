"""Throughput benchmark of the 2LPT f(R) forward path on GB300.

One step = one full forward pass over one realisation: Philox white noise ->
delta(k) -> the six phi_ij and the source term -> Psi1 + Psi2 (summed in k
space) -> particle positions -> CIC deposit -> 32-shell P(k).  The growth
tables D1(k,a), D2(k,a) depend only on the cosmology and are computed when the
plan is made; their time is reported separately ("growth_ms").

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: every rank makes its own realisation (seed 1 + rank),
no data-path collective (weak scaling); the time is the max over ranks.
--impl reference times the FP64 CPU oracle as it stands on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="fwd_512", n=512, box=1024.0, fr0=1e-5, seed=1, n_shells=32)
SAMPLE_N = 64                      # oracle sample: same cell size (2 Mpc/h), 64^3 grid
SAMPLE_BOX = WORKLOAD["box"] * SAMPLE_N / WORKLOAD["n"]


def workload_desc():
    return (f"{WORKLOAD['n']}^3 grid, {WORKLOAD['n']}^3 particles, L={WORKLOAD['box']:g} Mpc/h, "
            f"|fR0|={WORKLOAD['fr0']:g}, z=0: Philox noise -> 2LPT (T1) positions -> CIC -> "
            f"{WORKLOAD['n_shells']}-shell P(k)")


def workload_config(world):
    """The `config` object of the JSON line; both arms report the same workload."""
    return {"workload": workload_desc(), "grid": WORKLOAD["n"], "box_mpc_h": WORKLOAD["box"],
            "fr0_abs": WORKLOAD["fr0"], "outputs": "positions, CIC density (in workspace), P(k)",
            "l2": "inputs larger than L2 (every field 537 MB > 129 MB L2); no flush",
            "parallelism": f"{world} independent realisation(s), one per GPU"}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_seed(rank):
    """Seed of the realisation a rank runs: one independent realisation per rank."""
    return WORKLOAD["seed"] + rank


def max_over_ranks(dist, values, device):
    """Element-wise maximum over ranks of per-rank timings (ms); identity without a
    process group.  The slowest rank sets the whole job's time."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def whole_job_rate(per_rank, world, ms):
    """Units all ranks processed per second, from the max-over-ranks step time."""
    return per_rank * world / (ms / 1e3)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the kernels
# that can dominate the 512^3 step, from one ncu capture of the 256^3 case of the same
# kernels scaled by the cell count (x 8; the traffic of these passes is proportional to
# N^3, except that at 256^3 a field fits in L2, so the scaled figures are lower bounds).
# Source: profiles/kernels_256.md.  A kernel changed since its capture must be removed here
# (its traffic is then reported as null).
TRAFFIC_512 = {
    "z_source": (402.768896 + 52.556544) * 1e6 * 8,
    "cic": (270.255104 + 45.323008) * 1e6 * 8,
    "y_phi": (201.832704 + 345.711104) * 1e6 * 8,
    "x_delta": (100.722944 + 207.546368) * 1e6 * 8,   # k_x_tma<256, 0, 1> (sqrt(P) field form)
    "x_source": (135.116288 + 84.932864) * 1e6 * 8,
    "z_final": (201.371392 + 152.319744) * 1e6 * 8,
}


def measured_peak_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


ORACLE_SAMPLE_CODE = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import workloads as W
from oracle import growth, lpt2
n, box, reps, seed0 = {n}, {box}, {reps}, {seed0}
c = W.COSMO.replace(fr0_abs={fr0})
tables = growth.growth_tables(c, 1.0, n_steps=1024)
sys.stdout.write("ready\n")
sys.stdout.flush()
sys.stdin.readline()                   # start together with the other processes
t0 = time.perf_counter()
for r in range(reps):
    out = lpt2.run(n, box, c, seed=seed0 + r, tables=tables, n_shells={ns})
dt = time.perf_counter() - t0
print(json.dumps(dict(seconds=dt, particles=reps * n ** 3)))
"""


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_oracle_sample(reps, n=SAMPLE_N, box=SAMPLE_BOX, procs=1):
    """Runs the oracle in `procs` fresh single-threaded processes at once (exec'd, never
    forked from this one), each on `reps` realisations of its own seeds; returns the
    particles of all of them and the wall time from the common start to the last finish."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    ps = []
    for i in range(procs):
        code = ORACLE_SAMPLE_CODE.format(root=ROOT, n=n, box=box, reps=reps, seed0=1 + i * reps,
                                         fr0=WORKLOAD["fr0"], ns=WORKLOAD["n_shells"])
        ps.append(subprocess.Popen([sys.executable, "-c", code], stdin=subprocess.PIPE, stdout=subprocess.PIPE,
                                   stderr=subprocess.PIPE, text=True, env=env))
    for p in ps:                         # every process has its tables: start them together
        if p.stdout.readline().strip() != "ready":
            raise RuntimeError("oracle sample failed: " + p.stderr.read()[-2000:])
    t0 = time.perf_counter()
    for p in ps:
        p.stdin.write("go\n")
        p.stdin.flush()
    results = []
    for p in ps:
        out, err = p.communicate(timeout=1800)
        if p.returncode != 0:
            raise RuntimeError("oracle sample failed: " + err[-2000:])
        results.append(json.loads(out.strip().splitlines()[-1]))
    wall = time.perf_counter() - t0
    return dict(seconds=wall, particles=sum(r["particles"] for r in results), procs=procs)


def bench_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    cores = host_cores()
    per = []
    for i in range(args.warmup + args.steps):
        res = run_oracle_sample(1, procs=cores)   # one realisation per host core, all at once
        if i >= args.warmup:
            per.append(res["seconds"])
    sec = sum(per) / len(per)
    value = cores * SAMPLE_N ** 3 / sec
    line = {
        "impl": "reference", "metric": "particles_per_s", "value": value, "unit": "particles/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": dict(workload_config(world), sample=f"{SAMPLE_N}^3 grid, L={SAMPLE_BOX:g} Mpc/h "
                       f"(same cell size), one realisation per host core ({cores}) per step, growth "
                       "tables precomputed"),
        "cpu_baseline": {"value": value, "unit": "particles/s", "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(),
                         "sample": f"{SAMPLE_N}^3 sub-box at the workload's cell size, one per core per step"},
        "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def profile_run(args):
    """A short run for profilers (`--profile`): plan, args.warmup + args.steps forward steps
    (with --profile-vjp each followed by the adjoint of the density + P(k) loss against
    zero targets), no timing output beyond one line."""
    import torch

    import paper_1909_06282_gb300 as L
    import workloads as W
    n = args.grid
    box = WORKLOAD["box"] * n / WORKLOAD["n"]
    plan = L.Plan(W.Instance(n, box, 1, W.COSMO.replace(fr0_abs=WORKLOAD["fr0"])), n_steps=1024)
    for _ in range(args.warmup + args.steps):
        L.lpt2_displace(plan, psi1=False, psi2=False, pos=True)
        r = L.lpt2_cic_pk(plan, pos=None, density=args.profile_vjp, n_shells=WORKLOAD["n_shells"])
        if args.profile_vjp:
            gd = (2.0 / r["density"].numel()) * r["density"]
            L.lpt2_displace_vjp(plan, g_density=gd.contiguous(), g_pk=(1.0 / r["pk"].clamp_min(1e-30)).contiguous(),
                                n_shells=WORKLOAD["n_shells"])
    torch.cuda.synchronize()
    print(json.dumps({"profile_run": True, "grid": n, "box": box, "launches": L.lpt2_launch_count(plan)}))


def source_table(args):
    """The full-source diagnostic over output times and |fR0| (`--source-table`): for
    z = 0, 0.5, 1 and |fR0| = 1e-4, 1e-5, 1e-6 on one realisation (seed 1, the grid of
    --grid at a 2 Mpc/h cell), the shell mean and scatter of Re(S_MG/S_GR) and the T1
    ratio at each shell's mean |k|.  Prints one JSON line per (z, |fR0|)."""
    import torch

    import paper_1909_06282_gb300 as L
    import workloads as W
    n = args.grid
    box = WORKLOAD["box"] * n / WORKLOAD["n"]
    for z in (0.0, 0.5, 1.0):
        a = 1.0 / (1.0 + z)
        plan = L.Plan(W.Instance(n, box, 1, W.COSMO.replace(fr0_abs=1e-5), a_out=a), n_steps=1024)
        for fr0 in (1e-4, 1e-5, 1e-6):
            L.lpt2_set_fr0(plan, fr0)
            t0 = time.perf_counter()
            r = L.lpt2_source_ratio(plan, n_bins=WORKLOAD["n_shells"])
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3
            L.lpt2_device_status(plan)
            print(json.dumps({"source_table": True, "grid": n, "box": box, "z": z, "fr0": fr0, "ms": ms,
                              **{k: v.cpu().tolist() for k, v in r.items()}}), flush=True)
        del plan
        torch.cuda.empty_cache()


def bench_large(args, L, W, torch):
    """The large configuration: 1024^3 particles, L = 2048 Mpc/h (the same 2 Mpc/h cell),
    |fR0| = 1e-5, forward step (positions, CIC, 32-shell P(k)) on its own plan and stream."""
    n = 1024
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        plan = L.Plan(W.Instance(n, 2048.0, 1, W.COSMO.replace(fr0_abs=1e-5)), n_steps=1024, stream=st)
        pos = torch.empty((3, n, n, n), dtype=torch.float32, device="cuda")

        def step():
            L.lpt2_displace(plan, psi1=False, psi2=False, pos=pos)
            return L.lpt2_cic_pk(plan, pos=None, n_shells=WORKLOAD["n_shells"])

        for _ in range(2):
            step()
        st.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = 3
        e0.record(st)
        for _ in range(k):
            step()
        e1.record(st)
        st.synchronize()
        ms = e0.elapsed_time(e1) / k
    del plan, pos
    torch.cuda.empty_cache()
    return {"particles_per_step": n ** 3, "ms_per_step": ms, "value": n ** 3 / (ms / 1e3), "unit": "particles/s",
            "what": "1024^3, L = 2048 Mpc/h, |fR0| = 1e-5: positions + CIC + 32-shell P(k), 3 timed steps"}


def bench_batched(args, L, W, torch, stream):
    """96 instances (32 each of 96^3/384, 128^3/512, 192^3/768 Mpc/h; seeds 1..96; |fR0|
    log-uniform in [1e-6, 1e-4]): one graph-captured batched plan vs the same instances
    through single-instance plans one after the other.  Step = positions + CIC + P(k)."""
    insts = W.batched_96()
    parts = sum(i.n ** 3 for i in insts)
    with torch.cuda.stream(stream):
        plan = L.Plan(insts, n_steps=1024, stream=stream, graph=True)
        pos = torch.empty(3 * plan.cells, dtype=torch.float32, device="cuda")

        def bstep():
            L.lpt2_displace(plan, psi1=False, psi2=False, pos=pos)
            L.lpt2_cic_pk(plan, pos=None, n_shells=WORKLOAD["n_shells"])

        # instances per launch of each grid-size group, tuned on this GPU (whole groups first)
        for _ in range(args.warmup):
            bstep()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(max(1, args.steps // 2)):
            bstep()
        e1.record(stream)
        stream.synchronize()
        ms_whole = e0.elapsed_time(e1) / max(1, args.steps // 2)
        schedule = L.lpt2_autotune(plan, n_shells=WORKLOAD["n_shells"], reps=3)
        ytile, xtile = L.lpt2_tiles(plan)

        singles = [L.Plan(i, n_steps=1024, stream=stream) for i in insts]
        spos = [torch.empty((3, i.n, i.n, i.n), dtype=torch.float32, device="cuda") for i in insts]

        def sstep():
            for pl, ps in zip(singles, spos):
                L.lpt2_displace(pl, psi1=False, psi2=False, pos=ps)
                L.lpt2_cic_pk(pl, pos=None, n_shells=WORKLOAD["n_shells"])

        def sstep_tuned():   # the single plans with their group's autotuned tile choices
            if not getattr(sstep_tuned, "set", False):
                sizes = sorted({i.n for i in insts}, key=[i.n for i in insts].index)
                for pl, it in zip(singles, insts):
                    gi = sizes.index(it.n)
                    L.lpt2_set_tiles(pl, [ytile[gi]], [xtile[gi]])
                sstep_tuned.set = True
            sstep()

        res = {}
        for name, fn in (("batched", bstep), ("one_by_one", sstep), ("one_by_one_tuned_tiles", sstep_tuned)):
            for _ in range(args.warmup):
                fn()
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            k = max(1, args.steps // 2)
            e0.record(stream)
            for _ in range(k):
                fn()
            e1.record(stream)
            stream.synchronize()
            res[name] = e0.elapsed_time(e1) / k
        del singles, spos, plan, pos
    return {"instances": len(insts), "particles_per_step": parts,
            "value": parts / (res["batched"] / 1e3), "unit": "particles/s",
            "instances_per_s": len(insts) / (res["batched"] / 1e3),
            "ms_per_step": res["batched"],
            "one_by_one": {"value": parts / (res["one_by_one"] / 1e3), "ms_per_step": res["one_by_one"]},
            "speedup_vs_one_by_one": res["one_by_one"] / res["batched"],
            "one_by_one_tuned_tiles": {"ms_per_step": res["one_by_one_tuned_tiles"],
                                       "speedup": res["one_by_one_tuned_tiles"] / res["batched"]},
            "schedule": {"groups": ["96^3", "128^3", "192^3"], "instances_per_launch": schedule,
                         "y_pencils_per_cta": ytile, "x_tile_path": xtile,
                         "whole_group_ms_per_step": ms_whole},
            "what": "96 instances (32 x 96^3/384, 128^3/512, 192^3/768 Mpc/h), positions + CIC + P(k), "
                    "one CUDA graph with the autotuned launch schedule vs single-instance plans one by one"}


def cufft_pipeline(plan, L, torch, n, box, n_shells):
    """The same forward path with cuFFT (torch.fft) for every transform and unfused torch
    element-wise kernels for the k-space multipliers, source term, CIC (scatter-add) and
    P(k) (bincount); only the white noise and the growth tables come from the library.
    A timed comparison, not a product path."""
    import numpy as np
    f32 = torch.float32
    dev = "cuda"
    d1t, d2t, _, _ = L.lpt2_growth_tables(plan)
    kt = torch.logspace(-4, 1, plan.n_k, dtype=torch.float64, device=dev)
    c = plan.inst.cosmo
    kf = 2 * np.pi / box
    m = torch.fft.fftfreq(n, d=1.0 / n, device=dev).to(f32)
    mz = torch.arange(n // 2 + 1, device=dev, dtype=f32)
    kx, ky, kz = (kf * m)[:, None, None], (kf * m)[None, :, None], (kf * mz)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    zero = (k2 == 0) | (m.abs() == n // 2)[:, None, None] | (m.abs() == n // 2)[None, :, None] \
        | (mz == n // 2)[None, None, :]
    kk = torch.sqrt(k2).clamp_min(1e-30)
    lk = torch.log(kk.double())
    lt = torch.log(kt)
    idx = torch.clamp(torch.searchsorted(lt, lk) - 1, 0, plan.n_k - 2)
    fr = ((lk - lt[idx]) / (lt[idx + 1] - lt[idx])).clamp(0, 1)
    D1 = (d1t[idx] + fr * (d1t[idx + 1] - d1t[idx])).to(f32)
    D2 = (d2t[idx] + fr * (d2t[idx + 1] - d2t[idx])).to(f32)
    # sqrt(P(k) N^3 / V): Eisenstein-Hu no-wiggle fit, amplitude from sigma_8 (Simpson in ln k)
    h, wm, wb = c.h, c.omega_m * c.h ** 2, c.omega_b * c.h ** 2
    fb, th = c.omega_b / c.omega_m, c.t_cmb / 2.7
    ssnd = 44.5 * np.log(9.83 / wm) / np.sqrt(1 + 10 * wb ** 0.75)
    alpha = 1 - 0.328 * np.log(431 * wm) * fb + 0.38 * np.log(22.3 * wm) * fb * fb

    def transfer(kx_):
        gam = c.omega_m * h * (alpha + (1 - alpha) / (1 + (0.43 * kx_ * h * ssnd) ** 4))
        q = kx_ * th * th / gam
        l0 = np.log(2 * np.e + 1.8 * q) if isinstance(q, np.ndarray) else torch.log(2 * np.e + 1.8 * q)
        return l0 / (l0 + (14.2 + 731 / (1 + 62.5 * q)) * q * q)

    lk_ = np.linspace(np.log(1e-5), np.log(1e3), 20001)
    k_ = np.exp(lk_)
    x_ = 8 * k_
    f_ = k_ ** (3 + c.n_s) * transfer(k_) ** 2 * (3 * (np.sin(x_) - x_ * np.cos(x_)) / x_ ** 3) ** 2 / (2 * np.pi ** 2)
    wts = np.ones_like(f_)
    wts[1:-1:2], wts[2:-1:2] = 4, 2
    amp = c.sigma8 ** 2 / ((lk_[1] - lk_[0]) / 3 * np.dot(wts, f_))
    T = transfer(kk)
    sk = torch.where(zero, 0.0, np.sqrt(amp) * kk ** (c.n_s / 2) * T * np.sqrt(n ** 3 / box ** 3))
    inv = torch.where(zero, 0.0, 1.0 / k2)
    kv = (kx, ky, kz)
    qg = [torch.arange(n, device=dev, dtype=f32).view(s_) * (box / n)
          for s_ in ((n, 1, 1), (1, n, 1), (1, 1, n))]
    noise = L.lpt2_white_noise(plan)

    def run():
        dk = torch.fft.rfftn(noise) * sk
        pot = dk * inv
        names = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
        ph = {nm: torch.fft.irfftn(-kv[nm[0]] * kv[nm[1]] * pot, s=(n, n, n)) for nm in names}
        S = (ph[(0, 0)] * ph[(1, 1)] + ph[(0, 0)] * ph[(2, 2)] + ph[(1, 1)] * ph[(2, 2)]
             - ph[(0, 1)] ** 2 - ph[(0, 2)] ** 2 - ph[(1, 2)] ** 2)
        del ph
        u = (D1 * dk - D2 * torch.fft.rfftn(S) * torch.where(zero, 0.0, 1.0)) * inv
        rho = torch.zeros(n ** 3, dtype=f32, device=dev)
        uc = [torch.remainder(qg[c_] + torch.fft.irfftn(1j * kv[c_] * u, s=(n, n, n)), box) * (n / box)
              for c_ in range(3)]
        fl = [torch.floor(x) for x in uc]
        d = [x - f for x, f in zip(uc, fl)]
        i0 = [f.long() % n for f in fl]
        for ox in (0, 1):
            for oy in (0, 1):
                for oz in (0, 1):
                    w = (d[0] if ox else 1 - d[0]) * (d[1] if oy else 1 - d[1]) * (d[2] if oz else 1 - d[2])
                    cell = (((i0[0] + ox) % n) * n + (i0[1] + oy) % n) * n + (i0[2] + oz) % n
                    rho.index_add_(0, cell.reshape(-1), w.reshape(-1))
        dr = torch.fft.rfftn((rho - 1).view(n, n, n))
        pw = (dr.real ** 2 + dr.imag ** 2) * (box ** 3 / float(n) ** 6)
        nn = (k2 / (kf * kf)).round().long()
        ok = (nn > 0) & (4 * nn < n * n) & (mz < n // 2)[None, None, :]
        b = torch.floor(torch.sqrt(nn.double()) * (2 * n_shells / n)).long().clamp(0, n_shells - 1)
        wgt = torch.where(mz == 0, 1.0, 2.0)[None, None, :].expand_as(pw)
        sel = ok.reshape(-1)
        bb = b.reshape(-1)[sel]
        cnt = torch.bincount(bb, weights=wgt.reshape(-1)[sel].double(), minlength=n_shells)
        ps = torch.bincount(bb, weights=(pw * wgt).reshape(-1)[sel].double(), minlength=n_shells)
        return ps / cnt.clamp_min(1)

    return run


def bench_ours(args):
    import numpy as np
    import torch

    import paper_1909_06282_gb300 as L
    import workloads as W

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    n, box = WORKLOAD["n"], WORKLOAD["box"]
    inst = W.Instance(n, box, rank_seed(rank), W.COSMO.replace(fr0_abs=WORKLOAD["fr0"]))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        plan = L.Plan(inst, n_steps=1024, stream=stream, host_io=True, max_outputs=3, keep_state=True)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        L.lpt2_growth_tables(plan)
        g1.record(stream)
        stream.synchronize()
        growth_ms = g0.elapsed_time(g1)

        pos = torch.empty((3, n, n, n), dtype=torch.float32, device="cuda")
        pk = dict(pk=torch.empty(32, dtype=torch.float64, device="cuda"))

        def step():
            L.lpt2_displace(plan, psi1=False, psi2=False, pos=pos)
            return L.lpt2_cic_pk(plan, pos=None, n_shells=WORKLOAD["n_shells"])

        for _ in range(args.warmup):
            step()
        stream.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0 = L.lpt2_launch_count(plan)
        with ClockSampler(local) as clk:
            e0.record(stream)
            for _ in range(args.steps):
                res = step()
            e1.record(stream)
            stream.synchronize()
        launches = L.lpt2_launch_count(plan) - c0
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        # the per-kernel split (CUDA events around every launch) comes from a second run of
        # the same steps, so that the headline above is timed without that instrumentation
        L.lpt2_timing(plan, True)
        for _ in range(args.steps):
            step()
        kstats = L.lpt2_timing_report(plan)
        L.lpt2_timing(plan, False)
        torch.cuda.synchronize()

        # forward + adjoint (loss: mean squared density difference to the seed-7 field
        # plus the squared log P(k) ratio; cotangents formed by torch on the device)
        tinst = W.Instance(n, box, 7, inst.cosmo)
        tplan = L.Plan(tinst, n_steps=1024, stream=stream)
        L.lpt2_displace(tplan, psi1=False, psi2=False, pos=False)
        tr = L.lpt2_cic_pk(tplan, pos=None, density=True, n_shells=WORKLOAD["n_shells"])
        tgt_d, tgt_pk = tr["density"].clone(), tr["pk"].clone()
        del tplan, tr

        def fwd_vjp_step():
            L.lpt2_displace(plan, psi1=False, psi2=False, pos=False)
            r = L.lpt2_cic_pk(plan, pos=None, density=True, n_shells=WORKLOAD["n_shells"])
            d, pkv = r["density"], r["pk"]
            ok = (pkv > 0) & (tgt_pk > 0)
            lr = torch.where(ok, torch.log(torch.where(ok, pkv, 1.0) / torch.where(ok, tgt_pk, 1.0)), 0.0)
            gd = (2.0 / d.numel()) * (d - tgt_d)
            gp = torch.where(ok, 2.0 * lr / torch.where(ok, pkv, 1.0), 0.0)
            L.lpt2_displace_vjp(plan, g_density=gd, g_pk=gp, n_shells=WORKLOAD["n_shells"])

        for _ in range(args.warmup):
            fwd_vjp_step()
        stream.synchronize()
        e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        vsteps = max(1, args.steps // 2)
        e4.record(stream)
        for _ in range(vsteps):
            fwd_vjp_step()
        e5.record(stream)
        stream.synchronize()
        ms_fv = e4.elapsed_time(e5) / vsteps

        # several output times from one realisation: z = 1, 0.5, 0 with the a-independent
        # prefix (noise -> delta(k) -> phi_ij -> S) once, against three forward steps
        multi = None
        if not args.no_multi_a:
            a_list = [0.5, 2.0 / 3.0, 1.0]
            L.lpt2_set_outputs(plan, a_list)
            pos_m = torch.empty((len(a_list), 3, n, n, n), dtype=torch.float32, device="cuda")
            for _ in range(args.warmup):
                L.lpt2_displace_outputs(plan, pos=pos_m, n_shells=WORKLOAD["n_shells"])
            stream.synchronize()
            e8, e9 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            msteps = max(1, args.steps // 2)
            e8.record(stream)
            for _ in range(msteps):
                L.lpt2_displace_outputs(plan, pos=pos_m, n_shells=WORKLOAD["n_shells"])
            e9.record(stream)
            stream.synchronize()
            ms_m = e8.elapsed_time(e9) / msteps
            multi = {"a_out": a_list, "ms_per_call": ms_m, "ms_per_output": ms_m / len(a_list),
                     "particles_per_s": len(a_list) * n ** 3 / (ms_m / 1e3),
                     "vs_separate_steps": len(a_list) * ms / ms_m,
                     "what": "lpt2_displace_outputs: positions + 32-shell P(k) at each a; the noise -> "
                             "delta(k) -> phi_ij -> S(k) prefix runs once per call"}
            del pos_m

        # full second-order source term / GR diagnostic (Sec. 3), same plan and noise
        src = None
        if not args.no_source:
            L.lpt2_source_ratio(plan, n_bins=WORKLOAD["n_shells"])
            stream.synchronize()
            L.lpt2_timing(plan, True)
            e8, e9 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e8.record(stream)
            for _ in range(2):
                sr = L.lpt2_source_ratio(plan, n_bins=WORKLOAD["n_shells"])
            e9.record(stream)
            stream.synchronize()
            srep = L.lpt2_timing_report(plan)
            L.lpt2_timing(plan, False)
            ms_src = e8.elapsed_time(e9) / 2
            sbytes = sum(v["bytes"] for v in srep.values()) / 2
            sms = sum(v["total_ms"] for v in srep.values()) / 2
            src = {"ms_per_call": ms_src, "algorithmic_gb_per_call": sbytes / 1e9,
                   "achieved_gbs": sbytes / (sms / 1e3) / 1e9,
                   "launches_per_call": sum(v["launches"] for v in srep.values()) // 2,
                   "ratio_last_shells": [round(x, 4) for x in sr["mean"].cpu().tolist()[-4:]],
                   "t1_last_shells": [round(x, 4) for x in sr["t1"].cpu().tolist()[-4:]],
                   "what": "lpt2_source_ratio: full S1+S2+S3+S4 and S_GR (31 inverse + 5 forward 3-D "
                           "transforms), per-mode ratio binned in 32 shells, T1 curve"}

        batched = bench_batched(args, L, W, torch, stream) if not args.no_batched else None
        large = bench_large(args, L, W, torch) if not args.no_large else None

        # the same path with cuFFT transforms and unfused element-wise kernels
        cuf = None
        if not args.no_cufft:
            run = cufft_pipeline(plan, L, torch, n, box, WORKLOAD["n_shells"])
            for _ in range(2):
                pk_c = run()
            stream.synchronize()
            e6, e7 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            kc = max(1, args.steps // 4)
            e6.record(stream)
            for _ in range(kc):
                pk_c = run()
            e7.record(stream)
            stream.synchronize()
            ms_c = e6.elapsed_time(e7) / kc
            L.lpt2_displace(plan, psi1=False, psi2=False, pos=pos)
            pk_o = L.lpt2_cic_pk(plan, pos=None, n_shells=WORKLOAD["n_shells"])["pk"]
            okm = pk_o > 0
            cuf = {"value": n ** 3 / (ms_c / 1e3), "unit": "particles/s", "ms_per_step": ms_c,
                   "ours_over_cufft": ms_c / ms,
                   "pk_max_rel_diff": float(((pk_c - pk_o).abs() / pk_o.clamp_min(1e-300))[okm].max()),
                   "what": "same forward path, torch.fft (cuFFT) transforms + unfused torch element-wise "
                           "kernels, scatter-add CIC, bincount P(k)"}
            del run

        # end to end through the C ABI with host buffers: lpt2_displace_host takes pinned
        # host noise and returns positions + P(k) in pinned host memory; inside, the
        # upload of realisation i+1 and the download of i-1 overlap i's kernels (two
        # device buffer sets, two copy streams).  Every copy of every step is inside the
        # timed region, host wall clock around the call, which returns when the last
        # result is in host memory.
        noise_h = torch.from_numpy(W.white_noise(n, 1000 + rank)).pin_memory()
        pos_h = torch.empty((3, n, n, n), dtype=torch.float32).pin_memory()
        pk_h = torch.empty((max(args.steps, args.warmup, 1), WORKLOAD["n_shells"]), dtype=torch.float64).pin_memory()

        def e2e_run(k):
            L.lpt2_displace_host(plan, k, noise=noise_h, pos=pos_h, pk=pk_h[:k], n_shells=WORKLOAD["n_shells"])

        e2e_run(max(1, args.warmup))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_run(args.steps)
        ms_e2e = (time.perf_counter() - t0) * 1e3 / args.steps
        torch.cuda.synchronize()

    ms, ms_e2e, ms_fv = max_over_ranks(dist, [ms, ms_e2e, ms_fv], "cuda")

    if rank == 0:
        parts = n ** 3 * world
        value = whole_job_rate(n ** 3, world, ms)
        peak, peak_kind = measured_peak_gbs()
        total_ms = sum(v["total_ms"] for v in kstats.values())
        dom = max(kstats.items(), key=lambda kv: kv[1]["total_ms"])
        dname, dv = dom
        achieved = dv["bytes"] / (dv["total_ms"] / 1e3) / 1e9
        kernels = {k: {"launches": v["launches"], "ms_per_launch": v["total_ms"] / v["launches"],
                       "share": v["total_ms"] / total_ms,
                       "gbs": (v["bytes"] / (v["total_ms"] / 1e3) / 1e9) if v["bytes"] else None}
                   for k, v in sorted(kstats.items(), key=lambda kv: -kv[1]["total_ms"])}
        all_bytes = sum(v["bytes"] for v in kstats.values())
        line = {
            "metric": "particles_per_s", "value": value, "unit": "particles/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(world),
            "roofline": {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": peak,
                         "peak_kind": f"hbm_gbs of {peak_kind}", "unit": "GB/s", "frac": achieved / peak,
                         "traffic": TRAFFIC_512.get(dname) if n == 512 else None,
                         "algorithmic_bytes": dv["bytes"] / dv["launches"]},
            "path_roofline": {"algorithmic_gb_per_step": all_bytes / args.steps / 1e9,
                              "achieved_gbs": all_bytes / (total_ms / 1e3) / 1e9,
                              "frac": all_bytes / (total_ms / 1e3) / 1e9 / peak},
            "kernels": kernels,
            "growth_ms": growth_ms,
            "batched": batched,
            "cufft_pipeline": cuf,
            "source_diagnostic": src,
            "multi_a": multi,
            "large_1024": large,
            "fwd_vjp": {"value": parts / (ms_fv / 1e3), "unit": "particles/s", "ms_per_step": ms_fv,
                        "vjp_over_fwd": (ms_fv - ms) / ms,
                        "what": "forward + loss cotangents + lpt2_displace_vjp (noise and ln|fR0| gradients)"},
            "gpu_launches": launches,
            "e2e": {"value": parts / (ms_e2e / 1e3), "unit": "particles/s",
                    "h2d_bytes_per_step": n ** 3 * 4, "d2h_bytes_per_step": 3 * n ** 3 * 4 + 32 * 8},
            "clocks": clk.summary(),
        }
        if not args.no_cpu_baseline:
            # the oracle on every host core (one process per core, independent realisations)
            # and on one core, 64^3 samples at the workload's cell size
            reps, cores = 3, host_cores()
            res = run_oracle_sample(reps, procs=cores)
            one = run_oracle_sample(reps)
            line["cpu_baseline"] = {
                "value": res["particles"] / res["seconds"], "unit": "particles/s", "cores": cores,
                "kind": "oracle", "cpu_model": cpu_model(),
                "sample": f"{reps} realisations of a {SAMPLE_N}^3 grid at the workload's cell size "
                          f"(L={SAMPLE_BOX:g} Mpc/h) per core, {cores} single-threaded processes at once, "
                          f"growth tables precomputed, {res['seconds']:.1f} s",
                "one_core": {"value": one["particles"] / one["seconds"], "unit": "particles/s",
                             "sample": f"{reps} realisations of {SAMPLE_N}^3, {one['seconds']:.1f} s"}}
            if args.oracle_256:
                n2, b2 = 256, WORKLOAD["box"] * 256 / WORKLOAD["n"]
                r1 = run_oracle_sample(1, n=n2, box=b2)
                ra = run_oracle_sample(1, n=n2, box=b2, procs=cores)
                line["cpu_baseline"]["at_256"] = {
                    "one_core": r1["particles"] / r1["seconds"], "all_cores": ra["particles"] / ra["seconds"],
                    "unit": "particles/s",
                    "sample": f"one 256^3 realisation (L={b2:g} Mpc/h) on one core ({r1['seconds']:.0f} s) "
                              f"and one per core on {cores} cores ({ra['seconds']:.0f} s)"}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-256", action="store_true",
                    help="also time the oracle on a 256^3 realisation, on one core and on every core "
                         "(minutes of CPU time)")
    ap.add_argument("--no-batched", action="store_true", help="skip the 96-instance batched measurement")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT comparison pipeline")
    ap.add_argument("--no-source", action="store_true", help="skip the full-source diagnostic timing")
    ap.add_argument("--no-large", action="store_true", help="skip the 1024^3 forward timing")
    ap.add_argument("--no-multi-a", action="store_true", help="skip the several-output-times timing")
    ap.add_argument("--profile-vjp", action="store_true", help="with --profile: run the adjoint after each step")
    ap.add_argument("--profile", action="store_true",
                    help="forward-only run for ncu (no timing); grid from --grid")
    ap.add_argument("--grid", type=int, default=WORKLOAD["n"],
                    help="grid side for --profile (cell size kept at 2 Mpc/h)")
    ap.add_argument("--source-table", action="store_true",
                    help="full-source diagnostic at z = 0, 0.5, 1 and |fR0| = 1e-4, 1e-5, 1e-6 (grid from "
                         "--grid); prints one JSON line per case instead of the benchmark line")
    args = ap.parse_args()
    if args.profile:
        profile_run(args)
        return
    if args.source_table:
        source_table(args)
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
