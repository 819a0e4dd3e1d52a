"""ctypes marshalling for liblpt2.so (the C ABI of include/lpt2.h).

Tensors are PyTorch CUDA tensors; their data pointers and the current CUDA
stream are handed to the library.  Nothing here computes any part of the method.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
HEADER = os.path.join(ROOT, "include", "lpt2.h")

_ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EUNSUPPORTED", -5: "ETIMEOUT",
           -6: "ENOWORKSPACE"}


def _header_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lpt2_[a-z0-9_]+)\s*\(", txt)))


HEADER_FUNCTIONS = _header_functions()


class LPT2Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lpt2 error {code} ({_ERRORS.get(code, '?')}): {msg}")
        self.code = code


class _Cosmo(C.Structure):
    _fields_ = [("omega_m", C.c_double), ("omega_l", C.c_double), ("omega_b", C.c_double),
                ("h", C.c_double), ("n_s", C.c_double), ("sigma8", C.c_double),
                ("t_cmb", C.c_double), ("fr0_abs", C.c_double), ("hs_n", C.c_int),
                ("a_init", C.c_double), ("d2_variant", C.c_int)]


class _Instance(C.Structure):
    _fields_ = [("n", C.c_int), ("box", C.c_double), ("seed", C.c_uint64), ("a_out", C.c_double),
                ("cosmo", _Cosmo)]


class _KernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("total_ms", C.c_double),
                ("bytes", C.c_double)]


_lib = None


def library_path() -> str:
    """lib/liblpt2.so next to this file, or the file named by LPT2_LIBRARY."""
    return os.environ.get("LPT2_LIBRARY") or os.path.join(HERE, "lib", "liblpt2.so")


def load_library():
    """Loads liblpt2.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "or python paper_1909_06282_gb300/build.py")
    lib = C.CDLL(path)
    vp, i, d, u64, i64 = C.c_void_p, C.c_int, C.c_double, C.c_uint64, C.c_int64
    sig = {
        "lpt2_plan": (i, [C.POINTER(vp), C.POINTER(_Instance), i, i, d, d, i, vp, C.c_uint]),
        "lpt2_plan_destroy": (i, [vp]),
        "lpt2_workspace_size": (i, [vp, C.POINTER(C.c_size_t)]),
        "lpt2_workspace_bytes": (i, [C.POINTER(_Instance), i, i, C.c_uint, C.POINTER(C.c_size_t)]),
        "lpt2_debug_alloc_hook": (i, [i, C.POINTER(i64)]),
        "lpt2_set_wait_budget": (i, [vp, i64]),
        "lpt2_set_workspace": (i, [vp, vp, C.c_size_t]),
        "lpt2_growth_tables": (i, [vp, vp, vp, vp, vp]),
        "lpt2_white_noise": (i, [vp, vp]),
        "lpt2_philox_words": (i, [u64, u64, i64, vp, vp]),
        "lpt2_box_muller": (i, [vp, vp, i64, vp]),
        "lpt2_displace": (i, [vp, vp, vp, vp, vp, vp]),
        "lpt2_cic_pk": (i, [vp, vp, vp, vp, vp, vp, i]),
        "lpt2_fft_r2c": (i, [vp, vp, vp]),
        "lpt2_fft_c2r": (i, [vp, vp, vp]),
        "lpt2_last_error": (C.c_char_p, []),
        "lpt2_launch_count": (i64, [vp]),
        "lpt2_device_status": (i, [vp]),
        "lpt2_source_ratio": (i, [vp, vp, i, vp, vp, vp, vp, vp, vp, vp]),
        "lpt2_cic_pk_est": (i, [vp, vp, vp, vp, vp, vp, i, C.c_uint]),
        "lpt2_timing": (i, [vp, i]),
        "lpt2_cic_pk_noalloc": (i, [i, d, vp, vp, vp, vp, vp, i, vp]),
        "lpt2_set_fr0": (i, [vp, d]),
        "lpt2_displace_vjp": (i, [vp, vp, vp, vp, vp, i, vp, vp]),
        "lpt2_displace_host": (i, [vp, i, vp, i64, vp, i64, vp, i64, i]),
        "lpt2_set_outputs": (i, [vp, i, C.POINTER(d)]),
        "lpt2_schedule": (i, [vp, C.POINTER(i), i, C.POINTER(i)]),
        "lpt2_set_schedule": (i, [vp, C.POINTER(i), i]),
        "lpt2_tiles": (i, [vp, C.POINTER(i), C.POINTER(i), i, C.POINTER(i)]),
        "lpt2_set_tiles": (i, [vp, C.POINTER(i), C.POINTER(i), i]),
        "lpt2_autotune": (i, [vp, i, i]),
        "lpt2_displace_outputs": (i, [vp, vp, vp, vp, vp, vp, i]),
        "lpt2_timing_report": (i, [vp, C.POINTER(_KernelStat), i, C.POINTER(C.c_int)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def lpt2_last_error() -> str:
    return load_library().lpt2_last_error().decode()


def _check(rc):
    if rc != 0:
        raise LPT2Error(rc, lpt2_last_error())


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


GRAPH, HOST_IO, KEEP_STATE = 1, 2, 4


def plan_flags(graph=False, host_io=False, max_outputs=0, keep_state=False) -> int:
    """The lpt2_plan flags: LPT2_GRAPH, LPT2_HOST_IO, LPT2_KEEP_STATE, LPT2_MAX_OUTPUTS(max_outputs)."""
    return ((GRAPH if graph else 0) | (HOST_IO if host_io else 0) | (KEEP_STATE if keep_state else 0)
            | ((int(max_outputs) & 0xFF) << 8))


def _instances(insts):
    arr = (_Instance * len(insts))()
    for j, it in enumerate(insts):
        c = it.cosmo
        arr[j] = _Instance(int(it.n), float(it.box), int(it.seed) & (2 ** 64 - 1),
                           float(getattr(it, "a_out", 1.0)),
                           _Cosmo(c.omega_m, c.omega_l, c.omega_b, c.h, c.n_s, c.sigma8, c.t_cmb,
                                  c.fr0_abs, int(c.hs_n), c.a_init,
                                  int(getattr(c, "d2_variant", 0))))
    return arr


def lpt2_workspace_bytes(inst, n_k=512, graph=False, host_io=False, max_outputs=0) -> int:
    """Workspace bytes of a plan not made yet (host-side computation, no GPU needed)."""
    insts = list(inst) if isinstance(inst, (list, tuple)) else [inst]
    nb = C.c_size_t()
    _check(load_library().lpt2_workspace_bytes(_instances(insts), len(insts), int(n_k),
                                               plan_flags(graph, host_io, max_outputs), C.byref(nb)))
    return nb.value


def lpt2_debug_alloc_hook(fail_at: int) -> int:
    """Makes allocation number fail_at (from now on, counting from 0) fail; -1 turns that off.
    Returns the number of live device allocations of the library."""
    live = C.c_int64()
    _check(load_library().lpt2_debug_alloc_hook(int(fail_at), C.byref(live)))
    return live.value


class Plan:
    """Owns an lpt2 plan handle and its workspace (a torch uint8 CUDA tensor).

    `inst` is one instance or a list of instances (equal grid sizes contiguous);
    `graph=True` sets LPT2_GRAPH (needs a non-default stream); `host_io=True` sets
    LPT2_HOST_IO (lpt2_displace_host); `max_outputs=n` reserves room for n output times
    (lpt2_set_outputs); `keep_state=True` sets LPT2_KEEP_STATE (the adjoint reuses the
    forward map of the last lpt2_displace)."""

    def __init__(self, inst, n_k=512, k_min=1e-4, k_max=10.0, n_steps=1024, stream=None,
                 workspace=True, graph=False, host_io=False, max_outputs=0, keep_state=False):
        lib = load_library()
        insts = list(inst) if isinstance(inst, (list, tuple)) else [inst]
        self.insts = insts
        self.inst = insts[0]
        self.n_inst = len(insts)
        self.ns = [int(i.n) for i in insts]
        self.n = self.ns[0]
        self.cells = sum(n ** 3 for n in self.ns)
        self.n_k = int(n_k)
        self.n_steps = int(n_steps)
        self.flags = plan_flags(graph, host_io, max_outputs, keep_state)
        arr = _instances(insts)
        self._cinst = arr
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _check(lib.lpt2_plan(C.byref(h), arr, self.n_inst, self.n_k, float(k_min), float(k_max),
                             self.n_steps, _stream(self.stream), self.flags))
        self.handle = h
        self.workspace = None
        if workspace:
            nb = C.c_size_t()
            _check(lib.lpt2_workspace_size(h, C.byref(nb)))
            self.workspace = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
            _check(lib.lpt2_set_workspace(h, _ptr(self.workspace), nb.value))

    def split(self, flat, per_cell=1):
        """Views of a flat per-instance-concatenated tensor, one per instance."""
        out, off = [], 0
        for n in self.ns:
            m = per_cell * n ** 3
            out.append(flat[off:off + m])
            off += m
        return out

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load_library().lpt2_plan_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lpt2_plan(inst, **kw) -> Plan:
    return Plan(inst, **kw)


def lpt2_plan_destroy(plan: Plan):
    plan.close()


def lpt2_workspace_size(plan: Plan) -> int:
    nb = C.c_size_t()
    _check(load_library().lpt2_workspace_size(plan.handle, C.byref(nb)))
    return nb.value


def lpt2_launch_count(plan: Plan) -> int:
    return int(load_library().lpt2_launch_count(plan.handle))


PK_DECONVOLVE, PK_INTERLACE = 1, 2


def lpt2_cic_pk_est(plan: Plan, pos=None, density=False, n_shells=32, deconvolve=False, interlace=False):
    """lpt2_cic_pk with the CIC window deconvolution and / or interlacing refinements."""
    n = plan.n
    sh = (n_shells,) if plan.n_inst == 1 else (plan.n_inst, n_shells)
    res = dict(pk=torch.empty(sh, dtype=torch.float64, device="cuda"),
               k_mean=torch.empty(sh, dtype=torch.float64, device="cuda"),
               n_modes=torch.empty(sh, dtype=torch.int64, device="cuda"))
    if torch.is_tensor(density) or density:
        dsh = (n, n, n) if plan.n_inst == 1 else (plan.cells,)
        res["density"] = density if torch.is_tensor(density) else torch.empty(dsh, dtype=torch.float32, device="cuda")
    flags = (PK_DECONVOLVE if deconvolve else 0) | (PK_INTERLACE if interlace else 0)
    _check(load_library().lpt2_cic_pk_est(plan.handle, _ptr(pos), _ptr(res.get("density")), _ptr(res["pk"]),
                                          _ptr(res["k_mean"]), _ptr(res["n_modes"]), n_shells, flags))
    return res


def lpt2_source_ratio(plan: Plan, noise=None, n_bins=32, spectra=False):
    """Full second-order source term / GR, binned (mean, sigma, count, t1, k_mean); with
    spectra=True also the per-mode S_MG and S_GR half spectra (complex64 (N, N, N/2))."""
    n = plan.n
    f64 = lambda: torch.empty(n_bins, dtype=torch.float64, device="cuda")
    res = dict(mean=f64(), sigma=f64(), count=torch.empty(n_bins, dtype=torch.int64, device="cuda"),
               t1=f64(), k_mean=f64())
    if spectra:
        res["s_mg"] = torch.empty((n, n, n // 2), dtype=torch.complex64, device="cuda")
        res["s_gr"] = torch.empty((n, n, n // 2), dtype=torch.complex64, device="cuda")
    if noise is not None and (noise.dtype != torch.float32 or noise.numel() != plan.cells):
        raise ValueError("noise must be float32 with N^3 elements")
    _check(load_library().lpt2_source_ratio(plan.handle, _ptr(noise), n_bins, _ptr(res["mean"]),
                                            _ptr(res["sigma"]), _ptr(res["count"]), _ptr(res["t1"]),
                                            _ptr(res["k_mean"]), _ptr(res.get("s_mg")), _ptr(res.get("s_gr"))))
    return res


def lpt2_set_wait_budget(plan: Plan, cycles: int) -> None:
    """Cycle budget of the plan's bounded device-side waits (0: give up at once)."""
    _check(load_library().lpt2_set_wait_budget(plan.handle, int(cycles)))


def lpt2_device_status(plan: Plan) -> None:
    """Synchronises the plan's stream; raises LPT2Error if a bounded device-side wait
    gave up since the previous check."""
    _check(load_library().lpt2_device_status(plan.handle))


def lpt2_growth_tables(plan: Plan):
    """Returns (D1, D2, dD1/dln|fR0|, dD2/dln|fR0|), float64 CUDA tensors [n_k] (single
    instance) or [n_inst, n_k]."""
    shape = (plan.n_k,) if plan.n_inst == 1 else (plan.n_inst, plan.n_k)
    out = [torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(4)]
    _check(load_library().lpt2_growth_tables(plan.handle, *[_ptr(t) for t in out]))
    return tuple(out)


def lpt2_white_noise(plan: Plan, out=None):
    n = plan.n
    out = torch.empty((n, n, n), dtype=torch.float32, device="cuda") if out is None else out
    _check(load_library().lpt2_white_noise(plan.handle, _ptr(out)))
    return out


def lpt2_box_muller(plan: Plan, words):
    """Box-Muller transform of Philox word pairs: words is an int32 CUDA tensor (count, 2)
    holding uint32 bit patterns (x0, x1); returns float32 (count, 2) (cosine, sine outputs)."""
    if words.dtype != torch.int32 or words.dim() != 2 or words.shape[1] != 2:
        raise ValueError("words must be an int32 tensor of shape (count, 2)")
    out = torch.empty((words.shape[0], 2), dtype=torch.float32, device="cuda")
    _check(load_library().lpt2_box_muller(plan.handle, _ptr(words), int(words.shape[0]), _ptr(out)))
    return out


def lpt2_philox_words(seed: int, first: int, count: int, stream=None):
    """Raw Philox4x32-10 words for counters first..first+count-1: int32 tensor (count, 4)
    holding the uint32 bit patterns."""
    out = torch.empty((count, 4), dtype=torch.int32, device="cuda")
    _check(load_library().lpt2_philox_words(int(seed) & (2 ** 64 - 1), int(first), int(count),
                                            _ptr(out), _stream(stream)))
    return out


def lpt2_displace(plan: Plan, noise=None, psi1=True, psi2=True, pos=True, dk=False):
    """Forward 2LPT map. Returns dict with the requested outputs ('psi1', 'psi2' and 'pos'
    as float32 (3, N, N, N) tensors, 'dk' as complex64 (N, N, N/2) tensor; for a multi-instance
    plan flat tensors of the instances' arrays concatenated, see Plan.split)."""
    n = plan.n
    if plan.n_inst == 1:
        f3 = lambda: torch.empty((3, n, n, n), dtype=torch.float32, device="cuda")
        dshape = (n, n, n // 2)
    else:
        f3 = lambda: torch.empty(3 * plan.cells, dtype=torch.float32, device="cuda")
        dshape = (plan.cells // 2,)
    out = {}
    want = lambda v: torch.is_tensor(v) or bool(v)
    if want(psi1):
        out["psi1"] = psi1 if torch.is_tensor(psi1) else f3()
    if want(psi2):
        out["psi2"] = psi2 if torch.is_tensor(psi2) else f3()
    if want(pos):
        out["pos"] = pos if torch.is_tensor(pos) else f3()
    if want(dk):
        out["dk"] = dk if torch.is_tensor(dk) else torch.empty(dshape, dtype=torch.complex64, device="cuda")
    if noise is not None and (noise.dtype != torch.float32 or noise.numel() != plan.cells):
        raise ValueError("noise must be float32 with N^3 elements per instance")
    _check(load_library().lpt2_displace(plan.handle, _ptr(noise), _ptr(out.get("psi1")),
                                        _ptr(out.get("psi2")), _ptr(out.get("pos")),
                                        _ptr(out.get("dk"))))
    return out


def lpt2_cic_pk(plan: Plan, pos=None, density=False, n_shells=32):
    """CIC density contrast and shell P(k). pos None uses the density deposited by the
    last lpt2_displace on this plan."""
    n = plan.n
    sh = (n_shells,) if plan.n_inst == 1 else (plan.n_inst, n_shells)
    res = dict(pk=torch.empty(sh, dtype=torch.float64, device="cuda"),
               k_mean=torch.empty(sh, dtype=torch.float64, device="cuda"),
               n_modes=torch.empty(sh, dtype=torch.int64, device="cuda"))
    if torch.is_tensor(density) or density:
        dsh = (n, n, n) if plan.n_inst == 1 else (plan.cells,)
        res["density"] = density if torch.is_tensor(density) else torch.empty(
            dsh, dtype=torch.float32, device="cuda")
    if pos is not None and (pos.dtype != torch.float32 or pos.numel() != 3 * plan.cells):
        raise ValueError("pos must be float32 with 3 N^3 elements per instance")
    _check(load_library().lpt2_cic_pk(plan.handle, _ptr(pos), _ptr(res.get("density")),
                                      _ptr(res["pk"]), _ptr(res["k_mean"]), _ptr(res["n_modes"]),
                                      int(n_shells)))
    return res


def lpt2_schedule(plan: Plan):
    """Instances per launch of each grid-size group of the plan (a list)."""
    lib = load_library()
    ng = C.c_int()
    _check(lib.lpt2_schedule(plan.handle, None, 0, C.byref(ng)))
    arr = (C.c_int * max(ng.value, 1))()
    _check(lib.lpt2_schedule(plan.handle, arr, ng.value, C.byref(ng)))
    return list(arr[: ng.value])


def lpt2_set_schedule(plan: Plan, chunks):
    arr = (C.c_int * len(chunks))(*[int(c) for c in chunks])
    _check(load_library().lpt2_set_schedule(plan.handle, arr, len(chunks)))


def lpt2_tiles(plan: Plan):
    """Tile choices of each grid-size group: (ytile list, xtile list); 0 = build default."""
    lib = load_library()
    ng = C.c_int()
    _check(lib.lpt2_tiles(plan.handle, None, None, 0, C.byref(ng)))
    yt = (C.c_int * max(ng.value, 1))()
    xt = (C.c_int * max(ng.value, 1))()
    _check(lib.lpt2_tiles(plan.handle, yt, xt, ng.value, C.byref(ng)))
    return list(yt[: ng.value]), list(xt[: ng.value])


def lpt2_set_tiles(plan: Plan, ytile, xtile):
    if len(ytile) != len(xtile):
        raise ValueError("ytile and xtile need one entry per group each")
    yt = (C.c_int * len(ytile))(*[int(v) for v in ytile])
    xt = (C.c_int * len(xtile))(*[int(v) for v in xtile])
    _check(load_library().lpt2_set_tiles(plan.handle, yt, xt, len(ytile)))


def lpt2_autotune(plan: Plan, n_shells=32, reps=3):
    """Times each group's forward step at several instances-per-launch, then y-pass
    pencils per CTA and x-pass tile paths, and keeps the fastest; returns the chosen
    instances per launch (lpt2_tiles gives the tile choices)."""
    _check(load_library().lpt2_autotune(plan.handle, int(n_shells), int(reps)))
    return lpt2_schedule(plan)


def lpt2_set_outputs(plan: Plan, a_out):
    """Output scale factors for lpt2_displace_outputs (each in (a_init, 1])."""
    a = [float(x) for x in a_out]
    arr = (C.c_double * len(a))(*a)
    _check(load_library().lpt2_set_outputs(plan.handle, len(a), arr))
    plan.out_a = a


def lpt2_displace_outputs(plan: Plan, noise=None, pos=True, n_shells=32):
    """One realisation at every output scale factor of lpt2_set_outputs.  Returns a dict
    with pk (n_a, n_shells), k_mean and n_modes (n_shells,), and pos (n_a, 3, N, N, N)
    when pos is True or a tensor."""
    n = plan.n
    n_a = len(getattr(plan, "out_a", ()))
    if n_a == 0:
        raise ValueError("call lpt2_set_outputs first")
    res = dict(pk=torch.empty((n_a, n_shells), dtype=torch.float64, device="cuda"),
               k_mean=torch.empty(n_shells, dtype=torch.float64, device="cuda"),
               n_modes=torch.empty(n_shells, dtype=torch.int64, device="cuda"))
    if torch.is_tensor(pos) or pos:
        res["pos"] = pos if torch.is_tensor(pos) else torch.empty((n_a, 3, n, n, n), dtype=torch.float32,
                                                                   device="cuda")
        if res["pos"].dtype != torch.float32 or res["pos"].numel() != n_a * 3 * n ** 3:
            raise ValueError("pos must be float32 with n_a * 3 N^3 elements")
    if noise is not None and (noise.dtype != torch.float32 or noise.numel() != n ** 3):
        raise ValueError("noise must be float32 with N^3 elements")
    _check(load_library().lpt2_displace_outputs(plan.handle, _ptr(noise), _ptr(res.get("pos")), _ptr(res["pk"]),
                                                _ptr(res["k_mean"]), _ptr(res["n_modes"]), int(n_shells)))
    return res


def _hptr(t):
    if t is None:
        return None
    if t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous host (CPU) tensor")
    return C.c_void_p(t.data_ptr())


def lpt2_displace_host(plan: Plan, n_real=1, noise=None, pos=None, pk=None, n_shells=32):
    """The forward step end to end from and to host memory, n_real realisations,
    pipelined (copies overlap the kernels).  noise: CPU float32 (N, N, N) used by every
    realisation, or (n_real, N, N, N); None draws the plan's Philox noise on the device.
    pos: CPU float32 (3, N, N, N) that every realisation overwrites, or (n_real, 3, N, N, N);
    pk: CPU float64 (n_shells,) or (n_real, n_shells).  Pinned tensors (pin_memory())
    overlap best.  Returns (pos, pk) as given."""
    n = plan.n
    n3 = n ** 3

    def stride(t, dtype, one, name):
        if t is None:
            return 0
        if t.dtype != dtype or t.is_cuda:
            raise ValueError(f"{name} must be a host {dtype} tensor")
        if t.numel() == one:
            return 0
        if t.numel() == n_real * one:
            return one
        raise ValueError(f"{name} must hold one realisation or n_real of them")

    ns_ = stride(noise, torch.float32, n3, "noise")
    ps_ = stride(pos, torch.float32, 3 * n3, "pos")
    ks_ = stride(pk, torch.float64, int(n_shells), "pk")
    _check(load_library().lpt2_displace_host(plan.handle, int(n_real), _hptr(noise), ns_, _hptr(pos), ps_,
                                             _hptr(pk), ks_, int(n_shells)))
    return pos, pk


def lpt2_fft_r2c(plan: Plan, x, out=None):
    n = plan.n
    out = torch.empty((n, n, n // 2), dtype=torch.complex64, device="cuda") if out is None else out
    _check(load_library().lpt2_fft_r2c(plan.handle, _ptr(x), _ptr(out)))
    return out


def lpt2_fft_c2r(plan: Plan, X, out=None):
    n = plan.n
    out = torch.empty((n, n, n), dtype=torch.float32, device="cuda") if out is None else out
    _check(load_library().lpt2_fft_c2r(plan.handle, _ptr(X), _ptr(out)))
    return out


def lpt2_timing(plan: Plan, enable: bool):
    _check(load_library().lpt2_timing(plan.handle, 1 if enable else 0))


def lpt2_timing_report(plan: Plan):
    """{kernel name: dict(launches, total_ms, bytes)} of the launches recorded since
    lpt2_timing(plan, True) (waits for them)."""
    arr = (_KernelStat * 64)()
    n = C.c_int()
    _check(load_library().lpt2_timing_report(plan.handle, arr, 64, C.byref(n)))
    return {arr[i].name.decode(): dict(launches=int(arr[i].launches), total_ms=float(arr[i].total_ms),
                                       bytes=float(arr[i].bytes)) for i in range(n.value)}


def lpt2_set_fr0(plan: Plan, fr0_abs: float):
    """Changes |f_R0| of the plan and recomputes its growth tables on the plan's stream."""
    _check(load_library().lpt2_set_fr0(plan.handle, float(fr0_abs)))


def lpt2_displace_vjp(plan: Plan, g_density=None, g_pk=None, noise=None, n_shells=32, g_pos=None):
    """Adjoint of (noise, ln|fR0|) -> (positions, CIC density contrast, P(k)). Returns
    (g_noise, g_log_fr0) as a float32 (N, N, N) tensor and a float64 0-d tensor."""
    n = plan.n
    g_noise = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    g_t = torch.empty((), dtype=torch.float64, device="cuda")
    for tns, dt, cnt in ((g_density, torch.float32, n ** 3), (g_pk, torch.float64, n_shells),
                         (noise, torch.float32, n ** 3), (g_pos, torch.float32, 3 * n ** 3)):
        if tns is not None and (tns.dtype != dt or tns.numel() != cnt):
            raise ValueError("bad cotangent / noise tensor")
    _check(load_library().lpt2_displace_vjp(plan.handle, _ptr(noise), _ptr(g_pos), _ptr(g_density), _ptr(g_pk),
                                            int(n_shells), _ptr(g_noise), _ptr(g_t)))
    return g_noise, g_t


class Displace(torch.autograd.Function):
    """(noise, log|fR0|) -> (CIC density contrast, shell P(k)) with the hand-written
    adjoint of the library as backward.  The plan's |fR0| follows log_fr0."""

    @staticmethod
    def forward(ctx, noise, log_fr0, plan, n_shells):
        fr0 = float(torch.exp(log_fr0.detach().double()).item())
        if getattr(plan, "_fr0", plan.inst.cosmo.fr0_abs) != fr0:
            lpt2_set_fr0(plan, fr0)
        plan._fr0 = fr0
        nz = noise.detach().contiguous()
        lpt2_displace(plan, noise=nz, psi1=False, psi2=False, pos=False)
        r = lpt2_cic_pk(plan, pos=None, density=True, n_shells=n_shells)
        ctx.save_for_backward(nz)
        ctx.plan, ctx.n_shells = plan, n_shells
        return r["density"], r["pk"]

    @staticmethod
    def backward(ctx, g_density, g_pk):
        (nz,) = ctx.saved_tensors
        gd = None if g_density is None else g_density.contiguous().float()
        gp = None if g_pk is None else g_pk.contiguous().double()
        g_noise, g_t = lpt2_displace_vjp(ctx.plan, g_density=gd, g_pk=gp, noise=nz, n_shells=ctx.n_shells)
        return g_noise, g_t.to(torch.float64), None, None
