"""CPU-side checks of the C ABI: the library builds/loads, exports every symbol of
include/lpt2.h, and rejects bad arguments on the host before touching a GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1909_06282_gb300 import build as B
    B.build()
    from paper_1909_06282_gb300 import _lib
    return _lib.load_library()


def test_header_declares_the_boundary():
    from paper_1909_06282_gb300._lib import HEADER_FUNCTIONS
    for name in ("lpt2_plan", "lpt2_growth_tables", "lpt2_displace", "lpt2_cic_pk",
                 "lpt2_plan_destroy", "lpt2_workspace_size", "lpt2_set_workspace", "lpt2_last_error"):
        assert name in HEADER_FUNCTIONS


def test_library_exports_every_header_symbol(lib):
    from paper_1909_06282_gb300._lib import HEADER_FUNCTIONS, library_path
    out = subprocess.run(["nm", "-D", "--defined-only", library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lpt2_\w+)", out))
    missing = [f for f in HEADER_FUNCTIONS if f not in exported]
    assert not missing, missing
    for f in HEADER_FUNCTIONS:
        assert hasattr(lib, f)


def _inst(lib_mod, **over):
    from paper_1909_06282_gb300._lib import _Cosmo, _Instance
    c = dict(omega_m=0.3, omega_l=0.7, omega_b=0.0481, h=0.7, n_s=0.96, sigma8=0.8, t_cmb=2.7255,
             fr0_abs=1e-5, hs_n=1, a_init=1e-3, d2_variant=0)
    i = dict(n=64, box=256.0, seed=1, a_out=1.0)
    for k, v in over.items():
        (c if k in c else i)[k] = v
    return _Instance(i["n"], i["box"], i["seed"], i["a_out"], _Cosmo(**c))


@pytest.mark.parametrize("over,code", [
    (dict(n=100), -4), (dict(n=0), -4), (dict(n=2048), -4), (dict(box=0.0), -1), (dict(box=-5.0), -1),
    (dict(hs_n=2), -4), (dict(d2_variant=10), -4), (dict(d2_variant=-1), -4), (dict(fr0_abs=-1e-5), -1),
    (dict(omega_m=0.3, omega_l=0.6), -1), (dict(a_out=1.5), -1), (dict(a_init=0.0), -1),
    (dict(a_out=1e-4), -1), (dict(sigma8=0.0), -1),
])
def test_plan_rejects_bad_arguments_on_host(lib, over, code):
    h = C.c_void_p()
    inst = _inst(lib, **over)
    rc = lib.lpt2_plan(C.byref(h), C.byref(inst), 1, 512, 1e-4, 10.0, 1024, None, 0)
    assert rc == code
    assert h.value is None
    assert len(lib.lpt2_last_error()) > 0


@pytest.mark.parametrize("args,code", [
    ((2, 512, 1e-4, 10.0, 1024, 0), -4),       # n_inst != 1
    ((1, 1, 1e-4, 10.0, 1024, 0), -1),         # n_k < 2
    ((1, 512, 0.0, 10.0, 1024, 0), -1),        # k_min <= 0
    ((1, 512, 1.0, 0.5, 1024, 0), -1),         # k_max <= k_min
    ((1, 512, 1e-4, 10.0, 0, 0), -1),          # n_steps < 1
    ((1, 512, 1e-4, 10.0, 5000, 0), -1),       # n_steps too large
    ((1, 512, 1e-4, 10.0, 1024, 7), -1),       # flags
])
def test_plan_rejects_bad_table_arguments(lib, args, code):
    h = C.c_void_p()
    inst = _inst(lib)
    n_inst, nk, kmin, kmax, steps, flags = args
    assert lib.lpt2_plan(C.byref(h), C.byref(inst), n_inst, nk, kmin, kmax, steps, None, flags) == code


def test_null_pointers_rejected(lib):
    assert lib.lpt2_plan(None, None, 1, 512, 1e-4, 10.0, 1024, None, 0) == -1
    assert lib.lpt2_displace(None, None, None, None, None, None) == -1
    assert lib.lpt2_cic_pk(None, None, None, None, None, None, 32) == -1
    assert lib.lpt2_workspace_size(None, None) == -1
    assert lib.lpt2_philox_words(1, 0, 4, None, None) == -1
    assert lib.lpt2_plan_destroy(None) == 0


def test_null_plan_rejected_by_the_newer_entry_points(lib):
    """Host-buffer step, output times, launch schedule and autotuner refuse a null plan
    before touching the device (no GPU needed)."""
    ng = C.c_int(-1)
    assert lib.lpt2_displace_host(None, 1, None, 0, None, 0, None, 0, 32) == -1
    assert lib.lpt2_set_outputs(None, 1, (C.c_double * 1)(0.5)) == -1
    assert lib.lpt2_displace_outputs(None, None, None, None, None, None, 32) == -1
    assert lib.lpt2_schedule(None, None, 0, C.byref(ng)) == -1 and ng.value == -1
    assert lib.lpt2_set_schedule(None, (C.c_int * 1)(1), 1) == -1
    assert lib.lpt2_autotune(None, 32, 3) == -1
    assert len(lib.lpt2_last_error()) > 0
