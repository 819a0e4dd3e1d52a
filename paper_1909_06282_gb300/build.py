"""Builds the in-tree CUDA library liblpt2.so for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked with the shared CUDA
runtime.  Output: paper_1909_06282_gb300/lib/liblpt2.so (git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
BUILDDIR = os.path.join(HERE, "_build")
LIBNAME = "liblpt2.so"

SOURCES = ["api.cu", "misc.cu", "growth.cu", "noalloc.cu", "source.cu"] + [f"inst_{n}.cu" for n in (16, 32, 64, 96, 128, 192, 256, 512, 1024)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(os.path.dirname(HERE), "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _extra_flags():
    """Extra nvcc flags from LPT2_NVCC_EXTRA (e.g. tuning macros -DLPT2_W512=8)."""
    return os.environ.get("LPT2_NVCC_EXTRA", "").split()


def _compile(src: str, verbose_ptxas: bool, builddir: str) -> str:
    obj = os.path.join(builddir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *_extra_flags(), "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose_ptxas:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr[-6000:]}")
    if verbose_ptxas:
        sys.stderr.write(r.stderr)
    return obj


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    for d in (CSRC, os.path.join(os.path.dirname(HERE), "include")):
        for f in os.listdir(d):
            if os.path.getmtime(os.path.join(d, f)) > t:
                return True
    return False


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None,
          out: str | None = None) -> str:
    """Builds liblpt2.so (default: lib/liblpt2.so, or the path in LPT2_LIBRARY / `out`)."""
    lib = out or os.environ.get("LPT2_LIBRARY") or os.path.join(LIBDIR, LIBNAME)
    if not force and not _stale(lib):
        return lib
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    builddir = os.path.join(BUILDDIR, os.path.basename(os.path.dirname(lib)) or "default")
    os.makedirs(builddir, exist_ok=True)
    jobs = jobs or min(len(SOURCES), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose_ptxas, builddir), SOURCES))
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stderr[-4000:])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
