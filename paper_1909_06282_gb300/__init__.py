"""GB300-native 2LPT displacements in Hu-Sawicki f(R) gravity (Moretti et al. 2019).

Thin Python binding over the C ABI of `include/lpt2.h` (library
`lib/liblpt2.so`, built in-tree by `build.py`).  The functions here carry the
same names as the C entry points and only marshal arguments: device memory and
streams come from PyTorch, every step of the computation runs in the library's
CUDA kernels.  There is no CPU fallback: if the library is missing or no GPU
is present the calls raise.
"""
from __future__ import annotations

from ._lib import (  # noqa: F401
    LPT2Error, Plan, library_path, load_library, plan_flags, lpt2_workspace_bytes, lpt2_debug_alloc_hook,
    lpt2_plan, lpt2_plan_destroy, lpt2_workspace_size, lpt2_growth_tables, lpt2_white_noise,
    lpt2_philox_words, lpt2_box_muller, lpt2_displace, lpt2_cic_pk, lpt2_fft_r2c, lpt2_fft_c2r, lpt2_last_error,
    lpt2_launch_count, lpt2_device_status, lpt2_set_wait_budget, lpt2_source_ratio, lpt2_cic_pk_est, lpt2_timing, lpt2_timing_report, lpt2_set_fr0, lpt2_displace_vjp,
    lpt2_displace_host, lpt2_set_outputs, lpt2_displace_outputs, lpt2_schedule, lpt2_set_schedule, lpt2_tiles,
    lpt2_set_tiles, lpt2_autotune,
    Displace, HEADER_FUNCTIONS,
)
