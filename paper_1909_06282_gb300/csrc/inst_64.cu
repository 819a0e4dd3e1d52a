// Pass kernels instantiated for N = 64.
#include "passes.cuh"
LPT2_INSTANTIATE(64)
