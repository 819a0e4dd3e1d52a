// Pass kernels instantiated for N = 32.
#include "passes.cuh"
LPT2_INSTANTIATE(32)
