// Pass kernels instantiated for N = 16.
#include "passes.cuh"
LPT2_INSTANTIATE(16)
