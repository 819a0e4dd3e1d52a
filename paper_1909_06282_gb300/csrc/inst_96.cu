// Pass kernels instantiated for N = 96.
#include "passes.cuh"
LPT2_INSTANTIATE(96)
