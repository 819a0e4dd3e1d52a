// Pass kernels instantiated for N = 192.
#include "passes.cuh"
LPT2_INSTANTIATE(192)
