// Pass kernels instantiated for N = 256.
#include "passes.cuh"
LPT2_INSTANTIATE(256)
