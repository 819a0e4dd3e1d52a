// Pass kernels instantiated for N = 512.
#include "passes.cuh"
LPT2_INSTANTIATE(512)
