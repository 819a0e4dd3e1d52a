// Pass kernels instantiated for N = 128.
#include "passes.cuh"
LPT2_INSTANTIATE(128)
