// Pass kernels instantiated for N = 1024.
#include "passes.cuh"
LPT2_INSTANTIATE(1024)
