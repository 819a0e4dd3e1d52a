// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) and Box-Muller white noise.
// Each round multiplies counter words 0 and 2 by the two published multipliers,
// xors the high halves with words 1 / 3 and the key; the key is bumped by the
// two Weyl increments between rounds.  Key = (seed lo, seed hi); counter =
// (cell lo, cell hi, 0, 0) with cell = (ix N + iy) N + iz of the cell with even
// iy; cells (ix, iy, iz) and (ix, iy+1, iz) take the cosine and sine outputs of
// the same Box-Muller transform (boxmuller.cuh).
#pragma once
#include <stdint.h>

#include "boxmuller.cuh"

namespace lpt2 {

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
#ifdef __CUDA_ARCH__
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), hi1 = __umulhi(0xCD9E8D57u, c.z);
#else
    const uint32_t hi0 = (uint32_t)(((uint64_t)0xD2511F53u * c.x) >> 32);
    const uint32_t hi1 = (uint32_t)(((uint64_t)0xCD9E8D57u * c.z) >> 32);
#endif
    const uint32_t lo0 = 0xD2511F53u * c.x, lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// (g_even, g_odd) = sqrt(-2 ln u0) (cos, sin)(2 pi u1), u = ((x >> 8) + 1) 2^-24, for the
// pair drawn at `cell`, each the correctly rounded FP32 value (boxmuller.cuh).
__device__ __forceinline__ float2 philox_gauss2(uint64_t cell, uint32_t k0, uint32_t k1,
                                                const float4* bm) {
  const uint4 x = philox4x32_10(make_uint4((uint32_t)cell, (uint32_t)(cell >> 32), 0u, 0u), k0, k1);
  return bm_pair(x.x, x.y, bm);
}

}  // namespace lpt2
