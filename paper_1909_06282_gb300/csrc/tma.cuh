// Bulk asynchronous copies (TMA, cp.async.bulk) into shared memory with mbarrier
// completion, and bounded waits (sm_90+ PTX, used here on sm_103a).
//
// A stage of a copy ring is one mbarrier: the issuing thread announces the byte
// count (arrive.expect_tx) and starts the copies, the TMA unit counts the bytes in
// as they land, and consumers wait on the barrier's phase parity.  Every wait is
// bounded by a cycle budget (about one second at the maximum SM clock): a wait that
// runs out reports failure instead of spinning forever.
#pragma once
#include <stdint.h>

namespace lpt2 {

#ifndef LPT2_WAIT_CYCLES
#define LPT2_WAIT_CYCLES 2000000000LL   // ~1 s at 2 GHz
#endif

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes barrier initialisation visible to the async proxy (before the first copy).
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// 1-D bulk copy global -> shared; both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// 4-D tiled bulk-tensor copy global -> shared of the box at coordinates (c0, c1, c2, c3)
// (c0 in elements of the innermost dimension, its byte offset a multiple of 16).
__device__ __forceinline__ void tensor_load_4d(void* dst, const void* tmap, int c0, int c1, int c2, int c3,
                                               uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_addr(dst)),
      "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
      : "memory");
}

// Orders this CTA's earlier shared-memory accesses (generic proxy) before later bulk copies
// into the same memory (async proxy).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of `bar` to complete; false if the cycle budget ran out.  A
// budget of 0 gives up at once without looking at the barrier (how the timeout path is
// tested: the copies are real and land, only the consumer stops waiting for them).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long budget = LPT2_WAIT_CYCLES) {
  if (budget <= 0) return false;
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > budget) return false;
  return true;
}

// Records a device-side failure code in the caller's error word (if any).
__device__ __forceinline__ void report_device_error(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

}  // namespace lpt2
