// Shared-memory staging with 1-D bulk asynchronous copies (cp.async.bulk,
// completion counted in bytes on an mbarrier).  Every wait is bounded: after
// kWaitLimit polls it sets bit kStatusTimeout of the context's device status
// word (reported by the host as UGKS_ERR_TIMEOUT) and gives up.
#pragma once
#include <cstdint>

namespace ugks {

constexpr int kStatusTimeout = 2;        // device status bit: a bounded wait gave up
constexpr long kWaitLimit = 1L << 24;    // polls of one wait (far beyond any copy's latency)

__device__ __forceinline__ unsigned smem_u32(const void* p) { return unsigned(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes barriers initialised by this thread visible to the asynchronous
// proxy (the bulk copies complete on them); issue after the mbarrier.init
// calls and before the CTA barrier that publishes them.
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// Arrival of the issuing thread that also announces `bytes` of copies.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// Orders this thread's earlier shared-memory accesses (generic proxy) before
// later bulk copies into the same memory (async proxy): a consumer issues it
// before it releases a ring stage for refilling.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase of the given parity to complete; false (and the status
// bit set) if it did not within kWaitLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* status) {
  for (long it = 0; it < kWaitLimit; ++it)
    if (mbar_test(bar, parity)) return true;
  atomicOr(status, kStatusTimeout);
  return false;
}

// bytes (a multiple of 16, both addresses 16-byte aligned) from global to
// this CTA's shared memory; completion is counted on bar.
__device__ __forceinline__ void bulk_load(void* smem, const void* gmem, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(smem)),
      "l"(gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace ugks
