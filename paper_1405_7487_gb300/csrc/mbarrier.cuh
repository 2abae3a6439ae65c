// mbarrier.cuh -- shared-memory barriers and bulk copies (sm_90 and later)
// used by the kernels that stage data with the asynchronous copy engine.
#pragma once

#include <cstdint>

namespace gbfmm {

// Polls of a bounded mbarrier wait before it gives up.
constexpr long long kSpinLimit = 1ll << 20;
// Polls of the wait that drains a copy or tensor-core operation still in
// flight after a block gave up, before the block ends or frees its tensor
// memory (a block must not end while a copy into its shared memory can still
// land).
constexpr long long kDrainSpinLimit = 1ll << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar),
               "r"(bytes)
               : "memory");
}

// Bounded wait for the phase with the given parity; false if it gave up (it
// then sets *abort_flag) or another thread raised *abort_flag.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          long long limit = kSpinLimit) {
  for (long long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 1023) == 1023 && *abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

// Drain after a give-up: waits (bounded, kDrainSpinLimit polls, no abort) for
// the phase with the given parity; false if that also gave up.
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity) {
  volatile int none = 0;
  return mbar_wait(bar, parity, &none, kDrainSpinLimit);
}

// Orders this thread's (and, after a barrier, the block's) generic-proxy
// shared-memory accesses before its later async-proxy ones.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global to this CTA's shared memory, completing on the mbarrier bar.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

}  // namespace gbfmm
