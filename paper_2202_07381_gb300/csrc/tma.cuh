// Bulk-copy (TMA) and mbarrier helpers shared by the staged patch kernels:
// 1D cp.async.bulk global -> shared copies completing on an mbarrier, an L2
// evict-first policy for data streamed once, and bounded waits (a poll limit
// and a 2 s wall-clock limit) so that no wait can spin forever.
#pragma once

#include <cstdint>

namespace irkmg {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// L2 policy for data read exactly once per sweep (the patch inverses): evict
// first, so the stream does not push the residual and target vectors out of L2.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                         uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], "
      "%2, [%3], %4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) accesses to the same memory.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Non-blocking test of a phase (mbarrier.test_wait returns at once, where
// try_wait may suspend the thread for a while first).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on a stage barrier: at most `spins` polls, the first one
// non-blocking and the others (try_wait) allowed a short hardware-chosen
// suspension, and at most 2 s of wall time; false if either bound expired.
// spins = 1 is a single non-blocking poll.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int64_t spins) {
  if (mbar_test_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (int64_t k = 1; k < spins; ++k) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((k & 255) == 255 && global_ns() - t0 > 2000000000ull) return false;
  }
  return false;
}

// Wait for a copy this CTA issued before the CTA leaves after an expired wait.
// It has its own bound (2^26 polls and the 2 s wall-clock limit), not the
// caller's timeout, which may be tiny: a CTA must not exit while a bulk copy
// is still landing in its shared memory.
constexpr int64_t kDrainSpins = (int64_t)1 << 26;
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
  mbar_wait_bounded(bar, parity, kDrainSpins);
}

}  // namespace irkmg
