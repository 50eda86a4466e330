// mbarrier and bulk-copy (TMA, cp.async.bulk) helpers shared by the staged kernels. Every
// wait is bounded by a clock budget; on expiry the caller records an error and drains.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mlmc {

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* b, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return done != 0;
}
// bounded wait: one non-blocking test, then waits while fewer than `budget` SM clocks
// have passed (budget 0: give up at the first test that finds the phase incomplete)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* b, unsigned parity, long long budget) {
  if (mbar_test_wait(b, parity)) return true;
  const long long t0 = clock64();
  while (clock64() - t0 < budget)
    if (mbar_try_wait(b, parity)) return true;
  return false;
}
// budget of the drain after an expired wait (the copies still in flight must land before
// the CTA's shared memory is released): about one second of SM clock, whatever the
// budget of the normal waits
constexpr long long kDrainBudget = 2000000000LL;
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(b))
      : "memory");
}
// makes an mbarrier's initialisation visible to the async (bulk-copy) proxy
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
// orders this thread's generic-proxy shared-memory accesses before later async-proxy ones
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

}  // namespace mlmc
