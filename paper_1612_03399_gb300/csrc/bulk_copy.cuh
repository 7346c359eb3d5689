// mbarrier and bulk-copy primitives (PTX, sm_90 and later) shared by the
// kernels that move contiguous tables into shared memory with
// cp.async.bulk: one thread initialises the barrier, announces the bytes and
// issues the copies; every thread waits on phase 0 with a bounded spin.
#pragma once

#include <cuda_runtime.h>

namespace ibm {

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
  // the initialisation is visible to the bulk-copy unit before its first use
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// global -> shared, 16-byte aligned addresses, bytes a multiple of 16
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                          unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(r)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return r != 0;
}
// wait for phase 0 of the barrier, at most about `limit` SM clocks
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, long long limit) {
  const long long t0 = clock64();
  while (!mbar_test(bar, 0)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}
constexpr long long kCopyWaitClocks = 1ll << 31;   // about a second

}  // namespace ibm
