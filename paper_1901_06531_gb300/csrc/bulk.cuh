// Bulk asynchronous copies global -> shared (cp.async.bulk, executed by the
// TMA unit) completing on an mbarrier transaction count, and bounded waits on
// that barrier.  One thread issues a copy of a contiguous block; the block's
// threads wait on the barrier's phase parity.
//
// Every wait is bounded: bulk::wait returns false after max_polls unsuccessful
// polls, and the caller records a device timeout instead of spinning forever.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bulk {

__device__ __forceinline__ unsigned saddr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// barrier with `count` expected arrivals per phase
__device__ __forceinline__ void init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

// initialised barriers visible to the asynchronous proxy (the copy engine)
__device__ __forceinline__ void fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// orders this thread's earlier generic-proxy shared-memory accesses (after a
// barrier: the block's) before later asynchronous-proxy writes to the same
// bytes: needed before a copy refills a buffer the block has just read
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// one arrival that also expects `bytes` of copy transactions in this phase
__device__ __forceinline__ void expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}

// dst (shared, 16-byte aligned) <- src (global, 16-byte aligned), bytes a
// multiple of 16; completes `bytes` transactions on bar
__device__ __forceinline__ void g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   saddr(dst)),
               "l"(src), "r"(bytes), "r"(saddr(bar))
               : "memory");
}

__device__ __forceinline__ bool try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n"
      "  .reg .pred p;\n"
      "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "  selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// true once the phase with the given parity has completed; false after
// max_polls polls
__device__ __forceinline__ bool wait(uint64_t* bar, unsigned parity, int max_polls) {
  for (int k = 0; k < max_polls; ++k)
    if (try_wait(bar, parity)) return true;
  return false;
}

}  // namespace bulk
