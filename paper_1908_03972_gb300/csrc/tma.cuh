// tma.cuh -- bulk asynchronous copies from global to shared memory
// (cp.async.bulk: the TMA engine's untiled form) completed on an mbarrier,
// and a bounded wait for them.
//
// A kernel issues its copies from one thread at entry and waits for them
// where it first reads the data, so that the copies overlap the arithmetic
// before that point.  Sizes and both addresses must be multiples of 16 bytes.
// The wait gives up once its bound (wait_ns nanoseconds of the global timer,
// counted from its first unsuccessful poll, or 2^30 polls) has passed; the
// caller then records the failure in an error slot the host reads, uses the
// global-memory copy of the data instead, and before it exits drains the
// copies still in flight with mbar_drain0 (bounded by kWaitNs), so no thread
// hangs and no copy lands in the shared memory of a finished CTA.
#pragma once
#include <cuda_runtime.h>

namespace pmg {

#ifdef __CUDACC__
constexpr unsigned long long kWaitNs = 1000000000ull;   // one second

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// One-arrival barrier; the initialisation is made visible to the async proxy.
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// The single arrival, announcing the bytes the copies will deliver.
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Wait for phase 0 of the barrier; false once wait_ns have passed since the
// first unsuccessful poll.  A negative wait_ns gives up without polling (a
// diagnostic of the fallback path).
__device__ __forceinline__ bool mbar_wait0(unsigned long long* bar, double wait_ns) {
  if (wait_ns < 0.0) return false;
  const unsigned long long limit = (unsigned long long)wait_ns;
  const unsigned a = smem_u32(bar);
  unsigned long long t0 = 0;
  for (unsigned i = 0; i < (1u << 30); ++i) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a)
        : "memory");
    if (ok) return true;
    const unsigned long long t = global_ns();
    if (i == 0) t0 = t;
    else if (t - t0 > limit) return false;
  }
  return false;
}

// After a wait that gave up: wait (bounded by kWaitNs) for the copies still
// in flight, so that they land before the CTA's shared memory is released.
__device__ __forceinline__ void mbar_drain0(unsigned long long* bar) { (void)mbar_wait0(bar, (double)kWaitNs); }
#endif

}  // namespace pmg
