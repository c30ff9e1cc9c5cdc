// Asynchronous copies into shared memory for the step kernels (sm_100-class
// PTX): bulk tensor copies (TMA) completing on an mbarrier, and the mbarrier
// operations with a bounded wait.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace hyb {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// makes initialised barriers visible to the async (TMA) proxy
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// orders this thread's earlier shared-memory accesses (and those ordered
// before them by a block barrier) before later async-proxy accesses
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// Arrive on the barrier (release: this thread's earlier accesses, and those
// ordered before them by a warp barrier, happen before the phase completes).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Limit of the waits that drain a block's own copies before it exits.
constexpr long long kDrainCycles = 1LL << 29;

// Wait for the phase with the given parity of the barrier to complete, for
// at most `budget` clock cycles, giving up early once *abort is nonzero
// (another block timed out).  Returns false on timeout or abort.  Each try
// suspends the thread until the phase completes or the hint expires.  A
// negative budget only tests the phase once.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long budget, const int* abort) {
  const uint32_t a = smem_addr(bar);
  if (budget < 0) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    return done != 0;
  }
  const long long t0 = clock64();
  for (unsigned it = 1;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity), "r"(20000u)  // suspend for at most 20 us per try
        : "memory");
    if (done) return true;
    if ((it & 7) == 0 && (clock64() - t0 > budget || *(const volatile int*)abort != 0)) return false;
  }
}

// Tiled 3-D bulk tensor copy of one box into shared memory, completing
// (bytes) on the barrier.  x must be a multiple of 16 bytes / element size.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_addr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// Programmatic dependent launch: let the next launch in the stream start its
// blocks now (they wait in pdl_wait), and wait for the previous launch's
// completion and memory before touching what it wrote or read.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

}  // namespace hyb
