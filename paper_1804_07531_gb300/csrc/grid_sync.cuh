// Grid-wide barrier of a cooperative launch (every CTA resident), with a
// bounded wait: the persistent thin-QR kernels meet at one of these after
// each pass over the rows of a panel.
#pragma once
#include "common.cuh"

namespace lr {
namespace gridsync {

constexpr uint64_t kTimeoutNs = 2000000000ull;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier number `index` (0, 1, ... in launch order) over the grid: ctr
// (zero at launch) counts arrivals; thread 0 of each CTA waits for
// (index + 1) * gridDim.x of them, at most kTimeoutNs, then records
// LR_ERR_TIMEOUT and raises *abort so that the other CTAs stop waiting too.
// Global writes before the barrier are visible after it (release / acquire
// through the counter).  Returns false in every thread of the CTA when the
// barrier failed here or elsewhere.  sh: one shared int.
__device__ inline bool sync(unsigned* ctr, int* abort, int* status, unsigned index, int* sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
    const unsigned target = (index + 1) * gridDim.x;
    const uint64_t t0 = now_ns();
    int ok = 1;
    while (ld_acquire(ctr) < target) {
      if (*reinterpret_cast<volatile int*>(abort)) {
        ok = 0;
        break;
      }
      if (now_ns() - t0 > kTimeoutNs) {
        set_status(status, LR_ERR_TIMEOUT);
        atomicExch(abort, 1);
        ok = 0;
        break;
      }
    }
    __threadfence();
    *sh = ok;
  }
  __syncthreads();
  return *sh != 0;
}

}  // namespace gridsync
}  // namespace lr
