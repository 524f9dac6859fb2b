// Self-test of the bounded waits.  Every cluster kernel of the library waits
// on mbarrier phases completed by its peers (the core SVD's block exchanges
// and partial sums), each wait bounded so that a lost arrival ends in
// LR_ERR_TIMEOUT instead of a hung GPU.  This kernel runs that same bounded
// wait on a phase that nothing completes.
#include "cluster.cuh"
#include "common.cuh"
#include "kernels.h"

namespace lr {
namespace {

__global__ void bounded_wait_kernel(int* status, unsigned long long timeout_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // no thread arrives: phase 0 never completes
  const bool done = mbar_wait_bounded(smem_u32(&bar), 0u, timeout_ns);
  if (!done && threadIdx.x == 0) set_status(status, LR_ERR_TIMEOUT);
}

}  // namespace

void selftest_bounded_wait(int* status, uint64_t timeout_ns, cudaStream_t s) {
  bounded_wait_kernel<<<1, 32, 0, s>>>(status, static_cast<unsigned long long>(timeout_ns));
  LR_LAUNCH_CHECK();
}

}  // namespace lr
