// Device helpers shared by the thread-block-cluster kernels: the circle-method
// pairing of the one-sided Jacobi sweeps, distributed-shared-memory
// addressing, bounded mbarrier waits and cluster barriers.
#pragma once
#include <cstdint>

namespace lr {

// Pair pi of round rnd (0 <= rnd < np - 1) in the circle method over np
// positions (np even): position 0 is fixed, the others rotate by one per
// round, so np - 1 rounds pair every two positions exactly once.
__device__ __forceinline__ void round_pair(int pi, int rnd, int np, int& p, int& q) {
  int ia = pi - 1 + rnd;
  if (ia >= np - 1) ia -= np - 1;
  int ib = np - 2 - pi + rnd;
  if (ib >= np - 1) ib -= np - 1;
  const int a = (pi == 0) ? 0 : 1 + ia, b = 1 + ib;
  p = min(a, b);
  q = max(a, b);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// The shared::cluster address of `addr` (a shared::cta address) in CTA `rank`.
__device__ __forceinline__ uint32_t mapa(uint32_t addr, int rank) {
  uint32_t d;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(addr), "r"(rank));
  return d;
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for phase `parity` of the mbarrier for at most timeout_ns; false on
// timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t timeout_ns) {
  if (mbar_try_wait_cluster(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait_cluster(bar, parity))
    if (globaltimer() - t0 > timeout_ns) return false;
  return true;
}
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

}  // namespace lr
