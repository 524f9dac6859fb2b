// One-sided Jacobi SVD of a square core matrix on a thread-block cluster,
// rows split over the CTAs.
//
// The core SVD (the final tsvd of R_r or R_c in Alg. 2 and Alg. 9, and of the
// small factors of Alg. 7) is an n x n problem.  Cores of n <= 512 run on the
// column-block kernel (jacobi_block.cu), which exchanges data 2P - 1 times
// per sweep instead of once per round; this kernel serves the wider square
// cores whose W and V fit the cluster's shared memory.  One-sided Jacobi on
// M: W = M V, rotating column pairs of W (and V) until every pair is
// orthogonal to working precision; then sigma_i = |w_i|, u_i = w_i / sigma_i.
//
// The work is latency-bound: a sweep is n - 1 rounds of n / 2 disjoint
// rotations (circle-method ordering), and every round needs three inner
// products over all n rows before any rotation can be applied.  A cluster of
// P CTAs splits the rows of W and V (n / P each, in shared memory).  Per
// round every CTA
//   1. computes alpha = |w_p|^2, beta = |w_q|^2, gamma = w_p . w_q over its
//      rows for all pairs of the round;
//   2. pushes these partials into every CTA's shared memory with st.async,
//      each store completing transaction bytes on the receiver's mbarrier for
//      that buffer (no cluster-wide barrier);
//   3. while the peers' partials are in flight, applies the previous round's
//      rotations to its rows of V (V never feeds an inner product);
//   4. waits on its own mbarrier until all P partials have landed, sums them
//      in rank order -- the same order in every CTA, so all CTAs derive
//      bit-identical rotations and agree on convergence without more
//      communication -- and rotates its rows of W.
// The partial buffers alternate by a running round count; a CTA cannot run
// two rounds ahead of a peer (it needs the peer's partials of the round in
// between), so a buffer is never overwritten while it is read.
//
// The shared-memory layout keeps the float4 accesses free of bank conflicts:
// column strides and per-rank slot strides are odd numbers of 16-byte units.
//
// Rotation: zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| +
// sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2), s = c t, applied when
// gamma^2 > tol^2 alpha beta (tol = eps sqrt(n)).  W and V receive the same
// rotations, so W = M V holds throughout; finally sigma_i = |w_i| / |v_i|,
// u_i = w_i / |w_i|, v_i / |v_i|, sorted by sigma descending (ties by index).
#include <cooperative_groups.h>

#include <algorithm>

#include "cluster.cuh"
#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace lr {
namespace {

constexpr int kThreads = 512;  // upper bound of the block (npairs * G threads)
constexpr int kMaxSweeps = 40;
constexpr uint64_t kTimeoutNs = 2000000000ull;     // bound of every mbarrier wait
constexpr size_t kSmemLimit = size_t(225) * 1024;  // dynamic shared memory per CTA

// 16-byte store into a peer's shared memory that completes 16 transaction
// bytes on the peer's mbarrier.
__device__ __forceinline__ void st_async_v4(uint32_t dst, float a, float b, float c, float d, uint32_t mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(dst),
               "f"(a), "f"(b), "f"(c), "f"(d), "r"(mbar)
               : "memory");
}

// [x y] <- [x y] [[c, s], [-s, c]] on the lane's float4 rows.
__device__ __forceinline__ void rotate4(float4* xp, float4* yp, int rq, int gl, int G, float c, float s) {
  for (int j = gl; j < rq; j += G) {
    const float4 x = xp[j], y = yp[j];
    xp[j] = make_float4(c * x.x - s * y.x, c * x.y - s * y.y, c * x.z - s * y.z, c * x.w - s * y.w);
    yp[j] = make_float4(s * x.x + c * y.x, s * x.y + c * y.y, s * x.z + c * y.z, s * x.w + c * y.w);
  }
}

// Shared-memory geometry (in floats), used by the kernel and the host.
struct Geo {
  int rows, rq, ld, npairs, slot, PS;
  size_t floats;
  __host__ __device__ Geo(int n, int P) {
    rows = (n + P - 1) / P;     // rows of W and V per CTA
    rq = ((rows + 3) / 4) | 1;  // float4 per column, odd
    ld = 4 * rq;
    npairs = (n + 1) / 2;
    slot = npairs | 1;          // float4 slots per rank, odd
    PS = 4 * slot;
    // partials [2][P][slot] float4, W and V (ld x n each), norms, 1/|v|, order
    floats = size_t(2) * P * PS + size_t(2) * ld * n + size_t(3) * n;
  }
};

// Lanes are grouped G per column pair (npairs * G threads, rounded up to a
// warp; one lane per pair measured fastest, as the per-pair work -- pair
// indices, sums over ranks, the angle -- is then not replicated); each lane
// walks its rows four at a time (the padding rows are kept
// zero).  The group butterflies leave bit-identical sums in every lane.
template <int G>
__global__ void __launch_bounds__(kThreads) jacobi_cluster_kernel(const float* __restrict__ M, int ldm, int n,
                                                                  float* __restrict__ Uout, int ldu,
                                                                  float* __restrict__ Vout, int ldv,
                                                                  float* __restrict__ S, int* status) {
  cg::cluster_group cl = cg::this_cluster();
  const int P = int(cl.num_blocks());
  const int rank = int(cl.block_rank());
  const Geo g(n, P);
  const int rq = g.rq, ld = g.ld, npairs = g.npairs, PS = g.PS;
  const int r0 = rank * g.rows;
  const int nr = max(0, min(n, r0 + g.rows) - r0);
  const int np = n + (n & 1);
  const int nt = blockDim.x;

  extern __shared__ __align__(16) float sm[];
  float* part = sm;                        // [2][P][slot] float4 pushed partials
  float* W = part + size_t(2) * P * PS;    // ld x n, col-major
  float* V = W + size_t(ld) * n;           // ld x n, col-major
  float* norms = V + size_t(ld) * n;       // |w_j| / |v_j|
  float* vinv = norms + n;                 // 1 / |v_j|
  int* order = reinterpret_cast<int*>(vinv + n);
  float4* W4 = reinterpret_cast<float4*>(W);
  float4* V4 = reinterpret_cast<float4*>(V);
  __shared__ __align__(8) uint64_t arrived[2];  // per buffer: all P partials landed
  __shared__ int rotated, aborted;

  const int tid = threadIdx.x;
  const int gl = tid % G;    // lane within the pair group
  const int pi = tid / G;    // this group's pair
  for (int idx = tid; idx < ld * n; idx += nt) {
    const int r = idx % ld, c = idx / ld;
    W[idx] = (r < nr) ? M[(r0 + r) + int64_t(c) * ldm] : 0.f;
    V[idx] = (r < nr && r0 + r == c) ? 1.f : 0.f;
  }
  const float tol = 1.2e-7f * sqrtf(float(n));
  const float tol2 = tol * tol;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&arrived[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&arrived[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    aborted = 0;
  }
  // every CTA's mbarriers are initialised before any peer stores to them
  cluster_barrier();
  const uint32_t bytes_per_round = uint32_t(P) * uint32_t(npairs) * 16u;

  // the previous round's rotation of this group's pair, applied to V late
  int vp = 0, vq = 0;
  float vc = 1.f, vs = 0.f;
  bool vpending = false;
  int sweep = 0;
  uint32_t it = 0;  // running round count: buffer it & 1, phase (it >> 1) & 1
  for (; sweep < kMaxSweeps; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int rnd = 0; rnd < np - 1; ++rnd, ++it) {
      const uint32_t b = it & 1u;
      float* buf = part + b * P * PS;
      if (tid == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&arrived[b])),
                     "r"(bytes_per_round)
                     : "memory");
      int p = 0, q = n;
      if (pi < npairs) round_pair(pi, rnd, np, p, q);
      const bool live = q < n;
      // 1. partial inner products over this CTA's rows
      float al = 0.f, be = 0.f, ga = 0.f;
      if (live) {
        const float4* wp = W4 + p * rq;
        const float4* wq = W4 + q * rq;
        for (int j = gl; j < rq; j += G) {
          const float4 x = wp[j], y = wq[j];
          al = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, al))));
          be = fmaf(y.x, y.x, fmaf(y.y, y.y, fmaf(y.z, y.z, fmaf(y.w, y.w, be))));
          ga = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, ga))));
        }
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        al += __shfl_xor_sync(0xffffffffu, al, o);
        be += __shfl_xor_sync(0xffffffffu, be, o);
        ga += __shfl_xor_sync(0xffffffffu, ga, o);
      }
      // 2. push them into slot `rank` of every CTA's buffer (every pair of
      // the round, dead ones as zeros, so the byte count is fixed)
      if (pi < npairs) {
        const uint32_t src = smem_u32(buf + rank * PS + 4 * pi), bar = smem_u32(&arrived[b]);
        for (int k = gl; k < P; k += G) st_async_v4(mapa(src, k), al, be, ga, 0.f, mapa(bar, k));
      }
      // 3. the previous round's rotation of V, while the partials travel
      if (vpending) rotate4(V4 + vp * rq, V4 + vq * rq, rq, gl, G, vc, vs);
      // 4. wait until all P partials of this round have landed here
      {
        const uint32_t bar = smem_u32(&arrived[b]), par = (it >> 1) & 1u;
        if (!mbar_try_wait_cluster(bar, par)) {
          const uint64_t t0 = globaltimer();
          while (!mbar_try_wait_cluster(bar, par)) {
            if (globaltimer() - t0 > kTimeoutNs) {
              aborted = 1;
              set_status(status, LR_ERR_TIMEOUT);
              break;
            }
          }
        }
      }
      // identical sums in every CTA: lane gl takes ranks gl, gl + G, .. in
      // order, then the group butterfly
      float ta = 0.f, tb = 0.f, tg = 0.f;
      if (live)
        for (int k = gl; k < P; k += G) {
          const float4 v = *reinterpret_cast<const float4*>(buf + k * PS + 4 * pi);
          ta += v.x;
          tb += v.y;
          tg += v.z;
        }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        ta += __shfl_xor_sync(0xffffffffu, ta, o);
        tb += __shfl_xor_sync(0xffffffffu, tb, o);
        tg += __shfl_xor_sync(0xffffffffu, tg, o);
      }
      vpending = live && ta > 0.f && tb > 0.f && tg * tg > tol2 * ta * tb;
      if (vpending) {
        // The angle only needs to be close; orthogonality of the rotation
        // comes from c = rsqrt_rn(1 + t^2), s = c t (c^2 + s^2 = 1 to an
        // ulp for any t), so t uses the fast division and square root.
        const float zeta = __fdividef(tb - ta, 2.f * tg);
        const float t = copysignf(1.f, zeta) * __frcp_rn(fabsf(zeta) + __fsqrt_rn(fmaf(zeta, zeta, 1.f)));
        vc = __frsqrt_rn(fmaf(t, t, 1.f));
        vs = vc * t;
        vp = p;
        vq = q;
        rotate4(W4 + p * rq, W4 + q * rq, rq, gl, G, vc, vs);
        if (gl == 0) rotated = 1;
      }
      __syncthreads();
      if (aborted) break;
    }
    // converged once no pair needed a rotation (the same decision in every
    // CTA of the cluster)
    if (!rotated || aborted) break;
    __syncthreads();
  }
  if (vpending) rotate4(V4 + vp * rq, V4 + vq * rq, rq, gl, G, vc, vs);
  if (sweep == kMaxSweeps && rank == 0 && tid == 0) set_status(status, LR_ERR_NONFINITE);

  // Column norms of W and V: partials over local rows pushed to every CTA,
  // summed in rank order.  Peers may still read the last round's partials,
  // so the buffer is reused only after a cluster barrier (after a timeout the
  // outputs are meaningless, but every CTA passes the same barriers).
  cluster_barrier();
  for (int col = tid; col < n; col += nt) {
    float aw = 0.f, av = 0.f;
    for (int r = 0; r < nr; ++r) {
      aw = fmaf(W[r + col * ld], W[r + col * ld], aw);
      av = fmaf(V[r + col * ld], V[r + col * ld], av);
    }
    for (int k = 0; k < P; ++k) {
      float* dst = cl.map_shared_rank(part, k);
      dst[rank * n + col] = aw;
      dst[(P + rank) * n + col] = av;
    }
  }
  cluster_barrier();
  for (int col = tid; col < n; col += nt) {
    float sw = 0.f, sv = 0.f;
    for (int k = 0; k < P; ++k) {
      sw += part[k * n + col];
      sv += part[(P + k) * n + col];
    }
    const float iv = sv > 0.f ? 1.f / sqrtf(sv) : 0.f;
    norms[col] = sqrtf(sw) * iv;
    vinv[col] = iv;
  }
  __syncthreads();
  for (int col = tid; col < n; col += nt) {
    int rk = 0;
    const float v = norms[col];
    for (int d = 0; d < n; ++d) {
      const float o = norms[d];
      rk += (o > v) || (o == v && d < col);
    }
    order[rk] = col;
  }
  __syncthreads();
  for (int idx = tid; idx < nr * n; idx += nt) {
    const int r = idx % nr, j = idx / nr;
    const int col = order[j];
    const float sc = norms[col] / vinv[col];  // |w_col|
    Uout[(r0 + r) + int64_t(j) * ldu] = sc > 0.f ? W[r + col * ld] / sc : 0.f;
    Vout[(r0 + r) + int64_t(j) * ldv] = V[r + col * ld] * vinv[col];
  }
  if (rank == 0)
    for (int j = tid; j < n; j += nt) S[j] = norms[order[j]];
}

size_t cluster_smem(int n, int P) { return Geo(n, P).floats * sizeof(float) + 64; }

template <int G>
void launch(int P, size_t smem, cudaStream_t s, const float* M, int ldm, int n, float* U, int ldu, float* V, int ldv,
            float* S, int* status) {
  static std::atomic<bool> attr[64];  // attributes set, per device
  int dev = 0;
  LR_CHECK_CUDA(cudaGetDevice(&dev));
  if (!attr[dev & 63]) {
    LR_CHECK_CUDA(
        cudaFuncSetAttribute(jacobi_cluster_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmemLimit)));
    LR_CHECK_CUDA(cudaFuncSetAttribute(jacobi_cluster_kernel<G>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    attr[dev & 63] = true;
  }
  const int npairs = (n + 1) / 2;
  const int threads = (npairs * G + 31) / 32 * 32;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = P;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  LR_CHECK_CUDA(cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel<G>, M, ldm, n, U, ldu, V, ldv, S, status));
  LR_LAUNCH_CHECK();
}

}  // namespace

// Cluster size for an n x n core (0: W and V do not fit a cluster of <= 16).
int jacobi_cluster_size(int n) {
  const int P0 = n >= 128 ? 8 : n >= 64 ? 4 : 1;
  for (int P = P0; P <= 16; P *= 2)
    if (cluster_smem(n, P) <= kSmemLimit && (n + 1) / 2 <= kThreads) return P;
  return 0;
}

void jacobi_svd_cluster(const float* M, int ldm, int n, float* U, int ldu, float* V, int ldv, float* S, int* status,
                        cudaStream_t s, int P, int G) {
  if (P <= 0) P = jacobi_cluster_size(n);
  LR_REQUIRE(P == 1 || P == 2 || P == 4 || P == 8 || P == 16, LR_ERR_UNSUPPORTED, "core SVD too large for a cluster");
  const int npairs = (n + 1) / 2;
  if (G <= 0) G = 1;  // measured fastest: the per-pair work is not replicated
  LR_REQUIRE(npairs * G <= kThreads, LR_ERR_UNSUPPORTED, "core SVD too wide for the lane grouping");
  const size_t smem = cluster_smem(n, P);
  LR_REQUIRE(smem <= kSmemLimit, LR_ERR_UNSUPPORTED, "core SVD does not fit the cluster");
  switch (G) {
    case 1: launch<1>(P, smem, s, M, ldm, n, U, ldu, V, ldv, S, status); break;
    case 2: launch<2>(P, smem, s, M, ldm, n, U, ldu, V, ldv, S, status); break;
    case 4: launch<4>(P, smem, s, M, ldm, n, U, ldu, V, ldv, S, status); break;
    default: LR_REQUIRE(false, LR_ERR_UNSUPPORTED, "lanes per pair must be 1, 2 or 4");
  }
}

}  // namespace lr
