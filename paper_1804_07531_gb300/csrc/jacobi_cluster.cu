// One-sided Jacobi SVD of a square core matrix on a thread-block cluster.
//
// The core SVD (the final tsvd of R_r or R_c in Alg. 2 and Alg. 9)
// is an ell x ell problem with ell up to a few hundred.  One SM cannot hold W
// and V (2 ell^2 FP32 values) for ell > ~160 and its issue rate bounds a
// sweep at ~0.2 ms for ell = 240; so the rows of W and V are split across
// the P CTAs of a cluster (P <= 8, each CTA keeps its rows in shared memory).
// Each round of the circle-method ordering rotates ell/2 disjoint column
// pairs:
//   1. every CTA computes the partial alpha = |w_p|^2, beta = |w_q|^2,
//      gamma = w_p . w_q over its rows for all pairs;
//   2. one cluster barrier;
//   3. every CTA sums the P partials of each pair in the same fixed order
//      (through distributed shared memory), so all CTAs derive bit-identical
//      rotations, and rotates its own rows of W and V.
// Because the decisions are identical everywhere, convergence (a sweep with
// no rotation) is detected without further communication.  Partials are
// double-buffered by round parity, so one cluster barrier per round suffices.
// Rotation: zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| +
// sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2), s = c t, applied when
// |gamma| > tol sqrt(alpha beta); finally s_i = |w_i|, u_i = w_i / s_i,
// sorted descending (ties by index).
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace lr {
namespace {

constexpr int kThreads = 1024;
constexpr int kMaxSweeps = 40;

// Lanes are grouped G per column pair (G a power of two, npairs * G <= 1024),
// so every pair of a round is handled in one pass by the whole CTA and the
// per-pair reductions are G-lane shuffles.
__global__ void __launch_bounds__(kThreads) jacobi_cluster_kernel(const float* __restrict__ M, int ldm, int n, int G,
                                                                  float* Uout, int ldu, float* Vout, int ldv,
                                                                  float* S, int* status) {
  cg::cluster_group cl = cg::this_cluster();
  const int P = int(cl.num_blocks());
  const int rank = int(cl.block_rank());
  const int rpc = (n + P - 1) / P;  // rows per CTA
  const int r0 = rank * rpc;
  const int nr = max(0, min(n, r0 + rpc) - r0);
  const int np = n + (n & 1);
  const int npairs = np / 2;

  extern __shared__ float sm[];
  float* W = sm;                          // nr x n, col-major (ld rpc)
  float* V = W + size_t(rpc) * n;         // rows r0.. of V, col-major (ld rpc)
  float* part = V + size_t(rpc) * n;      // [2][npairs][3], reused for norms
  float* norms = part + size_t(max(6 * npairs, 2 * n));
  int* order = reinterpret_cast<int*>(norms + n);
  __shared__ int rotated;

  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32, nwarps = kThreads / 32;
  const int gl = tid % G;            // lane within the pair group
  const int gbase = lane - gl;       // first warp lane of the group
  const int slots = kThreads / G;    // pair slots per pass (>= npairs)
  const int pi = tid / G;            // this group's pair slot
  for (int idx = tid; idx < rpc * n; idx += kThreads) {
    const int r = idx % rpc, c = idx / rpc;
    W[idx] = (r < nr) ? M[(r0 + r) + int64_t(c) * ldm] : 0.f;
    V[idx] = (r < nr && r0 + r == c) ? 1.f : 0.f;
  }
  const float tol = 1.2e-7f * sqrtf(float(n));
  const float tol2 = tol * tol;
  __syncthreads();

  int sweep = 0;
  for (; sweep < kMaxSweeps; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      float* pb = part + (rnd & 1) * 3 * npairs;
      // circle method: position 0 fixed, the others rotate by one per round
      int p = 0, q = n;
      if (pi < npairs) {
        int ia = pi - 1 + rnd;
        if (ia >= np - 1) ia -= np - 1;
        int ib = np - 2 - pi + rnd;
        if (ib >= np - 1) ib -= np - 1;
        const int a = (pi == 0) ? 0 : 1 + ia, b = 1 + ib;
        p = min(a, b);
        q = max(a, b);
      }
      const bool live = q < n;
      // 1. partial inner products over this CTA's rows
      float al = 0.f, be = 0.f, ga = 0.f;
      if (live) {
        const float* wp = W + p * rpc;
        const float* wq = W + q * rpc;
        for (int r = gl; r < nr; r += G) {
          const float x = wp[r], y = wq[r];
          al = fmaf(x, x, al);
          be = fmaf(y, y, be);
          ga = fmaf(x, y, ga);
        }
      }
      for (int o = G / 2; o > 0; o >>= 1) {
        al += __shfl_xor_sync(0xffffffffu, al, o);
        be += __shfl_xor_sync(0xffffffffu, be, o);
        ga += __shfl_xor_sync(0xffffffffu, ga, o);
      }
      if (live && gl == 0) {
        pb[3 * pi] = al;
        pb[3 * pi + 1] = be;
        pb[3 * pi + 2] = ga;
      }
      // 2. every CTA's partials are visible cluster-wide
      if (P > 1) cl.sync();
      else __syncthreads();
      // 3. identical sums in every CTA (ranks in order), then local rotation
      // lane gl of the group sums ranks gl, gl + G, ... ; the group then sums
      // its lanes 0, 1, ... -- the same order in every CTA
      float ta = 0.f, tb = 0.f, tg = 0.f;
      if (live)
        for (int k = gl; k < P; k += G) {
          const float* rp = (P > 1) ? cl.map_shared_rank(pb, k) : pb;
          ta += rp[3 * pi];
          tb += rp[3 * pi + 1];
          tg += rp[3 * pi + 2];
        }
      al = 0.f;
      be = 0.f;
      ga = 0.f;
      const int nsum = min(G, P);
      for (int k = 0; k < nsum; ++k) {
        al += __shfl_sync(0xffffffffu, ta, gbase + k);
        be += __shfl_sync(0xffffffffu, tb, gbase + k);
        ga += __shfl_sync(0xffffffffu, tg, gbase + k);
      }
      // |gamma| > tol sqrt(alpha beta), tested without square roots
      if (live && al > 0.f && be > 0.f && ga * ga > tol2 * al * be) {
        // The angle only needs to be close; orthogonality of the rotation
        // comes from c = rsqrt_rn(1 + t^2), s = c t (c^2 + s^2 = 1 to an
        // ulp for any t), so t uses the fast division and square root.
        const float zeta = __fdividef(be - al, 2.f * ga);
        const float t = copysignf(1.f, zeta) * __frcp_rn(fabsf(zeta) + __fsqrt_rn(fmaf(zeta, zeta, 1.f)));
        const float c = __frsqrt_rn(fmaf(t, t, 1.f));
        const float s = c * t;
        float* wp = W + p * rpc;
        float* wq = W + q * rpc;
        float* vp = V + p * rpc;
        float* vq = V + q * rpc;
        for (int r = gl; r < nr; r += G) {
          const float x = wp[r], y = wq[r];
          wp[r] = c * x - s * y;
          wq[r] = s * x + c * y;
          const float u = vp[r], w = vq[r];
          vp[r] = c * u - s * w;
          vq[r] = s * u + c * w;
        }
        if (gl == 0) rotated = 1;
      }
      __syncthreads();
    }
    // converged once no pair needed a rotation (the same decision in every
    // CTA of the cluster)
    if (!rotated) break;
    __syncthreads();
  }
  (void)slots;
  (void)warp;
  (void)nwarps;
  if (sweep == kMaxSweeps && rank == 0 && tid == 0) set_status(status, LR_ERR_NONFINITE);
#ifdef LR_JACOBI_SWEEPS_OUT
  if (rank == 0 && tid == 0) LR_JACOBI_SWEEPS_OUT = sweep;
#endif
  // peers may still be reading the last round's partials from this CTA
  cl.sync();

  // Column norms of W: partial over local rows, cluster-wide sum, identical order.
  // V's columns are unit vectors in exact arithmetic; their norm drift is
  // removed the same way.
  float* pn = part;  // [n] partial |w_c|^2 then [n] partial |v_c|^2
  for (int c = tid; c < n; c += kThreads) {
    float aw = 0.f, av = 0.f;
    for (int r = 0; r < nr; ++r) {
      aw = fmaf(W[r + c * rpc], W[r + c * rpc], aw);
      av = fmaf(V[r + c * rpc], V[r + c * rpc], av);
    }
    pn[c] = aw;
    pn[n + c] = av;
  }
  cl.sync();
  for (int c = tid; c < n; c += kThreads) {
    float sw = 0.f, sv = 0.f;
    for (int k = 0; k < P; ++k) {
      const float* rp = (P > 1) ? cl.map_shared_rank(pn, k) : pn;
      sw += rp[c];
      sv += rp[n + c];
    }
    norms[c] = sqrtf(sw);
    const float inv = 1.f / sqrtf(sv);
    for (int r = 0; r < nr; ++r) V[r + c * rpc] *= inv;
  }
  __syncthreads();
  for (int c = tid; c < n; c += kThreads) {
    int rk = 0;
    const float v = norms[c];
    for (int d = 0; d < n; ++d) {
      const float o = norms[d];
      rk += (o > v) || (o == v && d < c);
    }
    order[rk] = c;
  }
  __syncthreads();
  for (int idx = tid; idx < nr * n; idx += kThreads) {
    const int r = idx % nr, j = idx / nr;
    const int c = order[j];
    const float nv = norms[c];
    Uout[(r0 + r) + int64_t(j) * ldu] = nv > 0.f ? W[r + c * rpc] / nv : 0.f;
    Vout[(r0 + r) + int64_t(j) * ldv] = V[r + c * rpc];
  }
  if (rank == 0)
    for (int j = tid; j < n; j += kThreads) S[j] = norms[order[j]];
  // no CTA may exit while a peer can still read its shared memory
  cl.sync();
}

size_t cluster_smem(int n, int P) {
  const int rpc = (n + P - 1) / P;
  const int npairs = (n + 1) / 2;
  return (size_t(2) * rpc * n + std::max(6 * npairs, 2 * n) + n) * sizeof(float) + size_t(n) * sizeof(int) + 64;
}

}  // namespace

// Cluster size for an n x n core (0: does not fit a cluster of <= 8).
int jacobi_cluster_size(int n) {
  // Smallest cluster whose CTAs hold their rows of W and V (wider clusters
  // pay more for the per-round cluster barrier than they save in work).
  for (int P = 1; P <= 8; P *= 2)
    if (cluster_smem(n, P) <= size_t(200) * 1024) return P;
  return 0;
}

void jacobi_svd_cluster(const float* M, int ldm, int n, float* U, int ldu, float* V, int ldv, float* S, int* status,
                        cudaStream_t s) {
  const int P = jacobi_cluster_size(n);
  LR_REQUIRE(P > 0, LR_ERR_UNSUPPORTED, "core SVD too large for a cluster");
  const size_t smem = cluster_smem(n, P);
  static bool attr[64] = {};
  int dev = 0;
  LR_CHECK_CUDA(cudaGetDevice(&dev));
  if (!attr[dev & 63]) {
    LR_CHECK_CUDA(cudaFuncSetAttribute(jacobi_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024));
    attr[dev & 63] = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = P;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const int npairs = (n + 1) / 2;
  int G = 32;
  while (G > 1 && npairs * G > kThreads) G /= 2;
  LR_REQUIRE(npairs * G <= kThreads, LR_ERR_UNSUPPORTED, "core SVD too wide");
  LR_CHECK_CUDA(cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel, M, ldm, n, G, U, ldu, V, ldv, S, status));
  LR_LAUNCH_CHECK();
}

}  // namespace lr
