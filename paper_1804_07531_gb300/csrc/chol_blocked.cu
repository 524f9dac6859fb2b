// Cholesky and triangular inverse of one small matrix (order <= 128) in one
// CTA, for the CholeskyQR passes of the thin QR (the paper's qr between
// views, Alg. 2 / Alg. 9) and for R^{-1} in the single-pass and row-streamed
// schedules.  The factorisation and inverse routines are in chol_cta.cuh;
// this file loads the FP64 Gram, handles breakdown (the shift of shifted
// CholeskyQR) and writes R^{-1} (FP32) and R (FP64).
//
// Orders that are not a multiple of 32 are padded with an identity block,
// whose factor and inverse are the identity.
#include "chol_cta.cuh"
#include "kernels.h"

namespace lr {
namespace {

using chol::kB;
using chol::kMaxN;
constexpr int kThreadsC = 384;

// Loads the n x n FP64 matrix G (ld n) into A (FP32, N x N, ld), identity
// padded, optionally adding shift to the diagonal; zeroes Xt.  Returns true
// (uniformly, after a barrier) when G has a non-finite entry.
__device__ bool load_gram(const double* __restrict__ G, int n, int N, int ld, float shift, float* A, float* Xt,
                          int* flag) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) *flag = 0;
  __syncthreads();
  bool bad = false;
  // loads issued eight at a time so that their latencies overlap
  for (int base = tid; base < N * N; base += 8 * nt) {
    double g[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * nt, r = idx % N, c = idx / N;
      g[u] = (idx < N * N && r < n && c < n) ? G[r + c * n] : (r == c ? 1.0 : 0.0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * nt, r = idx % N, c = idx / N;
      if (idx >= N * N) continue;
      if (!isfinite(g[u])) bad = true;
      A[r + c * ld] = float(g[u]) + ((r == c && r < n) ? shift : 0.f);
      Xt[r + c * ld] = 0.f;
    }
  }
  if (bad) *flag = 1;
  __syncthreads();
  return *flag != 0;
}

// Cholesky G = R^T R (G FP64 in global memory, factorised in FP32 in shared
// memory), then Rinv = R^{-1} and Racc = R (FP64; may be null).
// mode: CHOL_PLAIN           plain Cholesky (a non-positive pivot is a
//                            breakdown);
//       CHOL_SHIFT_IF_NEEDED plain first; on breakdown retry with the shift of
//                            shifted CholeskyQR (Fukaya et al. 2020),
//                            1e-5 trace(G), and set *needs_more = 1 so the
//                            caller's optional pass runs;
//       CHOL_SHIFT_IF_FLAGGED the shifted factorisation when *needs_more != 0
//                            (the pass after a shifted one, for
//                            rank-deficient input), the plain one otherwise;
//       CHOL_IF_FLAGGED      run only when *needs_more != 0 (else nothing).
__global__ void __launch_bounds__(kThreadsC) chol_inv_kernel(const double* __restrict__ G, int n, float* Rinv,
                                                             int ldr, double* Racc, int ldacc, int mode,
                                                             int* needs_more, int* status) {
  const bool flagged = needs_more != nullptr && *needs_more != 0;
  if (mode == CHOL_IF_FLAGGED && !flagged) return;
  extern __shared__ float4 sm4[];
  float* sm = reinterpret_cast<float*>(sm4);
  const int N = (n + kB - 1) / kB * kB, ld = chol::ld_of(N);
  float* A = sm;
  float* Xt = A + N * ld;
  float* Xd = Xt + N * ld;
  float* T = Xd + N * chol::kDld;
  float* dinv = T + kB * chol::t_ld(N);
  float* colbuf = dinv + N;
  __shared__ int flag;
  __shared__ double tr;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid < 32) {  // trace of G (the norm estimate for the shift)
    double t = 0.0;
    for (int i = tid; i < n; i += 32) t += G[i + i * n];
    t = warp_sum(t);
    if (tid == 0) tr = t;
  }
  bool broke = false, shifted = false;
  const bool shift_first = mode == CHOL_SHIFT_IF_FLAGGED && flagged;
  for (int attempt = shift_first ? 1 : 0; attempt < 2; ++attempt) {
    shifted = attempt == 1;
    // the shift sits above the FP32 Gram and Cholesky rounding level, so
    // the shifted factorisation cannot break down
    __syncthreads();
    const float shift = shifted ? float(1e-5 * tr) : 0.f;
    if (load_gram(G, n, N, ld, shift, A, Xt, &flag)) {
      if (tid == 0) set_status(status, LR_ERR_NONFINITE);
      return;
    }
    broke = chol::block_chol(A, N, ld, dinv, colbuf, &flag);
    if (!broke || mode != CHOL_SHIFT_IF_NEEDED) break;
  }
  if (!broke && shifted && mode == CHOL_SHIFT_IF_NEEDED && tid == 0 && needs_more) *needs_more = 1;
  if (broke) {
    if (tid == 0) set_status(status, LR_ERR_BREAKDOWN);
    // leave a harmless identity so later kernels stay finite
    for (int idx = tid; idx < n * n; idx += nt) {
      const int r = idx % n, c = idx / n;
      Rinv[r + c * ldr] = (r == c) ? 1.f : 0.f;
    }
    return;
  }
  chol::block_inverse(A, Xt, Xd, T, dinv, N, ld);
  // R^{-1} = X^T (upper), R = L^T
  for (int idx = tid; idx < n * n; idx += nt) {
    const int r = idx % n, c = idx / n;
    Rinv[r + c * ldr] = Xt[r + c * ld];
  }
  if (Racc)
    for (int idx = tid; idx < n * n; idx += nt) {
      const int r = idx % n, c = idx / n;
      Racc[r + c * ldacc] = (r <= c) ? double(A[c + r * ld]) : 0.0;
    }
}

// X = R^{-1} (FP32, upper) for an upper-triangular FP64 R of order n <= 128:
// L = R^T, its inverse by the routines above, R^{-1} = (L^{-1})^T.
__global__ void __launch_bounds__(kThreadsC) tri_inv_kernel(const double* __restrict__ R, int ldr, int n, float* Xout,
                                                            int ldx, int* status) {
  extern __shared__ float4 sm4[];
  float* sm = reinterpret_cast<float*>(sm4);
  const int N = (n + kB - 1) / kB * kB, ld = chol::ld_of(N);
  float* L = sm;
  float* Xt = L + N * ld;
  float* Xd = Xt + N * ld;
  float* T = Xd + N * chol::kDld;
  float* dinv = T + kB * chol::t_ld(N);
  const int tid = threadIdx.x, nt = blockDim.x;
  // loads issued eight at a time so that their latencies overlap
  for (int base = tid; base < N * N; base += 8 * nt) {
    double g[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * nt, r = idx % N, c = idx / N;
      g[u] = (idx < N * N && r < n && c < n) ? (r >= c ? R[c + r * ldr] : 0.0) : (r == c ? 1.0 : 0.0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * nt, r = idx % N, c = idx / N;
      if (idx >= N * N) continue;
      const float v = float(g[u]);
      if (r == c) {
        if (!(v != 0.f)) set_status(status, LR_ERR_BREAKDOWN);
        dinv[r] = 1.f / v;
      }
      L[r + c * ld] = v;
      Xt[r + c * ld] = 0.f;
    }
  }
  __syncthreads();
  chol::block_inverse(L, Xt, Xd, T, dinv, N, ld);
  for (int idx = tid; idx < n * n; idx += nt) {
    const int r = idx % n, c = idx / n;
    Xout[r + c * ldx] = Xt[r + c * ld];
  }
}

size_t smem_for(int n) {
  const int N = (n + kB - 1) / kB * kB;
  return size_t(chol::smem_floats(N)) * sizeof(float);
}

}  // namespace

void chol_inv(const double* G, int ell, float* Rinv, int ldr, double* Racc, int ldacc, bool init_acc, int mode,
              int* needs_more, int* status, cudaStream_t s) {
  LR_REQUIRE(ell >= 1 && ell <= kMaxN, LR_ERR_UNSUPPORTED, "chol_inv: block width must be <= 128");
  static std::atomic<bool> attr[64];  // attributes set, per device
  int dev = 0;
  LR_CHECK_CUDA(cudaGetDevice(&dev));
  if (!attr[dev & 63]) {
    LR_CHECK_CUDA(cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_for(kMaxN))));
    attr[dev & 63] = true;
  }
  LR_REQUIRE(init_acc, LR_ERR_INVALID_ARG, "chol_inv: Racc is written as R (init_acc)");
  chol_inv_kernel<<<1, kThreadsC, smem_for(ell), s>>>(G, ell, Rinv, ldr, Racc, ldacc, mode, needs_more, status);
  LR_LAUNCH_CHECK();
}

void tri_inv(const double* R, int ldr, int n, float* X, int ldx, int* status, cudaStream_t s) {
  LR_REQUIRE(n >= 1 && n <= kMaxN, LR_ERR_UNSUPPORTED, "tri_inv: n must be <= 128");
  static std::atomic<bool> attr[64];  // attributes set, per device
  int dev = 0;
  LR_CHECK_CUDA(cudaGetDevice(&dev));
  if (!attr[dev & 63]) {
    LR_CHECK_CUDA(cudaFuncSetAttribute(tri_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_for(kMaxN))));
    attr[dev & 63] = true;
  }
  tri_inv_kernel<<<1, kThreadsC, smem_for(n), s>>>(R, ldr, n, X, ldx, status);
  LR_LAUNCH_CHECK();
}

}  // namespace lr
