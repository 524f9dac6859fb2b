// Blocked Cholesky and triangular inverse of one small matrix (order <= 128)
// in one CTA, for the CholeskyQR passes of the thin QR (the paper's qr
// between views, Alg. 2 / Alg. 9) and for R^{-1} in the single-pass and
// row-streamed schedules.
//
// The factorisation G = L L^T (L = R^T) runs on 32 x 32 blocks.  For block
// column k:
//   A. one warp factors the diagonal block in registers (lane i holds row i;
//      column j's multipliers are broadcast through shared memory) and
//      inverts its factor L_kk by forward substitution (lane j computes
//      column j);
//   B. the whole CTA forms the panel L_ik = A_ik L_kk^{-T} for the blocks
//      below;
//   C. the whole CTA applies the trailing update A_ij -= L_ik L_jk^T.
// In B, C and the inverse's off-diagonal blocks a thread forms four entries
// of one row, so each shared-memory load of that row feeds four products.
// The off-diagonal blocks of X = L^{-1} then follow block row by block row:
// X_ij = -X_ii sum_{m=j..i-1} L_im X_mj.  About a dozen CTA barriers replace
// the one barrier per column (and per row of the inverse) of an unblocked
// factorisation, which is what bounds a matrix this small.
//
// Orders that are not a multiple of 32 are padded with an identity block,
// whose factor and inverse are the identity.
#include "common.cuh"
#include "kernels.h"

namespace lr {
namespace {

constexpr int kB = 32;        // block order
constexpr int kMaxN = 128;    // largest order served
constexpr int kThreadsC = 512;

// All matrices below are N x N, column-major with leading dimension
// ld = N + 1 (so that one-column-per-lane accesses hit distinct banks).

// Warp-level routines on one 32 x 32 block, each holding its working array
// in registers: every array index is a compile-time constant, and the
// routines are kept out of line (inlined into a runtime loop, the compiler
// would move the array to local memory).

// 1 / sqrt(d) and 1 / d from the hardware approximations refined by one
// Newton step (error ~1 ulp), instead of the longer correctly rounded
// sequences: these sit on the factorisation's serial dependency chain.
__device__ __forceinline__ float rsqrt_refined(float d) {
  const float y = rsqrtf(d);
  return y * fmaf(-0.5f * d * y, y, 1.5f);
}
__device__ __forceinline__ float rcp_refined(float d) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(d));
  return fmaf(y, fmaf(-d, y, 1.f), y);
}
// sum_m a[m * sa] * b[m * sb] for m in [m0, m1), four independent chains.
__device__ __forceinline__ float dot4(const float* a, int sa, const float* b, int sb, int m0, int m1) {
  float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
  int m = m0;
  for (; m + 3 < m1; m += 4) {
    c0 = fmaf(a[m * sa], b[m * sb], c0);
    c1 = fmaf(a[(m + 1) * sa], b[(m + 1) * sb], c1);
    c2 = fmaf(a[(m + 2) * sa], b[(m + 2) * sb], c2);
    c3 = fmaf(a[(m + 3) * sa], b[(m + 3) * sb], c3);
  }
  for (; m < m1; ++m) c0 = fmaf(a[m * sa], b[m * sb], c0);
  return (c0 + c1) + (c2 + c3);
}

// Factors the symmetric block at (k0, k0) of A (lower part used) as L L^T in
// registers -- lane i holds row i -- and writes the rows of L_kk (zeros above
// the diagonal) to L.  The pivot comes from lane j by one shuffle; column j
// of the factor is broadcast through shared memory (col, 32 floats): one
// store per lane, then independent loads, so the loads of a step overlap
// instead of serialising like a chain of warp shuffles.  Returns false in every lane on a pivot that is not positive and
// finite.
__device__ __noinline__ bool warp_factor_block(const float* A, float* L, int ld, int k0, int lane, float* col) {
  float a[kB];
#pragma unroll
  for (int c = 0; c < kB; ++c) a[c] = A[(k0 + lane) + (k0 + c) * ld];
  bool ok = true;
#pragma unroll
  for (int j = 0; j < kB; ++j) {
    // the pivot: lane j's updated diagonal entry
    const float d = __shfl_sync(0xffffffffu, a[j], j);
    ok = ok && (d > 0.f) && isfinite(d);
    const float dd = fmaxf(d, 1e-30f);
    const float inv = rsqrt_refined(dd);  // 1 / l_jj
    a[j] = (lane > j) ? a[j] * inv : (lane == j ? dd * inv : a[j]);
    col[lane] = a[j];  // column j of L (entries below the diagonal used)
    __syncwarp();
#pragma unroll
    for (int c = j + 1; c < kB; ++c) a[c] = (lane >= c) ? fmaf(-a[j], col[c], a[c]) : a[c];
    __syncwarp();
  }
#pragma unroll
  for (int c = 0; c < kB; ++c) L[(k0 + lane) + (k0 + c) * ld] = (c <= lane) ? a[c] : 0.f;
  return __all_sync(0xffffffffu, ok);
}

// X_kk = L_kk^{-1} (lower) by forward substitution, lane j computing column
// j: x_i = (delta_{i,j} - sum_{m<i} l_im x_m) / l_ii (L read by broadcast).
__device__ __noinline__ void warp_invert_block(const float* L, float* X, int ld, int k0, int lane) {
  float x[kB];
#pragma unroll
  for (int i = 0; i < kB; ++i) {
    const float* li = L + (k0 + i) + k0 * ld;  // row i of the block
    float acc0 = (i == lane) ? 1.f : 0.f, acc1 = 0.f;
#pragma unroll
    for (int m = 0; m < i; ++m) {
      if (m & 1) acc1 = fmaf(-li[m * ld], x[m], acc1);
      else acc0 = fmaf(-li[m * ld], x[m], acc0);
    }
    x[i] = (acc0 + acc1) * rcp_refined(li[i * ld]);
  }
#pragma unroll
  for (int i = 0; i < kB; ++i) X[(k0 + i) + (k0 + lane) * ld] = x[i];
}

// Blocked factorisation of the N x N matrix in A (lower part used): L and
// the diagonal blocks of X = L^{-1}.  A is overwritten by Schur
// complements.  Returns true (uniformly) on a non-positive pivot.
__device__ __forceinline__ bool block_cholesky(float* A, float* L, float* X, int N, int ld, int* bad, float* colbuf) {
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid / 32, lane = tid % 32;
  const int nb = N / kB;
  for (int k = 0; k < nb; ++k) {
    const int k0 = k * kB;
    if (warp == 0) {
      const bool ok = warp_factor_block(A, L, ld, k0, lane, colbuf);
      __syncwarp();
      warp_invert_block(L, X, ld, k0, lane);
      if (lane == 0) *bad = ok ? 0 : 1;
    }
    __syncthreads();
    if (*bad) return true;
    const int k1 = k0 + kB, rows = N - k1;
    if (rows == 0) break;
    // B. panel L_ik = A_ik X_kk^T: row r, columns c0..c0+3 of the block per
    // thread (X_kk is exactly zero above its diagonal, so the four sums can
    // share the range m <= c0 + 3)
    for (int idx = tid; idx < rows * (kB / 4); idx += nt) {
      const int r = k1 + idx % rows, c0 = (idx / rows) * 4;
      const float* ar = A + r + k0 * ld;
      const float* xc = X + (k0 + c0) + k0 * ld;
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
      for (int m = 0; m <= c0 + 3; ++m) {
        const float a = ar[m * ld];
        const float* xm = xc + m * ld;
        a0 = fmaf(a, xm[0], a0);
        a1 = fmaf(a, xm[1], a1);
        a2 = fmaf(a, xm[2], a2);
        a3 = fmaf(a, xm[3], a3);
      }
      float* lo = L + r + (k0 + c0) * ld;
      lo[0] = a0;
      lo[ld] = a1;
      lo[2 * ld] = a2;
      lo[3 * ld] = a3;
    }
    __syncthreads();
    // C. trailing update of the lower part: A_ij -= L_ik L_jk^T, row i and
    // columns j0..j0+3 per thread
    for (int idx = tid; idx < rows * (rows / 4); idx += nt) {
      const int i = k1 + idx % rows, j0 = k1 + (idx / rows) * 4;
      if (i < j0) continue;
      const float* li = L + i + k0 * ld;
      const float* lj = L + j0 + k0 * ld;
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll 8
      for (int m = 0; m < kB; ++m) {
        const float l = li[m * ld];
        const float* lm = lj + m * ld;
        a0 = fmaf(l, lm[0], a0);
        a1 = fmaf(l, lm[1], a1);
        a2 = fmaf(l, lm[2], a2);
        a3 = fmaf(l, lm[3], a3);
      }
      float* ai = A + i + j0 * ld;
      ai[0] -= a0;
      if (i >= j0 + 1) ai[ld] -= a1;
      if (i >= j0 + 2) ai[2 * ld] -= a2;
      if (i >= j0 + 3) ai[3 * ld] -= a3;
    }
    __syncthreads();
  }
  return false;
}

// Off-diagonal blocks of X = L^{-1} (diagonal blocks already in X), using T
// as scratch: block row i, for all j < i at once,
//   T_ij = sum_{m=j..i-1} L_im X_mj,  X_ij = -X_ii T_ij.
// A thread forms four columns of a row (they share the block column, so the
// same summation range): each L or X entry it loads feeds four products.
__device__ __forceinline__ void block_inverse_offdiag(const float* L, float* X, float* T, int N, int ld) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nb = N / kB;
  for (int i = 1; i < nb; ++i) {
    const int i0 = i * kB;
    for (int idx = tid; idx < kB * (i0 / 4); idx += nt) {
      const int r = idx % kB, c0 = (idx / kB) * 4;  // row i0 + r, columns c0..c0+3 < i0
      const int m0 = (c0 / kB) * kB;
      const float* lr = L + (i0 + r);
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
      for (int m = m0; m < i0; ++m) {
        const float l = lr[m * ld];
        const float* xm = X + m + c0 * ld;
        a0 = fmaf(l, xm[0], a0);
        a1 = fmaf(l, xm[ld], a1);
        a2 = fmaf(l, xm[2 * ld], a2);
        a3 = fmaf(l, xm[3 * ld], a3);
      }
      float* t = T + (i0 + r) + c0 * ld;
      t[0] = a0;
      t[ld] = a1;
      t[2 * ld] = a2;
      t[3 * ld] = a3;
    }
    __syncthreads();
    for (int idx = tid; idx < kB * (i0 / 4); idx += nt) {
      const int r = idx % kB, c0 = (idx / kB) * 4;
      const float* xr = X + (i0 + r) + i0 * ld;  // row i0 + r of X_ii
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
      for (int m = 0; m <= r; ++m) {
        const float x = xr[m * ld];
        const float* tm = T + (i0 + m) + c0 * ld;
        a0 = fmaf(x, tm[0], a0);
        a1 = fmaf(x, tm[ld], a1);
        a2 = fmaf(x, tm[2 * ld], a2);
        a3 = fmaf(x, tm[3 * ld], a3);
      }
      float* xo = X + (i0 + r) + c0 * ld;
      xo[0] = -a0;
      xo[ld] = -a1;
      xo[2 * ld] = -a2;
      xo[3 * ld] = -a3;
    }
    __syncthreads();
  }
}

// Cholesky G = R^T R (G FP64 in global memory, factorised in FP32 in shared
// memory), then Rinv = R^{-1} and Racc <- R Racc (or Racc = R when init).
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
                                                             int ldr, double* Racc, int ldacc, int init_acc, int mode,
                                                             int* needs_more, int* status) {
  const bool flagged = needs_more != nullptr && *needs_more != 0;
  if (mode == CHOL_IF_FLAGGED && !flagged) return;
  extern __shared__ float sm[];
  const int N = (n + kB - 1) / kB * kB, ld = N + 1;
  float* A = sm;
  float* L = A + N * ld;
  float* X = L + N * ld;
  __shared__ int bad, nonfinite;
  __shared__ double tr;
  __shared__ float colbuf[kB + 1];  // column broadcast of the warp factorisation
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) nonfinite = 0;
  if (tid < 32) {  // trace of G (the norm estimate for the shift)
    double t = 0.0;
    for (int i = tid; i < n; i += 32) t += G[i + i * n];
    t = warp_sum(t);
    if (tid == 0) tr = t;
  }
  __syncthreads();
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
      if (!isfinite(g[u])) nonfinite = 1;
      A[r + c * ld] = float(g[u]);
      L[r + c * ld] = 0.f;  // blocks above the diagonal are never written
      X[r + c * ld] = 0.f;
    }
  }
  __syncthreads();
  if (nonfinite) {
    if (tid == 0) set_status(status, LR_ERR_NONFINITE);
    return;
  }
  bool broke = false, shifted = false;
  const bool shift_first = mode == CHOL_SHIFT_IF_FLAGGED && flagged;
  for (int attempt = shift_first ? 1 : 0; attempt < 2; ++attempt) {
    if (attempt == 1) {
      shifted = true;
      // the shift sits above the FP32 Gram and Cholesky rounding level, so
      // the shifted factorisation cannot break down
      const float shift = float(1e-5 * tr);
      for (int idx = tid; idx < N * N; idx += nt) {
        const int r = idx % N, c = idx / N;
        A[r + c * ld] = (r < n && c < n) ? float(G[r + c * n]) + (r == c ? shift : 0.f) : (r == c ? 1.f : 0.f);
      }
      __syncthreads();
    }
    broke = block_cholesky(A, L, X, N, ld, &bad, colbuf);
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
  block_inverse_offdiag(L, X, A, N, ld);
  // R^{-1} = X^T (upper)
  for (int idx = tid; idx < n * n; idx += nt) {
    const int r = idx % n, c = idx / n;
    Rinv[r + c * ldr] = X[c + r * ld];
  }
  if (!Racc) return;
  if (init_acc) {
    for (int idx = tid; idx < n * n; idx += nt) {
      const int r = idx % n, c = idx / n;
      Racc[r + c * ldacc] = (r <= c) ? double(L[c + r * ld]) : 0.0;
    }
    return;
  }
  // Racc <- R Racc with R = L^T (both upper): FP32 copy of Racc in A first
  for (int base = tid; base < n * n; base += 4 * nt) {
    double v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = base + u * nt, r = idx % n, c = idx / n;
      v[u] = (idx < n * n && r <= c) ? Racc[r + c * ldacc] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = base + u * nt;
      if (idx < n * n) A[idx % n + (idx / n) * ld] = float(v[u]);
    }
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += nt) {
    const int r = idx % n, c = idx / n;
    Racc[r + c * ldacc] = (r <= c) ? double(dot4(L + r * ld, 1, A + c * ld, 1, r, c + 1)) : 0.0;
  }
}

// X = R^{-1} (FP32, upper) for an upper-triangular FP64 R of order n <= 128:
// with L = R^T, each warp inverts one diagonal block of L in registers, the
// off-diagonal blocks follow as above, and R^{-1} = (L^{-1})^T.
__global__ void __launch_bounds__(kThreadsC) tri_inv_kernel(const double* __restrict__ R, int ldr, int n, float* Xout,
                                                            int ldx, int* status) {
  extern __shared__ float sm[];
  const int N = (n + kB - 1) / kB * kB, ld = N + 1;
  float* L = sm;
  float* X = L + N * ld;
  float* T = X + N * ld;
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid / 32, lane = tid % 32;
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
      if (r == c && !(v != 0.f)) set_status(status, LR_ERR_BREAKDOWN);
      L[r + c * ld] = v;
      X[r + c * ld] = 0.f;  // blocks above the diagonal are never written
    }
  }
  __syncthreads();
  const int nb = N / kB;
  if (warp < nb) warp_invert_block(L, X, ld, warp * kB, lane);
  __syncthreads();
  block_inverse_offdiag(L, X, T, N, ld);
  for (int idx = tid; idx < n * n; idx += nt) {
    const int r = idx % n, c = idx / n;
    Xout[r + c * ldx] = X[c + r * ld];
  }
}

size_t smem_for(int n) {
  const int N = (n + kB - 1) / kB * kB;
  return size_t(3) * N * (N + 1) * sizeof(float);
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
  chol_inv_kernel<<<1, kThreadsC, smem_for(ell), s>>>(G, ell, Rinv, ldr, Racc, ldacc, init_acc ? 1 : 0, mode,
                                                      needs_more, status);
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
