// Small dense kernels: the ell x ell factorisations between views and
// elementwise helpers.
//
// GB300's FP64 pipe runs at about 1/60 of its FP32 rate (1.25 TFLOP/s per
// GPU), so O(ell^3) work in FP64 on one SM would cost milliseconds.  The
// Grams reach these kernels FP64-accumulated (their dominant error, the
// m-term summation, is gone); the Cholesky, the triangular inverse and the
// core SVD then run in FP32 inside one CTA with the matrix in shared memory.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace lr {

namespace {

__global__ void f32_to_bf16_kernel(const float* __restrict__ src, int64_t lds, __nv_bfloat16* __restrict__ dst,
                                   __nv_bfloat16* __restrict__ lo, int64_t ldd, int64_t rows, int64_t cols) {
  for (int64_t c = blockIdx.y; c < cols; c += gridDim.y)
    for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < rows; r += int64_t(gridDim.x) * blockDim.x) {
      const float x = src[r + c * lds];
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      dst[r + c * ldd] = h;
      if (lo) lo[r + c * ldd] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
}

__global__ void copy_kernel(const float* __restrict__ src, int64_t lds, float* __restrict__ dst, int64_t ldd,
                            int64_t rows, int64_t cols, const int* run_if) {
  if (run_if && *run_if == 0) return;
  for (int64_t c = blockIdx.y; c < cols; c += gridDim.y)
    for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < rows; r += int64_t(gridDim.x) * blockDim.x) {
      dst[r + c * ldd] = src[r + c * lds];
    }
}

// One block per column i: find the entry of U(:, i) with the largest
// magnitude (lowest index on ties) and flip (u_i, v_i) if it is negative.
// 1024 threads and float4 loads (when the column is 16-byte aligned) keep
// enough loads in flight for a column of 64k rows.
__device__ __forceinline__ void take_max(float a, int64_t r, float& best, int64_t& bidx) {
  if (a > best) {  // rows are visited in increasing order: the first maximum stays
    best = a;
    bidx = r;
  }
}
// The row of the largest-magnitude entry of u (m entries; lowest row on
// ties; 0 when m == 0).  Called by every thread of the block.
__device__ int64_t col_absmax_row(const float* u, int64_t m) {
  float best = -1.f;
  int64_t bidx = 0;
  const bool vec = (reinterpret_cast<uintptr_t>(u) & 15) == 0;
  const int64_t m4 = vec ? m / 4 : 0;
  const float4* u4 = reinterpret_cast<const float4*>(u);
#pragma unroll 4
  for (int64_t q = threadIdx.x; q < m4; q += blockDim.x) {
    const float4 x = u4[q];
    take_max(fabsf(x.x), 4 * q, best, bidx);
    take_max(fabsf(x.y), 4 * q + 1, best, bidx);
    take_max(fabsf(x.z), 4 * q + 2, best, bidx);
    take_max(fabsf(x.w), 4 * q + 3, best, bidx);
  }
  for (int64_t r = 4 * m4 + threadIdx.x; r < m; r += blockDim.x) take_max(fabsf(u[r]), r, best, bidx);
  __shared__ float sb[32];
  __shared__ int64_t si[32];
  for (int o = 16; o > 0; o >>= 1) {
    float ob = __shfl_xor_sync(0xffffffffu, best, o);
    int64_t oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
  }
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) { sb[w] = best; si[w] = bidx; }
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x / 32;
    best = l < nw ? sb[l] : -1.f;
    bidx = l < nw ? si[l] : 0;
    for (int o = 16; o > 0; o >>= 1) {
      float ob = __shfl_xor_sync(0xffffffffu, best, o);
      int64_t oi = __shfl_xor_sync(0xffffffffu, bidx, o);
      if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
    }
    if (l == 0) si[0] = bidx;
  }
  __syncthreads();
  const int64_t r = si[0];
  __syncthreads();  // si is reused by the next call
  return r;
}

__device__ void negate_pair(float* u, int64_t m, float* v, int64_t n) {
  const bool vec = (reinterpret_cast<uintptr_t>(u) & 15) == 0;
  const int64_t m4 = vec ? m / 4 : 0;
  float4* w4 = reinterpret_cast<float4*>(u);
  for (int64_t q = threadIdx.x; q < m4; q += blockDim.x) {
    const float4 x = w4[q];
    w4[q] = make_float4(-x.x, -x.y, -x.z, -x.w);
  }
  for (int64_t r = 4 * m4 + threadIdx.x; r < m; r += blockDim.x) u[r] = -u[r];
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) v[r] = -v[r];
}

__global__ void __launch_bounds__(1024) fix_signs_kernel(float* U, int64_t ldu, int64_t m, float* V, int64_t ldv,
                                                         int64_t n) {
  const int col = blockIdx.x;
  float* u = U + col * ldu;
  const int64_t r = col_absmax_row(u, m);
  if (u[r] < 0.f) negate_pair(u, m, V + col * ldv, n);
}

// Rows of U split over ranks: rank `slot` writes the signed peak entry of
// each of its columns to peaks[slot * k + col] (the caller zeroes the
// buffer; a sum over the ranks then holds every rank's peak).
__global__ void __launch_bounds__(1024) col_peak_kernel(const float* U, int64_t ldu, int64_t m, float* peaks,
                                                        int slot, int k) {
  const int col = blockIdx.x;
  const float* u = U + col * ldu;
  const int64_t r = col_absmax_row(u, m);
  if (threadIdx.x == 0) peaks[int64_t(slot) * k + col] = m > 0 ? u[r] : 0.f;
}

// The global peak of column col is the largest |peaks[g * k + col]| (the
// lowest rank on ties, i.e. the lowest global row); (u_col, v_col) flips
// when it is negative.
__global__ void __launch_bounds__(1024) flip_by_peak_kernel(float* U, int64_t ldu, int64_t m, float* V,
                                                            int64_t ldv, int64_t n, const float* peaks, int world,
                                                            int k) {
  const int col = blockIdx.x;
  float best = -1.f, val = 0.f;
  for (int g = 0; g < world; ++g) {
    const float x = peaks[int64_t(g) * k + col];
    if (fabsf(x) > best) { best = fabsf(x); val = x; }
  }
  if (val < 0.f) negate_pair(U + col * ldu, m, V + col * ldv, n);
}

// Upper-triangular inverse of R (n x n, column-major FP32 in smem, lda n):
__global__ void add_block_kernel(double* R, int ldr, int r0, int c0, const double* C, int ldc, int rows, int cols) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < rows * cols; idx += gridDim.x * blockDim.x) {
    const int r = idx % rows, c = idx / rows;
    R[(r0 + r) + int64_t(c0 + c) * ldr] += C[r + int64_t(c) * ldc];
  }
}

__global__ void f64_to_f32_kernel(const double* src, int lds, float* dst, int ldd, int rows, int cols) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < rows * cols; idx += gridDim.x * blockDim.x) {
    const int r = idx % rows, c = idx / rows;
    dst[r + int64_t(c) * ldd] = float(src[r + int64_t(c) * lds]);
  }
}

__global__ void r_to_f32_kernel(const double* R, int ldr, int n, float* out, int ldo, int trans) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * n; idx += gridDim.x * blockDim.x) {
    const int r = idx % n, c = idx / n;
    const double v = (r <= c) ? R[r + int64_t(c) * ldr] : 0.0;
    if (trans) out[c + int64_t(r) * ldo] = float(v);
    else out[r + int64_t(c) * ldo] = float(v);
  }
}

__global__ void scale_cols_kernel(float* A, int64_t lda, int64_t rows, int cols, const float* scale) {
  for (int64_t c = blockIdx.y; c < cols; c += gridDim.y)
    for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < rows; r += int64_t(gridDim.x) * blockDim.x) {
      A[r + c * lda] *= scale[c];
    }
}

// --------------------------------------------------------- Jacobi SVD
// One-sided (Hestenes) Jacobi in one CTA.  W (rows x cols) starts as M and
// V as the identity; each round of the circle-method ordering rotates
// disjoint column pairs (one warp per pair) until a sweep makes no rotation:
//   alpha = |w_p|^2, beta = |w_q|^2, gamma = w_p . w_q,
//   rotate when |gamma| > tol sqrt(alpha beta),
//   zeta = (beta - alpha) / (2 gamma), t = sign(zeta)/(|zeta| + sqrt(1+zeta^2)),
//   c = 1/sqrt(1+t^2), s = c t, [w_p, w_q] <- [c w_p - s w_q, s w_p + c w_q].
// Then s_i = |w_i|, u_i = w_i / s_i, sorted descending.  W and V live in
// shared memory when they fit, else in the global buffers.
template <bool SMEM>
__global__ void __launch_bounds__(1024) jacobi_kernel(const float* __restrict__ M, int ldm, int rows, int cols,
                                                      float* Wg, int ldw, float* Vg, int ldv, float* S, double* S64,
                                                      int* status) {
  extern __shared__ float sm[];
  float* W = SMEM ? sm : Wg;
  const int ldW = SMEM ? rows : ldw;
  float* V = SMEM ? sm + rows * cols : Vg;
  const int ldV = SMEM ? cols : ldv;
  __shared__ int rotated;
  __shared__ float norms[1024];
  __shared__ int order[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid / 32, lane = tid % 32, nwarps = nt / 32;
  for (int idx = tid; idx < rows * cols; idx += nt) {
    const int r = idx % rows, c = idx / rows;
    W[r + c * ldW] = M[r + int64_t(c) * ldm];
  }
  for (int idx = tid; idx < cols * cols; idx += nt) {
    const int r = idx % cols, c = idx / cols;
    V[r + c * ldV] = (r == c) ? 1.f : 0.f;
  }
  __syncthreads();
  const float tol = 1.2e-7f * sqrtf(float(rows));
  const int np = cols + (cols & 1);  // even number of positions
  const int npairs = np / 2;
  int sweep = 0;
  for (; sweep < 40; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      for (int pi = warp; pi < npairs; pi += nwarps) {
        // circle method: s_0 = 0, s_k = 1 + (k - 1 + rnd) mod (np - 1)
        int a = (pi == 0) ? 0 : 1 + (pi - 1 + rnd) % (np - 1);
        int b = 1 + (np - 2 - pi + rnd) % (np - 1);
        int p = min(a, b), q = max(a, b);
        if (q >= cols) continue;
        float* wp = W + p * ldW;
        float* wq = W + q * ldW;
        float al = 0.f, be = 0.f, ga = 0.f;
        for (int r = lane; r < rows; r += 32) {
          const float x = wp[r], y = wq[r];
          al = fmaf(x, x, al);
          be = fmaf(y, y, be);
          ga = fmaf(x, y, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (al > 0.f && be > 0.f && fabsf(ga) > tol * sqrtf(al) * sqrtf(be)) {
          const float zeta = (be - al) / (2.f * ga);
          const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          // correctly rounded sqrt and division keep c^2 + s^2 = 1 to an
          // unbiased half ulp, so V drifts from orthogonality only as a
          // random walk over the rotations
          const float c = 1.f / sqrtf(1.f + t * t);
          const float s = c * t;
          for (int r = lane; r < rows; r += 32) {
            const float x = wp[r], y = wq[r];
            wp[r] = c * x - s * y;
            wq[r] = s * x + c * y;
          }
          float* vp = V + p * ldV;
          float* vq = V + q * ldV;
          for (int r = lane; r < cols; r += 32) {
            const float x = vp[r], y = vq[r];
            vp[r] = c * x - s * y;
            vq[r] = s * x + c * y;
          }
          if (lane == 0) rotated = 1;
        }
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  if (sweep == 40 && tid == 0) set_status(status, LR_ERR_NONFINITE);
  // Columns of V are unit vectors in exact arithmetic; remove the norm drift
  // accumulated over the rotations.
  for (int c = warp; c < cols; c += nwarps) {
    float acc = 0.f;
    for (int r = lane; r < cols; r += 32) acc = fmaf(V[r + c * ldV], V[r + c * ldV], acc);
    acc = warp_sum(acc);
    const float inv = 1.f / sqrtf(acc);
    for (int r = lane; r < cols; r += 32) V[r + c * ldV] *= inv;
  }
  __syncthreads();
  // norms and descending order (stable: ties keep the lower index first)
  for (int c = warp; c < cols; c += nwarps) {
    float acc = 0.f;
    for (int r = lane; r < rows; r += 32) acc = fmaf(W[r + c * ldW], W[r + c * ldW], acc);
    acc = warp_sum(acc);
    if (lane == 0) norms[c] = sqrtf(acc);
  }
  __syncthreads();
  for (int c = tid; c < cols; c += nt) {
    int rank = 0;
    const float v = norms[c];
    for (int d = 0; d < cols; ++d) {
      const float o = norms[d];
      rank += (o > v) || (o == v && d < c);
    }
    order[rank] = c;
  }
  __syncthreads();
  // Outputs: S, U into Wg (normalised, permuted), V into Vg (permuted).
  // In the smem case the global buffers are free to write directly.  In the
  // global case W/V alias the outputs, so the permutation goes through a
  // column at a time with a barrier.
  if (SMEM) {
    for (int idx = tid; idx < rows * cols; idx += nt) {
      const int r = idx % rows, j = idx / rows;
      const int c = order[j];
      const float nv = norms[c];
      Wg[r + int64_t(j) * ldw] = nv > 0.f ? W[r + c * ldW] / nv : 0.f;
    }
    for (int idx = tid; idx < cols * cols; idx += nt) {
      const int r = idx % cols, j = idx / cols;
      Vg[r + int64_t(j) * ldv] = V[r + order[j] * ldV];
    }
  } else {
    // normalise in place, then permute by cycles using one column of scratch
    // per step (done serially over columns; cols is small).
    for (int idx = tid; idx < rows * cols; idx += nt) {
      const int r = idx % rows, c = idx / rows;
      const float nv = norms[c];
      W[r + c * ldW] = nv > 0.f ? W[r + c * ldW] / nv : 0.f;
    }
    __syncthreads();
    __shared__ int done[1024];
    for (int c = tid; c < cols; c += nt) done[c] = 0;
    __syncthreads();
    for (int j = 0; j < cols; ++j) {
      if (done[j] || order[j] == j) continue;
      // cycle starting at j: dst j <- src order[j] <- ...
      float tw = 0.f;  // each thread carries one element per row/col slot
      // save column j of W and V
      float savew[8], savev[8];
      int cnt = 0;
      for (int r = tid; r < rows; r += nt) savew[cnt++] = W[r + j * ldW];
      cnt = 0;
      for (int r = tid; r < cols; r += nt) savev[cnt++] = V[r + j * ldV];
      __syncthreads();
      int d = j;
      while (true) {
        const int src = order[d];
        if (src == j) break;
        for (int r = tid; r < rows; r += nt) W[r + d * ldW] = W[r + src * ldW];
        for (int r = tid; r < cols; r += nt) V[r + d * ldV] = V[r + src * ldV];
        __syncthreads();
        if (tid == 0) done[d] = 1;
        d = src;
      }
      cnt = 0;
      for (int r = tid; r < rows; r += nt) W[r + d * ldW] = savew[cnt++];
      cnt = 0;
      for (int r = tid; r < cols; r += nt) V[r + d * ldV] = savev[cnt++];
      if (tid == 0) done[d] = 1;
      __syncthreads();
      (void)tw;
    }
  }
  for (int j = tid; j < cols; j += nt) {
    S[j] = norms[order[j]];
    if (S64) S64[j] = double(norms[order[j]]);
  }
}

// M (n x n FP32) <- copyltu(M - C) with C FP64 (may be null):
// out(i,j) = in(max(i,j), min(i,j)), the symmetric matrix built from the
// lower triangle (used by the thin-QR reverse rule).
__global__ void qr_bwd_sym_kernel(const float* M, const double* C, int n, float* out) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * n; idx += gridDim.x * blockDim.x) {
    const int i = idx % n, j = idx / n;
    const int r = max(i, j), c = min(i, j);
    float v = M[r + c * n];
    if (C) v -= float(C[r + c * n]);
    out[idx] = v;
  }
}

inline int grid_for(int64_t total) { return int(std::min<int64_t>(4096, std::max<int64_t>(1, (total + 255) / 256))); }

// Racc <- R2 Racc for upper-triangular n x n FP64 factors (Racc ld ldr,
// R2 ld ld2): CTA c owns column c of Racc, staged in shared memory so the
// column can be overwritten in place.  A no-op when *run_if == 0.
__global__ void upper_product_kernel(const double* __restrict__ R2, int ld2, double* Racc, int ldr, int n,
                                     const int* run_if) {
  if (run_if && *run_if == 0) return;
  extern __shared__ double colc[];
  const int c = blockIdx.x;
  for (int m = threadIdx.x; m <= c; m += blockDim.x) colc[m] = Racc[m + int64_t(c) * ldr];
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    double acc = 0.0;
    if (r <= c)
      for (int m = r; m <= c; ++m) acc = fma(R2[r + int64_t(m) * ld2], colc[m], acc);
    Racc[r + int64_t(c) * ldr] = acc;
  }
}

// The minimum-variance choice of Section 6.6 from the trial spectra
// lam[l_c * k + i] (l_c = 0 .. nl - 1): for 0 <= l_c < nl - 1 the vector
// s(l_c) = [lam(l_c - 1) / lam(l_c), 1, lam(l_c + 1) / lam(l_c)] (the first
// block absent for l_c = 0); *sel = argmin of its population variance
// (ties: the smaller l_c).  One thread per trial, then a serial argmin.
__global__ void minvar_select_kernel(const float* lam, int nl, int k, int* sel) {
  extern __shared__ double var[];
  for (int lc = threadIdx.x; lc < nl - 1; lc += blockDim.x) {
    const float* cur = lam + size_t(lc) * k;
    double sum = 0.0, sq = 0.0;
    int cnt = 0;
    for (int blk = (lc == 0 ? 1 : 0); blk < 3; ++blk) {
      const float* other = lam + size_t(lc + blk - 1) * k;
      for (int i = 0; i < k; ++i) {
        const double r = double(other[i]) / double(cur[i]);
        sum += r;
        sq += r * r;
        ++cnt;
      }
    }
    const double mean = sum / cnt;
    var[lc] = sq / cnt - mean * mean;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int best = 0;
    for (int lc = 1; lc < nl - 1; ++lc)
      if (var[lc] < var[best]) best = lc;
    *sel = best;
  }
}

}  // namespace

void minvar_select(const float* lam, int nl, int k, int* sel, cudaStream_t s) {
  LR_REQUIRE(nl >= 2 && k >= 1, LR_ERR_INVALID_ARG, "minimum-variance selection needs l_1 >= 1");
  minvar_select_kernel<<<1, 256, size_t(nl) * sizeof(double), s>>>(lam, nl, k, sel);
  LR_LAUNCH_CHECK();
}

void upper_product(const double* R2, int ld2, double* Racc, int ldr, int n, const int* run_if, cudaStream_t s) {
  if (n <= 0) return;
  upper_product_kernel<<<n, 128, size_t(n) * sizeof(double), s>>>(R2, ld2, Racc, ldr, n, run_if);
  LR_LAUNCH_CHECK();
}

__global__ void zero_if_kernel(float* __restrict__ p, int64_t ld, int64_t rows, int64_t cols, const int* run_if) {
  if (*run_if == 0) return;
  for (int64_t c = blockIdx.y; c < cols; c += gridDim.y)
    for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < rows; r += int64_t(gridDim.x) * blockDim.x)
      p[r + c * ld] = 0.f;
}

void zero_f32(float* p, int64_t rows, int64_t cols, int64_t ld, cudaStream_t s, const int* run_if) {
  if (rows <= 0 || cols <= 0) return;
  if (run_if) {
    zero_if_kernel<<<grid_2d(rows, cols), 256, 0, s>>>(p, ld, rows, cols, run_if);
    LR_LAUNCH_CHECK();
    return;
  }
  if (ld == rows) {
    LR_CHECK_CUDA(cudaMemsetAsync(p, 0, size_t(rows) * cols * sizeof(float), s));
  } else {
    LR_CHECK_CUDA(cudaMemset2DAsync(p, size_t(ld) * sizeof(float), 0, size_t(rows) * sizeof(float), size_t(cols), s));
  }
}

// ---- small helpers of the normal-matrix TEVDs (Alg. 4)
__global__ void sumsq_kernel(const float* __restrict__ Y, int64_t ld, int64_t rows, int64_t cols, double* out) {
  double acc = 0.0;
  for (int64_t c = blockIdx.y; c < cols; c += gridDim.y)
    for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < rows; r += int64_t(gridDim.x) * blockDim.x) {
      const double y = Y[r + c * ld];
      acc += y * y;
    }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}
// Y += nu Q with nu = scale * sqrt(*sumsq)
__global__ void shift_add_kernel(float* __restrict__ Y, int64_t ldy, const float* __restrict__ Q, int64_t ldq,
                                 int64_t rows, int64_t cols, const double* sumsq, float scale) {
  const float nu = float(scale * sqrt(*sumsq));
  for (int64_t c = blockIdx.y; c < cols; c += gridDim.y)
    for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < rows; r += int64_t(gridDim.x) * blockDim.x)
      Y[r + c * ldy] = fmaf(nu, Q[r + c * ldq], Y[r + c * ldy]);
}
__global__ void sym_f64_kernel(double* B, int n) {
  const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (idx >= int64_t(n) * n) return;
  const int i = int(idx % n), j = int(idx / n);
  if (i < j) {
    const double m = 0.5 * (B[i + int64_t(j) * n] + B[j + int64_t(i) * n]);
    B[i + int64_t(j) * n] = m;
    B[j + int64_t(i) * n] = m;
  }
}
// out_i = max(S_i^2 - nu, 0) with nu = scale * sqrt(*sumsq) (or S_i^2 when sumsq is null)
__global__ void sq_shift_kernel(const float* S, int k, const double* sumsq, float scale, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  const float nu = sumsq ? float(scale * sqrt(*sumsq)) : 0.f;
  out[i] = fmaxf(S[i] * S[i] - nu, 0.f);
}

void sumsq_f32(const float* Y, int64_t ld, int64_t rows, int64_t cols, double* out, cudaStream_t s) {
  LR_CHECK_CUDA(cudaMemsetAsync(out, 0, sizeof(double), s));
  if (rows <= 0 || cols <= 0) return;
  sumsq_kernel<<<grid_2d(rows, cols), 256, 0, s>>>(Y, ld, rows, cols, out);
  LR_LAUNCH_CHECK();
}
void shift_add_f32(float* Y, int64_t ldy, const float* Q, int64_t ldq, int64_t rows, int64_t cols, const double* sumsq,
                   float scale, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  shift_add_kernel<<<grid_2d(rows, cols), 256, 0, s>>>(Y, ldy, Q, ldq, rows, cols, sumsq, scale);
  LR_LAUNCH_CHECK();
}
void symmetrize_f64(double* B, int n, cudaStream_t s) {
  sym_f64_kernel<<<grid_for(int64_t(n) * n), 256, 0, s>>>(B, n);
  LR_LAUNCH_CHECK();
}
void sq_shift(const float* S, int k, const double* sumsq, float scale, float* out, cudaStream_t s) {
  sq_shift_kernel<<<(k + 127) / 128, 128, 0, s>>>(S, k, sumsq, scale, out);
  LR_LAUNCH_CHECK();
}

// Phi = D F P (n x s, column-major): Phi[j, t] = signs[j] c_k sqrt(2 / n)
// cos(pi (2j + 1) k / (2n)) with k = cols[t] (c_0 = 1 / sqrt(2), else 1).  The
// phase (2j + 1) k is reduced modulo 4n in integers, so cospif sees an
// argument below 2 whatever n and k are.
__global__ void srft_kernel(int64_t n, int s, const float* __restrict__ signs, const int* __restrict__ cols,
                            float* __restrict__ phi, int64_t ld) {
  const float base = sqrtf(2.f / float(n));
  for (int t = blockIdx.y; t < s; t += gridDim.y) {
    const int64_t k = cols[t];
    const float scale = k == 0 ? base * 0.70710678118654752f : base;
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x) {
      const int64_t ph = ((2 * j + 1) * k) % (4 * n);
      phi[j + int64_t(t) * ld] = signs[j] * scale * cospif(float(ph) / float(2 * n));
    }
  }
}

void srft(int64_t n, int s, const float* signs, const int* cols, float* phi, int64_t ld, cudaStream_t st) {
  if (n <= 0 || s <= 0) return;
  srft_kernel<<<grid_2d(n, s), 256, 0, st>>>(n, s, signs, cols, phi, ld);
  LR_LAUNCH_CHECK();
}

// Reverse of a square SVD R = W diag(s) Z^T (full, distinct s) for
// gradients on the k kept pairs: with Xw = W^T Wb and Xz = Z^T Zb (ell x k,
// the columns past k of Wb, Zb being zero), the middle factor of
// Rb = W inner Z^T is inner_ij = F_ij ((Xw_ij - Xw_ji) s_j + s_i (Xz_ij - Xz_ji))
// for i != j, F_ij = 1 / (s_j^2 - s_i^2) (0 where the two coincide), and
// inner_ii = dS_i (i < k).
__global__ void svd_bwd_inner_kernel(int ell, int k, const float* __restrict__ S, const float* __restrict__ dS,
                                     const float* __restrict__ Xw, const float* __restrict__ Xz, float* inner) {
  const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (idx >= int64_t(ell) * ell) return;
  const int i = int(idx % ell), j = int(idx / ell);
  float v = 0.f;
  if (i == j) {
    v = (dS && i < k) ? dS[i] : 0.f;
  } else {
    const float xw_ij = (Xw && j < k) ? Xw[i + int64_t(j) * ell] : 0.f;
    const float xw_ji = (Xw && i < k) ? Xw[j + int64_t(i) * ell] : 0.f;
    const float xz_ij = (Xz && j < k) ? Xz[i + int64_t(j) * ell] : 0.f;
    const float xz_ji = (Xz && i < k) ? Xz[j + int64_t(i) * ell] : 0.f;
    const float si = S[i], sj = S[j];
    const float d = sj * sj - si * si;
    const float f = fabsf(d) > 1e-30f ? 1.f / d : 0.f;
    v = f * ((xw_ij - xw_ji) * sj + si * (xz_ij - xz_ji));
  }
  inner[idx] = v;
}
__global__ void add_f32_kernel(float* __restrict__ Y, int64_t ldy, const float* __restrict__ X, int64_t ldx,
                               int64_t rows, int64_t cols) {
  for (int64_t c = blockIdx.y; c < cols; c += gridDim.y)
    for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < rows; r += int64_t(gridDim.x) * blockDim.x)
      Y[r + c * ldy] += X[r + c * ldx];
}

void svd_bwd_inner(int ell, int k, const float* S, const float* dS, const float* Xw, const float* Xz, float* inner,
                   cudaStream_t s) {
  svd_bwd_inner_kernel<<<grid_for(int64_t(ell) * ell), 256, 0, s>>>(ell, k, S, dS, Xw, Xz, inner);
  LR_LAUNCH_CHECK();
}
void add_f32(float* Y, int64_t ldy, const float* X, int64_t ldx, int64_t rows, int64_t cols, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  add_f32_kernel<<<grid_2d(rows, cols), 256, 0, s>>>(Y, ldy, X, ldx, rows, cols);
  LR_LAUNCH_CHECK();
}

void zero_bytes(void* p, size_t bytes, cudaStream_t s) {
  if (bytes) LR_CHECK_CUDA(cudaMemsetAsync(p, 0, bytes, s));
}

void f32_to_bf16(const float* src, int64_t lds, __nv_bfloat16* dst, __nv_bfloat16* lo, int64_t ldd, int64_t rows,
                 int64_t cols, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  f32_to_bf16_kernel<<<grid_2d(rows, cols), 256, 0, s>>>(src, lds, dst, lo, ldd, rows, cols);
  LR_LAUNCH_CHECK();
}

void copy_f32(const float* src, int64_t lds, float* dst, int64_t ldd, int64_t rows, int64_t cols, cudaStream_t s,
              const int* run_if) {
  if (rows <= 0 || cols <= 0) return;
  copy_kernel<<<grid_2d(rows, cols), 256, 0, s>>>(src, lds, dst, ldd, rows, cols, run_if);
  LR_LAUNCH_CHECK();
}

void fix_signs(float* U, int64_t ldu, int64_t m, float* V, int64_t ldv, int64_t n, int k, cudaStream_t s) {
  if (k <= 0) return;
  fix_signs_kernel<<<k, 1024, 0, s>>>(U, ldu, m, V, ldv, n);
  LR_LAUNCH_CHECK();
}

void col_peaks(const float* U, int64_t ldu, int64_t m, float* peaks, int slot, int k, cudaStream_t s) {
  if (k <= 0) return;
  col_peak_kernel<<<k, 1024, 0, s>>>(U, ldu, m, peaks, slot, k);
  LR_LAUNCH_CHECK();
}

void flip_by_peaks(float* U, int64_t ldu, int64_t m, float* V, int64_t ldv, int64_t n, const float* peaks,
                   int world, int k, cudaStream_t s) {
  if (k <= 0) return;
  flip_by_peak_kernel<<<k, 1024, 0, s>>>(U, ldu, m, V, ldv, n, peaks, world, k);
  LR_LAUNCH_CHECK();
}

void add_block_f64(double* R, int ldr, int r0, int c0, const double* C, int ldc, int rows, int cols, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  add_block_kernel<<<grid_for(int64_t(rows) * cols), 256, 0, s>>>(R, ldr, r0, c0, C, ldc, rows, cols);
  LR_LAUNCH_CHECK();
}

void f64_to_f32(const double* src, int lds, float* dst, int ldd, int rows, int cols, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  f64_to_f32_kernel<<<grid_for(int64_t(rows) * cols), 256, 0, s>>>(src, lds, dst, ldd, rows, cols);
  LR_LAUNCH_CHECK();
}

void r_to_f32(const double* R, int ldr, int n, float* out, int ldo, bool trans, cudaStream_t s) {
  r_to_f32_kernel<<<grid_for(int64_t(n) * n), 256, 0, s>>>(R, ldr, n, out, ldo, trans ? 1 : 0);
  LR_LAUNCH_CHECK();
}

void qr_bwd_sym(const float* M, const double* C, int n, float* out, cudaStream_t s) {
  qr_bwd_sym_kernel<<<grid_for(int64_t(n) * n), 256, 0, s>>>(M, C, n, out);
  LR_LAUNCH_CHECK();
}

void scale_cols_f32(float* A, int64_t lda, int64_t rows, int cols, const float* scale, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  scale_cols_kernel<<<grid_2d(rows, cols), 256, 0, s>>>(A, lda, rows, cols, scale);
  LR_LAUNCH_CHECK();
}

void jacobi_svd(float* M, int ldm, int rows, int cols, float* Wk, int ldw, float* V, int ldv, float* S,
                double* S64, int* status, cudaStream_t s) {
  LR_REQUIRE(rows >= cols && cols >= 1 && cols <= 1024, LR_ERR_UNSUPPORTED, "jacobi_svd: need rows >= cols, cols <= 1024");
  const size_t need = (size_t(rows) * cols + size_t(cols) * cols) * sizeof(float);
  int dev = 0;
  LR_CHECK_CUDA(cudaGetDevice(&dev));
  const size_t cap = size_t(dev_info(dev).max_smem_optin) - 16 * 1024;
  // square cores: column blocks over a cluster (2P - 1 exchanges per sweep);
  // wider ones: rows split over a cluster
  if (rows == cols && S64 == nullptr && jacobi_block_size(cols) > 0) {
    jacobi_svd_block(M, ldm, cols, Wk, ldw, V, ldv, S, status, s);
    return;
  }
  if (rows == cols && S64 == nullptr && jacobi_cluster_size(cols) > 0) {
    jacobi_svd_cluster(M, ldm, cols, Wk, ldw, V, ldv, S, status, s);
    return;
  }
  if (need <= cap) {
    static std::atomic<bool> attr[64];  // attributes set, per device
    if (!attr[dev & 63]) {
      LR_CHECK_CUDA(cudaFuncSetAttribute(jacobi_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(cap)));
      attr[dev & 63] = true;
    }
    jacobi_kernel<true><<<1, 1024, need, s>>>(M, ldm, rows, cols, Wk, ldw, V, ldv, S, S64, status);
  } else {
    LR_REQUIRE(rows <= 8 * 1024 && cols <= 8 * 1024, LR_ERR_UNSUPPORTED, "jacobi_svd: too large");
    jacobi_kernel<false><<<1, 1024, 0, s>>>(M, ldm, rows, cols, Wk, ldw, V, ldv, S, S64, status);
  }
  LR_LAUNCH_CHECK();
}

DevInfo dev_info(int device) {
  // filled once per device; concurrent first calls both query and store the same values
  static std::atomic<int> sms[64], smem[64];
  DevInfo d;
  d.sms = sms[device & 63].load();
  d.max_smem_optin = smem[device & 63].load();
  if (d.sms == 0 || d.max_smem_optin == 0) {
    LR_CHECK_CUDA(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, device));
    LR_CHECK_CUDA(cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    smem[device & 63].store(d.max_smem_optin);
    sms[device & 63].store(d.sms);
  }
  return d;
}

}  // namespace lr
