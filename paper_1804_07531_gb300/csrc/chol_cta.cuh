// Cholesky factorisation and triangular inverse of one small SPD matrix
// (order N <= 128, a multiple of 32) by one CTA in shared memory, FP32.
// These are the factorisation steps of CholeskyQR (the thin QR between the
// views of Alg. 2 / Alg. 9: G = Y^T Y = R^T R, Q = Y R^{-1}).
//
// Layout: every matrix is column-major with leading dimension ld = N + 4, so
// each column starts on a 16-byte boundary and four consecutive rows of a
// column load as one float4.
//
// Factorisation (right-looking, 32-column blocks), for block column k:
//   1. one warp factors the diagonal block in registers (lane i holds row i;
//      column j of the factor is broadcast through shared memory);
//   2. each thread of the CTA solves one row of the panel, L_kk l_i^T = a_i^T,
//      by forward substitution in registers;
//   3. the CTA applies the trailing update A_ij -= L_ik L_jk^T on 4 x 4
//      register tiles (two float4 loads feed sixteen products).
// The serial part is the 128 pivots of step 1; steps 2 and 3 take a few
// hundred cycles each.  The inverse X = L^{-1} follows: diagonal blocks by
// forward substitution (one warp per block, lane j solving for column j),
// then block row by block row X_IJ = -X_II sum_{M=J..I-1} L_IM X_MJ; it is
// kept transposed, which is R^{-1} column-major.
#pragma once
#include "common.cuh"

namespace lr {
namespace chol {

constexpr int kB = 32;
constexpr int kMaxN = 128;
constexpr int kDld = 36;  // leading dimension of the inverse's diagonal blocks

__host__ __device__ constexpr int ld_of(int N) { return N + 4; }
__host__ __device__ constexpr int t_ld(int N) { return N - kB + 4; }
// Shared-memory floats of the factorisation and inverse of order N: A and Xt
// (N x ld each), Xd (N / 32 blocks of kDld x 32), T (32 x t_ld), dinv (N),
// colbuf (64).
__host__ __device__ constexpr int smem_floats(int N) {
  return 2 * N * ld_of(N) + (N / kB) * kB * kDld + kB * t_ld(N) + N + 2 * kB;
}

// 1 / sqrt(d) and 1 / d from the hardware approximations refined by one
// Newton step (error about 1 ulp): they sit on the serial pivot chain.
__device__ __forceinline__ float rsqrt_refined(float d) {
  const float y = rsqrtf(d);
  return y * fmaf(-0.5f * d * y, y, 1.5f);
}

// v <- L^{-1} v for a 32 x 32 lower-triangular block L (column-major, ld;
// columns 16-byte aligned) whose reciprocal diagonal is dinv[0..31].
// Right-looking: once v_c is final, it updates every later entry, so the
// products of one step are independent of each other.
__device__ __forceinline__ void fwd_subst32(float (&v)[kB], const float* L, int ld, const float* dinv) {
#pragma unroll
  for (int c = 0; c < kB; ++c) {
    v[c] *= dinv[c];
    const float* col = L + c * ld;
#pragma unroll
    for (int q = (c + 1) / 4; q < kB / 4; ++q) {
      const float4 l = *reinterpret_cast<const float4*>(col + 4 * q);
      if (4 * q + 0 > c) v[4 * q + 0] = fmaf(-v[c], l.x, v[4 * q + 0]);
      if (4 * q + 1 > c) v[4 * q + 1] = fmaf(-v[c], l.y, v[4 * q + 1]);
      if (4 * q + 2 > c) v[4 * q + 2] = fmaf(-v[c], l.z, v[4 * q + 2]);
      if (4 * q + 3 > c) v[4 * q + 3] = fmaf(-v[c], l.w, v[4 * q + 3]);
    }
  }
}

// Factors the diagonal block at (k0, k0) of A (its lower part: the Schur
// complement left by the earlier block steps) in registers, lane i holding
// row i.  Writes L_kk (zeros above its diagonal) back to A and 1 / l_jj to
// dinv[k0 + j].  The pivot comes from lane j by one shuffle; column j of the
// factor is broadcast through colbuf (two halves of 32 floats used in turn,
// so one __syncwarp per pivot suffices) and read back as float4.  Returns
// false in every lane when a pivot is not positive and finite.
static __device__ __noinline__ bool warp_chol32(float* A, int ld, int k0, float* dinv, float* colbuf, int lane) {
  float a[kB];
#pragma unroll
  for (int c = 0; c < kB; ++c) a[c] = A[(k0 + lane) + (k0 + c) * ld];
  bool ok = true;
#pragma unroll
  for (int j = 0; j < kB; ++j) {
    const float d = __shfl_sync(0xffffffffu, a[j], j);
    ok = ok && (d > 0.f) && (d < INFINITY);
    const float dd = fmaxf(d, 1e-30f);
    const float inv = rsqrt_refined(dd);
    a[j] = (lane > j) ? a[j] * inv : (lane == j ? dd * inv : a[j]);
    if (lane == j) dinv[k0 + j] = inv;
    float* cb = colbuf + (j & 1) * kB;
    cb[lane] = a[j];  // column j of L (entries below the diagonal used)
    __syncwarp();
#pragma unroll
    for (int q = (j + 1) / 4; q < kB / 4; ++q) {
      const float4 l = reinterpret_cast<const float4*>(cb)[q];
      if (4 * q + 0 > j) a[4 * q + 0] = fmaf(-a[j], l.x, a[4 * q + 0]);
      if (4 * q + 1 > j) a[4 * q + 1] = fmaf(-a[j], l.y, a[4 * q + 1]);
      if (4 * q + 2 > j) a[4 * q + 2] = fmaf(-a[j], l.z, a[4 * q + 2]);
      if (4 * q + 3 > j) a[4 * q + 3] = fmaf(-a[j], l.w, a[4 * q + 3]);
    }
  }
#pragma unroll
  for (int c = 0; c < kB; ++c) A[(k0 + lane) + (k0 + c) * ld] = (c <= lane) ? a[c] : 0.f;
  return __all_sync(0xffffffffu, ok);
}

// Lower-triangular tile index t -> (ig, jg), jg <= ig, row by row.
__device__ __forceinline__ void tri_tile(int t, int& ig, int& jg) {
  int i = int((sqrtf(8.f * float(t) + 1.f) - 1.f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  while (i * (i + 1) / 2 > t) --i;
  ig = i;
  jg = t - i * (i + 1) / 2;
}

// In-place blocked Cholesky of the N x N matrix in A (lower part used;
// N a multiple of 32): A's lower triangle becomes L with G = L L^T, and
// dinv[j] = 1 / l_jj.  Entries above the diagonal are left as scratch.
// Returns true (in every thread) when a pivot is not positive and finite.
// Called by every thread of the CTA.
__device__ __forceinline__ bool block_chol(float* A, int N, int ld, float* dinv, float* colbuf, int* bad) {
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31;
  const int nb = N / kB;
  for (int k = 0; k < nb; ++k) {
    const int k0 = k * kB, k1 = k0 + kB, rows = N - k1;
    if (warp == 0) {
      const bool ok = warp_chol32(A, ld, k0, dinv, colbuf, lane);
      if (lane == 0) *bad = ok ? 0 : 1;
    }
    __syncthreads();
    if (*bad) return true;
    if (rows == 0) break;
    // panel: row i of L_ik solves L_kk l_i^T = a_i^T
    for (int r = tid; r < rows; r += nt) {
      float v[kB];
      float* row = A + (k1 + r) + k0 * ld;
#pragma unroll
      for (int c = 0; c < kB; ++c) v[c] = row[c * ld];
      fwd_subst32(v, A + k0 + k0 * ld, ld, dinv + k0);
#pragma unroll
      for (int c = 0; c < kB; ++c) row[c * ld] = v[c];
    }
    __syncthreads();
    // trailing update of the lower part on 4 x 4 tiles (a diagonal tile
    // also writes its upper half, which is scratch)
    const int g = rows / 4, ntiles = g * (g + 1) / 2;
    for (int t = tid; t < ntiles; t += nt) {
      int ig, jg;
      tri_tile(t, ig, jg);
      const int i0 = k1 + 4 * ig, j0 = k1 + 4 * jg;
      const float* Li = A + i0 + k0 * ld;
      const float* Lj = A + j0 + k0 * ld;
      float acc[4][4] = {};
#pragma unroll 8
      for (int m = 0; m < kB; ++m) {
        const float4 x = *reinterpret_cast<const float4*>(Li + m * ld);
        const float4 y = *reinterpret_cast<const float4*>(Lj + m * ld);
        const float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[u][b] = fmaf(xs[u], ys[b], acc[u][b]);
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        float4* col = reinterpret_cast<float4*>(A + i0 + (j0 + b) * ld);
        float4 v = *col;
        v.x -= acc[0][b];
        v.y -= acc[1][b];
        v.z -= acc[2][b];
        v.w -= acc[3][b];
        *col = v;
      }
    }
    __syncthreads();
  }
  return false;
}

// X = L^{-1} for the lower-triangular L in A (N x N, ld; reciprocal diagonal
// in dinv), written as Xt = X^T column-major -- which is R^{-1} for R = L^T
// -- with Xt[c + r ld] = X[r, c].  Xt must be zero on entry.  Scratch: Xd
// (the diagonal blocks of X, column-major, kDld x 32 each) and T (32 x
// (N - 32) row-major, ld t_ld(N)).  Every product below loads both of its
// operands as float4:
//   diagonal blocks: warp w, lane j solves L_ww x = e_j;
//   block row I:     T = sum_{m >= 32 J}^{32 I - 1} L[I rows, m] X[m, J cols]
//                    (X rows read from Xt), then X_IJ = -X_II T.
// Called by every thread of the CTA; ends with a barrier.
__device__ __forceinline__ void block_inverse(const float* A, float* Xt, float* Xd, float* T, const float* dinv,
                                              int N, int ld) {
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31;
  const int nb = N / kB, tld = t_ld(N);
  for (int w = warp; w < nb; w += nt / 32) {
    float v[kB];
#pragma unroll
    for (int i = 0; i < kB; ++i) v[i] = (i == lane) ? 1.f : 0.f;
    fwd_subst32(v, A + kB * w * (ld + 1), ld, dinv + kB * w);
    float* xd = Xd + w * kB * kDld;
#pragma unroll
    for (int i = 0; i < kB; ++i) {
      xd[i + lane * kDld] = v[i];
      Xt[(kB * w + lane) + (kB * w + i) * ld] = v[i];
    }
  }
  __syncthreads();
  for (int I = 1; I < nb; ++I) {
    const int i0 = I * kB;
    const int tiles = 8 * (i0 / 4);  // 4 x 4 tiles of the 32 x i0 block row
    for (int t = tid; t < tiles; t += nt) {
      const int r0 = 4 * (t % 8), c0 = 4 * (t / 8);
      float acc[4][4] = {};
      for (int m = (c0 / kB) * kB; m < i0; ++m) {
        const float4 l = *reinterpret_cast<const float4*>(A + (i0 + r0) + m * ld);
        const float4 x = *reinterpret_cast<const float4*>(Xt + c0 + m * ld);
        const float ls[4] = {l.x, l.y, l.z, l.w}, xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[u][b] = fmaf(ls[u], xs[b], acc[u][b]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        *reinterpret_cast<float4*>(T + (r0 + u) * tld + c0) = make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
    }
    __syncthreads();
    const float* xd = Xd + I * kB * kDld;
    for (int t = tid; t < tiles; t += nt) {
      const int r0 = 4 * (t % 8), c0 = 4 * (t / 8);
      float acc[4][4] = {};
      for (int m = 0; m < r0 + 4; ++m) {
        const float4 x = *reinterpret_cast<const float4*>(xd + r0 + m * kDld);
        const float4 y = *reinterpret_cast<const float4*>(T + m * tld + c0);
        const float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[u][b] = fmaf(xs[u], ys[b], acc[u][b]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        *reinterpret_cast<float4*>(Xt + c0 + (i0 + r0 + u) * ld) =
            make_float4(-acc[u][0], -acc[u][1], -acc[u][2], -acc[u][3]);
    }
    __syncthreads();
  }
}

}  // namespace chol
}  // namespace lr
