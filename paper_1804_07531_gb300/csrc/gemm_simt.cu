// FP32 SIMT GEMM for the thin products of the method: the FP32 form of the
// views (Y = A X, Z = A^T W), Grams and cross-Grams (FP32 products, FP64
// accumulation across K slices), block projections, application of R^{-1},
// the lift U = Q U^ and the backward's rank-(v ell) update of dA.
//
//   C[M x N] = alpha * op(A)[M x K] * op(B)[K x N] (+ beta * C)
//   A col-major: op(A)(i,k) = A[i + k*lda]       (TA = false)
//                op(A)(i,k) = A[k + i*lda]       (TA = true)
//   B col-major: op(B)(k,j) = B[k + j*ldb]       (TB = false)
//                op(B)(k,j) = B[j + k*ldb]       (TB = true)
//   C col-major: C[i + j*ldc]
//
// A row-major matrix A_rm (m x n, ld) is the col-major n x m matrix with the
// same ld, so Y = A_rm X uses TA = true and Z = A_rm^T W uses TA = false.
// K is split across gridDim.z; the slices are combined with atomics (FP32 or
// FP64) into a C that the caller has zeroed.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace lr {

namespace {

constexpr int BK = 16;
constexpr int NT = 256;

template <bool TA, bool TB, int BM, int BN, int MODE>
__global__ void __launch_bounds__(NT) sgemm_kernel(int M, int N, int K, int kchunk, float alpha,
                                                   const float* __restrict__ A, int64_t lda,
                                                   const float* __restrict__ B, int64_t ldb,
                                                   float beta, float* C, double* C64, int64_t ldc,
                                                   const int* run_if) {
  if (run_if && *run_if == 0) return;
  constexpr int TM = BM / 16;  // rows per thread
  constexpr int TN = BN / 16;  // cols per thread
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];

  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t i0 = int64_t(blockIdx.x) * BM;
  const int64_t j0 = int64_t(blockIdx.y) * BN;
  const int64_t kbeg = int64_t(blockIdx.z) * kchunk;
  const int64_t kend = (K < kbeg + kchunk) ? int64_t(K) : kbeg + kchunk;

  float acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = 0.f;

  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    // ---- A tile: BM x BK
#pragma unroll
    for (int r = 0; r < (BM * BK) / NT; ++r) {
      int idx = tid + r * NT;
      int ii, kk;
      if (TA) { kk = idx % BK; ii = idx / BK; } else { ii = idx % BM; kk = idx / BM; }
      int64_t gi = i0 + ii, gk = k0 + kk;
      float val = 0.f;
      if (gi < M && gk < kend) val = TA ? A[gk + gi * lda] : A[gi + gk * lda];
      As[kk][ii] = val;
    }
    // ---- B tile: BK x BN
#pragma unroll
    for (int r = 0; r < (BN * BK + NT - 1) / NT; ++r) {
      int idx = tid + r * NT;
      if (idx < BN * BK) {
        int jj, kk;
        if (TB) { jj = idx % BN; kk = idx / BN; } else { kk = idx % BK; jj = idx / BK; }
        int64_t gj = j0 + jj, gk = k0 + kk;
        float val = 0.f;
        if (gj < N && gk < kend) val = TB ? B[gj + gk * ldb] : B[gk + gj * ldb];
        Bs[kk][jj] = val;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float av[TM], bv[TN];
#pragma unroll
      for (int a = 0; a < TM; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < TN; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int a = 0; a < TM; ++a) {
    int64_t gi = i0 + ty + 16 * a;
    if (gi >= M) continue;
#pragma unroll
    for (int b = 0; b < TN; ++b) {
      int64_t gj = j0 + tx + 16 * b;
      if (gj >= N) continue;
      int64_t o = gi + gj * ldc;
      if (MODE == GEMM_STORE) {
        float v = alpha * acc[a][b];
        if (beta != 0.f) v += beta * C[o];
        C[o] = v;
      } else if (MODE == GEMM_ATOMIC_F32) {
        atomicAdd(C + o, alpha * acc[a][b]);
      } else {
        atomicAdd(C64 + o, double(alpha) * double(acc[a][b]));
      }
    }
  }
}

template <bool TA, bool TB, int BM, int BN>
void launch_t(const GemmArgs& g, cudaStream_t s) {
  int kchunk = g.K;
  int splits = 1;
  if (g.mode != GEMM_STORE && g.split_k > 1) {
    splits = g.split_k;
    kchunk = ceil_div(ceil_div(g.K, splits), BK) * BK;
    splits = ceil_div(g.K, kchunk);
  }
  dim3 grid(ceil_div(g.M, BM), ceil_div(g.N, BN), splits);
  switch (g.mode) {
    case GEMM_STORE:
      sgemm_kernel<TA, TB, BM, BN, GEMM_STORE><<<grid, NT, 0, s>>>(
          g.M, g.N, g.K, kchunk, g.alpha, g.A, g.lda, g.B, g.ldb, g.beta, g.C, g.C64, g.ldc, g.run_if);
      break;
    case GEMM_ATOMIC_F32:
      sgemm_kernel<TA, TB, BM, BN, GEMM_ATOMIC_F32><<<grid, NT, 0, s>>>(
          g.M, g.N, g.K, kchunk, g.alpha, g.A, g.lda, g.B, g.ldb, g.beta, g.C, g.C64, g.ldc, g.run_if);
      break;
    default:
      sgemm_kernel<TA, TB, BM, BN, GEMM_ATOMIC_F64><<<grid, NT, 0, s>>>(
          g.M, g.N, g.K, kchunk, g.alpha, g.A, g.lda, g.B, g.ldb, g.beta, g.C, g.C64, g.ldc, g.run_if);
      break;
  }
  LR_LAUNCH_CHECK();
}

template <bool TA, bool TB>
void launch_bn(const GemmArgs& g, cudaStream_t s) {
  if (g.N <= 32) launch_t<TA, TB, 128, 32>(g, s);
  else if (g.N <= 64) launch_t<TA, TB, 128, 64>(g, s);
  else launch_t<TA, TB, 128, 128>(g, s);
}

}  // namespace

void sgemm(const GemmArgs& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return;
  LR_REQUIRE(g.K > 0, LR_ERR_INVALID_ARG, "sgemm: empty inner dimension");
  if (g.ta) {
    if (g.tb) launch_bn<true, true>(g, s); else launch_bn<true, false>(g, s);
  } else {
    if (g.tb) launch_bn<false, true>(g, s); else launch_bn<false, false>(g, s);
  }
}

int split_for(int64_t M, int64_t N, int64_t K, int sms) {
  int64_t tiles = int64_t(ceil_div(M, 128)) * ceil_div(N, 128);
  int64_t want = (2 * sms + tiles - 1) / tiles;
  int64_t maxs = std::max<int64_t>(1, K / 256);
  return int(std::max<int64_t>(1, std::min<int64_t>(want, maxs)));
}

}  // namespace lr
