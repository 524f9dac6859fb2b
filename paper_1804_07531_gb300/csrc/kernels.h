// Internal launchers of liblowrank (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lr {

// ------------------------------------------------------------ SIMT GEMM
enum GemmMode { GEMM_STORE = 0, GEMM_ATOMIC_F32 = 1, GEMM_ATOMIC_F64 = 2 };
struct GemmArgs {
  int64_t M = 0, N = 0, K = 0;
  bool ta = false, tb = false;
  float alpha = 1.f, beta = 0.f;
  const float* A = nullptr;
  int64_t lda = 0;
  const float* B = nullptr;
  int64_t ldb = 0;
  float* C = nullptr;
  double* C64 = nullptr;
  int64_t ldc = 0;
  int mode = GEMM_STORE;
  int split_k = 1;
  const int* run_if = nullptr;  // device flag: the launch is a no-op when *run_if == 0
};
void sgemm(const GemmArgs& g, cudaStream_t s);
int split_for(int64_t M, int64_t N, int64_t K, int sms);

// ------------------------------------------------------- tensor-core views
struct ViewBf16Args {
  int device = 0;
  int mode = 0;  // 0: out[row0 + i] += A[row0 + i, :] B ; 1: out += A[band]^T B[band]
  const __nv_bfloat16* A = nullptr;
  int64_t lda = 0, row0 = 0, rows = 0, n = 0;
  const __nv_bfloat16* B = nullptr;  // col-major thin operand: n x ell (mode 0) or the band's rows x ell (mode 1)
  int64_t ldb = 0;
  int ell = 0;
  float* out = nullptr;  // col-major FP32, pre-zeroed (partials are added)
  int64_t ldo = 0;
  int* status = nullptr;
};
void view_bf16(const ViewBf16Args& a, cudaStream_t s);

// Y = A X and Z = A^T W from one pass over a BF16 A (each staged tile of A
// feeds both products); Y and Z are zeroed by the caller and receive FP32
// sums.  X (n x ell1) and W (m x ell2) are BF16 column-major.
struct DualBf16Args {
  int device = 0;
  const __nv_bfloat16* A = nullptr;
  int64_t lda = 0, m = 0, n = 0;
  const __nv_bfloat16* X = nullptr;
  int64_t ldx = 0;
  int ell1 = 0;
  const __nv_bfloat16* W = nullptr;
  int64_t ldw = 0;
  int ell2 = 0;
  float* Y = nullptr;
  int64_t ldy = 0;
  float* Z = nullptr;
  int64_t ldz = 0;
  int* status = nullptr;
};
bool dual_bf16_supported(int ell1, int ell2);
void view_dual_bf16(const DualBf16Args& a, cudaStream_t s);
int view_bf16_ncol(int ell);

// FP32 form on the tensor cores (3xTF32).  The thin operand is given split:
// Bhi = x with the low 13 mantissa bits cleared, Blo = x - Bhi (split_tf32);
// both col-major with the same ld (ld * 4 a multiple of 16 bytes).
struct ViewTf32Args {
  int device = 0;
  int mode = 0;
  const float* A = nullptr;
  int64_t lda = 0, row0 = 0, rows = 0, n = 0;
  const float* Bhi = nullptr;
  const float* Blo = nullptr;
  int64_t ldb = 0;
  int ell = 0;
  float* out = nullptr;
  int64_t ldo = 0;
  int* status = nullptr;
  const int* run_if = nullptr;  // device flag: the launch is a no-op when *run_if == 0
};
void view_tf32x3(const ViewTf32Args& a, cudaStream_t s);
// C64 (a x b, ld ldc) += P^T Q for tall FP32 panels P (m x a, ld lda) and Q
// (m x b, ld ldb), both col-major, on the tensor cores (3xTF32, both operands
// split in shared memory; FP32 partial sums per CTA, added in FP64).  lda,
// ldb multiples of 4 and 16-byte aligned bases (TMA).
struct GramTf32Args {
  int device = 0;
  const float* P = nullptr;
  int64_t lda = 0;
  int a = 0;
  const float* Q = nullptr;
  int64_t ldb = 0;
  int b = 0;
  int64_t m = 0;
  double* C64 = nullptr;
  int64_t ldc = 0;
  int* status = nullptr;
  const int* run_if = nullptr;
};
void gram_tf32x3(const GramTf32Args& a, cudaStream_t s);
// hi + lo = scale * src (rows x cols, column-major), or scale * src^T when
// trans (src then cols x rows, column-major).
void split_tf32(const float* src, int64_t lds, float* hi, float* lo, int64_t ldd, int64_t rows, int64_t cols,
                cudaStream_t s, float scale = 1.f, bool trans = false);

// ---------------------------------------------------------- elementwise
// run_if (device int, optional): zero only when *run_if != 0.
void zero_f32(float* p, int64_t rows, int64_t cols, int64_t ld, cudaStream_t s, const int* run_if = nullptr);
void zero_bytes(void* p, size_t bytes, cudaStream_t s);
// Reverse of a square SVD: the middle factor of Rb = W inner Z^T from
// Xw = W^T Wb, Xz = Z^T Zb (ell x k; either may be null) and dS (k; may be null).
void svd_bwd_inner(int ell, int k, const float* S, const float* dS, const float* Xw, const float* Xz, float* inner,
                   cudaStream_t s);
// Y += X (rows x cols, column-major).
void add_f32(float* Y, int64_t ldy, const float* X, int64_t ldx, int64_t rows, int64_t cols, cudaStream_t s);
// SRFT test matrix Phi = D F P (n x s): Rademacher signs (F32 +-1, n), DCT-II
// columns cols (s distinct indices in [0, n)).
void srft(int64_t n, int s, const float* signs, const int* cols, float* phi, int64_t ld, cudaStream_t st);
// Normal-matrix TEVD helpers: *out = sum of squares (FP64); Y += nu Q and
// out_i = max(S_i^2 - nu, 0) with nu = scale * sqrt(*sumsq); B = (B + B^T) / 2.
void sumsq_f32(const float* Y, int64_t ld, int64_t rows, int64_t cols, double* out, cudaStream_t s);
void shift_add_f32(float* Y, int64_t ldy, const float* Q, int64_t ldq, int64_t rows, int64_t cols, const double* sumsq,
                   float scale, cudaStream_t s);
void symmetrize_f64(double* B, int n, cudaStream_t s);
void sq_shift(const float* S, int k, const double* sumsq, float scale, float* out, cudaStream_t s);
// dst (bf16, col-major rows x cols, ldd) = round(src); with lo != nullptr
// also lo = round(src - hi) (the hi/lo split of a thin operand).
void f32_to_bf16(const float* src, int64_t lds, __nv_bfloat16* dst, __nv_bfloat16* lo, int64_t ldd, int64_t rows,
                 int64_t cols, cudaStream_t s);
// run_if (device int, optional): skip the copy when *run_if == 0.
void copy_f32(const float* src, int64_t lds, float* dst, int64_t ldd, int64_t rows, int64_t cols, cudaStream_t s,
              const int* run_if = nullptr);
// The sign rule of the outputs: flip (u_i, v_i), i < k, when the
// largest-magnitude entry of u_i (lowest row on ties) is negative.
void fix_signs(float* U, int64_t ldu, int64_t m, float* V, int64_t ldv, int64_t n, int k, cudaStream_t s);
// Rows of U split over ranks: the signed largest-magnitude entry of each
// column into peaks[slot * k + col]; after the caller sums the world x k
// buffer over the ranks, flip_by_peaks applies the sign rule of fix_signs
// with the peak taken over all ranks (lowest rank on ties).
void col_peaks(const float* U, int64_t ldu, int64_t m, float* peaks, int slot, int k, cudaStream_t s);
void flip_by_peaks(float* U, int64_t ldu, int64_t m, float* V, int64_t ldv, int64_t n, const float* peaks,
                   int world, int k, cudaStream_t s);

// ---------------------------------------------------- small dense kernels
// Cholesky of an FP64-accumulated Gram (ell <= 128) in one CTA:
//   G (ell x ell, FP64 col-major, ld ell) = R^T R; writes Rinv (FP32,
//   ell x ell, ldr) and, unless Racc is nullptr, Racc (FP64, ldacc) = R
//   (init_acc must be true).  Breakdown / non-finite -> status.
enum CholMode { CHOL_PLAIN = 0, CHOL_SHIFT_IF_NEEDED = 1, CHOL_IF_FLAGGED = 2, CHOL_SHIFT_IF_FLAGGED = 3 };
void chol_inv(const double* G, int ell, float* Rinv, int ldr, double* Racc, int ldacc, bool init_acc, int mode,
              int* needs_more, int* status, cudaStream_t s);
// CholeskyQR2 of one column block (w <= 128 columns at Y, rows m, column-
// major, in place) in one cooperative persistent kernel with tensor-core row
// products (orth_tc.cu); shifted CholeskyQR3 after a breakdown, or the
// four-pass form with robust.  R (w x w, ld ldr) receives the triangular
// factor when not null.  scratch: orth_tc_scratch_doubles(w) doubles.
// ybf (optional): a BF16 copy of the final Q (column-major, ld ldbf).
bool orth_tc_supported(int64_t m, int w);
size_t orth_tc_scratch_doubles(int w);
void orth_tc(float* Y, int64_t ldy, int64_t m, int w, double* R, int ldr, double* scratch, int robust, int* status,
             int device, cudaStream_t s, __nv_bfloat16* ybf = nullptr, int64_t ldbf = 0);
// *sel = the minimum-variance l_c (Section 6.6) from nl trial spectra of k
// singular values each (lam[l_c * k + i]).
void minvar_select(const float* lam, int nl, int k, int* sel, cudaStream_t s);
// Racc <- R2 Racc (upper-triangular FP64, n x n); no-op when *run_if == 0.
void upper_product(const double* R2, int ld2, double* Racc, int ldr, int n, const int* run_if, cudaStream_t s);
// X = R^{-1} (FP32) for an upper-triangular FP64 R (n <= 128).
void tri_inv(const double* R, int ldr, int n, float* X, int ldx, int* status, cudaStream_t s);
// R (ell x ell FP64) block (rows r0.., cols c0..) += C (FP64 in, col-major)
void add_block_f64(double* R, int ldr, int r0, int c0, const double* C, int ldc, int rows, int cols, cudaStream_t s);
void f64_to_f32(const double* src, int lds, float* dst, int ldd, int rows, int cols, cudaStream_t s);
// One-sided Jacobi SVD of M (rows x cols, FP32 col-major, rows >= cols):
//   M = U diag(S) V^T; U overwrites Wk (rows x cols), V (cols x cols), S desc.
// M is scratch: its contents are destroyed.
void jacobi_svd(float* M, int ldm, int rows, int cols, float* Wk, int ldw, float* V, int ldv, float* S,
                double* S64, int* status, cudaStream_t s);
// Cluster variant for square n x n (rows of W and V split over the P CTAs of
// a cluster, G lanes per column pair; 0 = the defaults); size 0 when n does
// not fit.
int jacobi_cluster_size(int n);
// Column-block cluster Jacobi (jacobi_block.cu): cluster size for an n x n
// core (0 if it does not fit), and the SVD itself (P = 0: that size).
int jacobi_block_size(int n);
// One CTA waits, through the cluster kernels' bounded-wait routine, on an
// mbarrier phase that nothing completes; records LR_ERR_TIMEOUT after
// timeout_ns (selftest.cu).
void selftest_bounded_wait(int* status, uint64_t timeout_ns, cudaStream_t s);
// M (n x n, ld ldm) is read, then overwritten: it holds V while the kernel runs.
void jacobi_svd_block(float* M, int ldm, int n, float* U, int ldu, float* V, int ldv, float* S, int* status,
                      cudaStream_t s, int P = 0);
void jacobi_svd_cluster(const float* M, int ldm, int n, float* U, int ldu, float* V, int ldv, float* S, int* status,
                        cudaStream_t s, int P = 0, int G = 0);
// Copy a square FP64 upper-triangular R into FP32 (transposed if trans).
void r_to_f32(const double* R, int ldr, int n, float* out, int ldo, bool trans, cudaStream_t s);
// Small dense QR helper for the single-pass core: see single_pass driver.
void scale_cols_f32(float* A, int64_t lda, int64_t rows, int cols, const float* scale, cudaStream_t s);
// out = copyltu(M - C): symmetric n x n from the lower triangle (C FP64 or null).
void qr_bwd_sym(const float* M, const double* C, int n, float* out, cudaStream_t s);

}  // namespace lr
