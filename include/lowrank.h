/*
 * lowrank.h -- C ABI of liblowrank.so: pass-efficient randomized low-rank SVD
 * on one GB300 GPU (sm_103a), after E. K. Bjarkason, "Pass-Efficient
 * Randomized Algorithms for Low-Rank Matrix Approximation Using Any Number of
 * Views" (2018).
 *
 * Notation.  The paper's target rank p, oversampling l and sketch width
 * k = p + l are called k, p and ell = k + p here.  A is m x n (the paper's
 * n_r x n_c).  Omega (n x ell) and Psi (m x ell2) are the caller's random
 * test matrices (the paper's Omega_r and Omega_c); the library draws no random
 * numbers.
 *
 * Conventions shared by every call.
 *  - Memory.  Every lr_mat is a non-owning view of caller memory.  Unless a
 *    call says otherwise, data points to device memory of the handle's device.
 *    The library never allocates in a compute call: scratch comes from the
 *    workspace given to lr_set_workspace (size from lr_workspace_size).
 *  - Layout.  A is row-major (col_major = 0), ld = elements between rows,
 *    ld >= cols, ld*elem_size a multiple of 16 bytes and data 16-byte
 *    aligned (TMA).  Thin matrices (Omega, Psi, Y, Z, U, V) are column-major
 *    FP32 (col_major = 1, ld >= rows).  S is a vector of k FP32 (or FP64)
 *    values in a rows = k, cols = 1 view.  Small square factors (R) are FP64
 *    column-major.
 *  - Precision.  A in LR_F32 runs the FP32 form (FP32 operands, FP32
 *    products); A in LR_BF16 runs the BF16 form (A and the thin operands in
 *    BF16 on the tensor cores with FP32 accumulation).  Orthonormalisation,
 *    small factorisations and outputs are FP32 with FP64-accumulated Grams.
 *  - Streams.  stream is a cudaStream_t (NULL = legacy default stream).
 *    Calls are asynchronous; outputs are valid once the stream has synced.
 *    Argument errors are returned synchronously and nothing is launched.
 *    Numerical failures found on the device (Cholesky breakdown, non-finite
 *    values) and bounded-wait timeouts are recorded in a device status word
 *    that lr_get_status reads (it synchronises the stream).
 *  - Outputs.  S is sorted in descending order; U and V have orthonormal
 *    columns; the sign of each pair (u_i, v_i) makes the largest-magnitude
 *    entry of u_i positive.
 *  - Threading.  A handle may be used by one host thread at a time.
 */
#ifndef LOWRANK_H
#define LOWRANK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LR_OK = 0,
  LR_ERR_INVALID_ARG = 1,  /* NULL pointer, k/p/v out of range           */
  LR_ERR_SHAPE = 2,        /* inconsistent rows/cols/ld                   */
  LR_ERR_DTYPE = 3,        /* unsupported element type or layout          */
  LR_ERR_ALIGNMENT = 4,    /* pointer or stride not 16-byte aligned       */
  LR_ERR_BREAKDOWN = 5,    /* Cholesky pivot <= 0 (sketch rank-deficient) */
  LR_ERR_NONFINITE = 6,    /* NaN or Inf in a Gram matrix                 */
  LR_ERR_TIMEOUT = 7,      /* a bounded device-side wait ran out          */
  LR_ERR_CUDA = 8,         /* CUDA runtime error (see lr_last_error)      */
  LR_ERR_NOMEM = 9,        /* workspace missing or too small              */
  LR_ERR_UNSUPPORTED = 10  /* valid request this build does not serve     */
} lr_status;

typedef enum { LR_F32 = 0, LR_BF16 = 1, LR_F64 = 2 } lr_dtype;

/* Non-owning matrix view. */
typedef struct {
  void* data;
  int64_t rows, cols, ld;
  int32_t dtype;     /* lr_dtype */
  int32_t col_major; /* 1 column-major, 0 row-major */
} lr_mat;

/* lr_opts.l_c value: choose l_c by the minimum-variance rule of Section 6.6. */
#define LR_LC_MINVAR (-2)

/* Options; zero-initialise for defaults. */
typedef struct {
  int32_t l_c;              /* Alg. 7 truncation oversampling: 0 <= l_c <= l_1; -1 (or any other
                               negative value but LR_LC_MINVAR) means l_c = l_1 (the baseline);
                               LR_LC_MINVAR picks l_c from the sketches (the call then
                               synchronises its stream once, as the choice sizes the rest) */
  int32_t enhanced;         /* lr_block_krylov: 1 = row-streamed variant of Section 7.3 */
  int32_t split_last;       /* BF16 form: last view's operand as BF16 hi + lo (two products) */
  int32_t shifted_fallback; /* 0: every thin QR retries a Cholesky breakdown of its first
                               pass with a shifted Gram and adds a third pass (shifted
                               CholeskyQR3): full-rank sketches up to kappa ~ 1e7.  1: also
                               rank-deficient sketches (A of rank below k + p; a block
                               Krylov basis of three or more blocks whose later blocks,
                               projected out of the earlier ones, keep directions near FP32
                               rounding): a flagged block takes shifted, shifted, plain,
                               plain passes; without it such a sketch ends in
                               LR_ERR_BREAKDOWN */
  int32_t band_mb;          /* one-read sketches (dual, chained): 0 = default: the dual
                               sketch of a BF16 A with ell1 <= 128 and ell2 <= 64, or
                               ell1 <= 64 and ell2 <= 128, runs the fused kernel that
                               feeds each staged tile of A to both products (A read
                               once), other widths two full passes;
                               -2 = the fused kernel whenever ell1 <= 128, ell2 <= 256;
                               -1 = two full passes; > 0 = L2 bands of that many MiB of
                               A, each read by the two products back to back */
  int32_t host_panels;      /* host-streamed calls: 0 = A_host row-major m x n (ld); 1 = A_host
                               stored as ceil(n / panel_cols) column panels, panel i at
                               element offset i * m * panel_cols, each m x panel_cols
                               row-major (ld = panel_cols; the last panel's columns past n
                               unused): every panel then crosses the host link as one
                               contiguous copy.  panel_cols must be a multiple of 4 */
  int32_t reserved[2];
} lr_opts;

typedef struct lr_handle_s* lr_handle;

/* Handle on `device`.  Allocates a small device status word (the only
 * allocation the library makes).  Errors: LR_ERR_INVALID_ARG, LR_ERR_CUDA. */
lr_status lr_create(lr_handle* handle, int device);
lr_status lr_destroy(lr_handle handle);

/* Static description of a status code; never NULL. */
const char* lr_status_string(lr_status status);
/* Detail of the last error on this handle (empty string if none). */
const char* lr_last_error(lr_handle handle);

/* Workspace bytes sufficient for any call of this library on an m x n A with
 * sketch widths ell1 (range) and ell2 (co-range, 0 if unused) and v views. */
lr_status lr_workspace_size(lr_handle handle, int64_t m, int64_t n, int ell1, int ell2, int v,
                            size_t* bytes);
/* Device workspace owned by the caller, 256-byte aligned, kept until replaced. */
lr_status lr_set_workspace(lr_handle handle, void* dev_ptr, size_t bytes);

/* Synchronise `stream`, return the device status word (an lr_status) in
 * *device_status and clear it. */
lr_status lr_get_status(lr_handle handle, void* stream, int* device_status);

/* One view of A (Section 4 and Alg. 2; the sketches of Section 6.5, Alg. 7):
 *   Y = A X   (X: n x ell1, Y: m x ell1) when X != NULL,
 *   Z = A^T W (W: m x ell2, Z: n x ell2) when W != NULL.
 * With both X and W the two products share one read of A from HBM (the
 * paper's steps a) and b) of Alg. 7 done in parallel).  Y and Z are
 * overwritten.  A is F32 or BF16 row-major; X, W, Y, Z are F32 column-major. */
lr_status lr_sketch(lr_handle handle, const lr_mat* A, const lr_mat* X, const lr_mat* W,
                    lr_mat* Y, lr_mat* Z, const lr_opts* opts, void* stream);

/* Chained view (Section 6.8): Y = A X and Z = A^T Y from one read of A.
 * Same argument rules as lr_sketch; Y and Z are overwritten. */
lr_status lr_sketch_chained(lr_handle handle, const lr_mat* A, const lr_mat* X, lr_mat* Y,
                            lr_mat* Z, const lr_opts* opts, void* stream);

/* Thin QR in place, Y (m x ell, F32 column-major, m >= ell) -> Q with
 * Y = Q R, Q^T Q = I, R upper triangular with positive diagonal (the qr of
 * Section 2).  Computed by block CholeskyQR2: column blocks of width <= 128,
 * each projected out of the previous ones twice (BCGS2) and factorised by
 * CholeskyQR2 with FP64-accumulated Grams.  When a block's first Cholesky
 * breaks down (Y ill-conditioned in FP32), that pass is redone with the
 * shifted Gram of shifted CholeskyQR and a third pass follows (shifted
 * CholeskyQR3); LR_ERR_BREAKDOWN enters the status word only if even the
 * shifted factorisation fails (Y numerically rank-deficient).  R (ell x ell,
 * F64 column-major) may be NULL. */
lr_status lr_orth(lr_handle handle, lr_mat* Y, lr_mat* R, const lr_opts* opts, void* stream);

/* Generalized subspace iteration, Alg. 2 (Section 4): v >= 2 views, sketch
 * width ell = k + p, Omega n x ell.  Outputs U (m x k), S (k), V (n x k). */
lr_status lr_subspace_iter(lr_handle handle, const lr_mat* A, int k, int p, int v,
                           const lr_mat* Omega, lr_mat* U, lr_mat* S, lr_mat* V,
                           const lr_opts* opts, void* stream);

/* Single-pass TSVD, Alg. 7 (Section 6.5, Tropp variant): Omega n x ell1,
 * Psi m x ell2 with ell2 >= ell1 > k; opts->l_c in [0, ell1 - k] truncates
 * Q_c to its leading k + l_c left singular vectors (l_c < 0: none, the
 * baseline of Section 6.2).  Both sketches come from one read of A. */
lr_status lr_single_pass(lr_handle handle, const lr_mat* A, int k, const lr_mat* Omega,
                         const lr_mat* Psi, lr_mat* U, lr_mat* S, lr_mat* V,
                         const lr_opts* opts, void* stream);

/* Generalized block Krylov, Alg. 9 (Section 7.2), v >= 2 views.  With
 * opts->enhanced = 1: the row-streamed variant of Section 7.3, in which each
 * of the first v-1 views yields A X and A^T (A X) from one read of A, giving
 * the co-range Krylov space of Alg. 9 with 2v-1 views. */
lr_status lr_block_krylov(lr_handle handle, const lr_mat* A, int k, int p, int v,
                          const lr_mat* Omega, lr_mat* U, lr_mat* S, lr_mat* V,
                          const lr_opts* opts, void* stream);

/* Row-streamed one-pass QB of Section 6.8: Y = A Omega and A^T Y from one
 * read, Q_c R_c = Y, B^T = (A^T Y) R_c^{-1}, then the TSVD of B. */
lr_status lr_rowwise_single_pass(lr_handle handle, const lr_mat* A, int k, const lr_mat* Omega,
                                 lr_mat* U, lr_mat* S, lr_mat* V, const lr_opts* opts,
                                 void* stream);

/* Host-streamed single pass (Section 6.1 streaming model, A = sum of column
 * panels): A_host is F32 row-major in pinned host memory; it is copied to the
 * device in panels of panel_cols columns through two device panel buffers
 * (carved from the workspace) on a copy stream overlapped with the sketches,
 * so A crosses the host link once.  With opts->host_panels = 1 A_host is
 * stored panel by panel (see lr_opts) and each panel is one contiguous copy.  The workspace needs
 * lr_workspace_size(m, n, ell1, ell2, 1) plus 2 * m * round4(panel_cols) * 4
 * bytes.  Errors: LR_ERR_INVALID_ARG also when A_host is not page-locked.
 * Otherwise as lr_single_pass. */
lr_status lr_single_pass_host(lr_handle handle, const lr_mat* A_host, int64_t panel_cols, int k,
                              const lr_mat* Omega, const lr_mat* Psi, lr_mat* U, lr_mat* S,
                              lr_mat* V, const lr_opts* opts, void* stream);

/* Alg. 2 (generalized subspace iteration, any v >= 2) on an A kept in pinned
 * host memory (the out-of-core setting of Section 6.1; every view streams A
 * once).  A_host: F32 row-major m x n, page-locked (cudaHostAlloc or
 * cudaHostRegister), never copied whole: each view moves panels of
 * panel_cols columns through two device buffers on a copy stream while the
 * previous panel is multiplied.  The workspace needs lr_workspace_size(m, n,
 * k + p, 0, v) plus 2 * m * round4(panel_cols) * 4 bytes.  Other arguments and
 * outputs as lr_subspace_iter; errors as lr_single_pass_host. */
lr_status lr_subspace_iter_host(lr_handle handle, const lr_mat* A_host, int64_t panel_cols, int k, int p, int v,
                                const lr_mat* Omega, lr_mat* U, lr_mat* S, lr_mat* V, const lr_opts* opts,
                                void* stream);

/* Alg. 9 (as lr_block_krylov) end to end from host buffers: A_host (F32 or
 * BF16 row-major, page-locked) and Omega_host (F32 column-major n x (k+p))
 * are copied once into the device workspace on `stream`, the factorisation
 * runs on the device (all v views read the device copy), and U_host,
 * S_host, V_host (F32; U m x k and V n x k column-major, page-locked) receive
 * the results by device-to-host copies queued on `stream`: they are valid
 * once `stream` has finished.  The workspace needs lr_workspace_size(m, n,
 * k + p, 0, v) plus the staging of A (m * ld * element size), Omega, U, S
 * and V, each rounded up to 256 bytes.  Errors as lr_block_krylov, and
 * LR_ERR_INVALID_ARG when a host buffer is not page-locked. */
lr_status lr_block_krylov_host(lr_handle handle, const lr_mat* A_host, int k, int p, int v,
                               const lr_mat* Omega_host, lr_mat* U_host, lr_mat* S_host, lr_mat* V_host,
                               const lr_opts* opts, void* stream);

/* ---------------------------------------------------------------------
 * Matrix-free operators (Section 4.2.3; the paper's J applied by direct and
 * adjoint methods).
 * ------------------------------------------------------------------- */

/* J (rows x cols) as a callback: apply(ctx, 0, X, ldx, ncols, Y, ldy, stream)
 * writes Y = J X (X: cols x ncols, Y: rows x ncols); apply(ctx, 1, ...)
 * writes Y = J^T X (X: rows x ncols, Y: cols x ncols).  X and Y are F32
 * column-major device arrays owned by the library (X must not be written),
 * and the work is enqueued on `stream` (the stream of the calling entry
 * point); the callback returns 0 on success, anything else aborts the call
 * with LR_ERR_INVALID_ARG.  The callback must not use the same lr_handle. */
typedef int (*lr_apply_fn)(void* ctx, int transpose, const float* X, int64_t ldx, int64_t ncols, float* Y,
                           int64_t ldy, void* stream);
typedef struct {
  int64_t rows, cols;
  lr_apply_fn apply;
  void* ctx;
} lr_operator;

/* Alg. 2 with J given as an operator (every view one callback).  Arguments
 * and outputs as lr_subspace_iter with A replaced by J. */
lr_status lr_subspace_iter_op(lr_handle handle, const lr_operator* J, int k, int p, int v, const lr_mat* Omega,
                              lr_mat* U, lr_mat* S, lr_mat* V, const lr_opts* opts, void* stream);

/* Alg. 4 (Nystrom / prolonged sketch): approximate rank-k EVD V diag(Lambda2)
 * V^T of J^T J from v >= 2 views of J.  Omega (F32 column-major) is
 * cols x (k+p) for even v (the start of Alg. 3 on J; orthonormalised for
 * v = 2) and rows x (k+p) for odd v (Alg. 3 on J^T).  The shift is
 * nu = 2^-23 ||Y_r||_F (the paper's 2.2e-16 ||Y_r|| scaled to FP32; subtracted
 * again, eigenvalues below it clipped to 0).  k + p <= 128 (the Cholesky of
 * the (k+p) x (k+p) core runs in one CTA).  Outputs: V (cols x k, F32
 * column-major, orthonormal, each column's largest entry positive),
 * Lambda2 (k F32, descending).  Errors as lr_subspace_iter; a Cholesky
 * breakdown sets LR_ERR_BREAKDOWN in the status word. */
lr_status lr_nystrom_tevd(lr_handle handle, const lr_operator* J, int k, int p, int v, const lr_mat* Omega,
                          lr_mat* V, lr_mat* Lambda2, const lr_opts* opts, void* stream);

/* Alg. 5 (pinched sketch): rank-k EVD of J^T J from v >= 2 views of J:
 * Q_r from v - 1 views (Alg. 3 on J^T from an Omega of rows x (k+p) for
 * even v, on J from cols x (k+p) for odd v), B_c = J Q_r, and the EVD of
 * B_c^T B_c through the SVD of B_c's triangular factor.  Outputs as
 * lr_nystrom_tevd. */
lr_status lr_pinched_tevd(lr_handle handle, const lr_operator* J, int k, int p, int v, const lr_mat* Omega,
                          lr_mat* V, lr_mat* Lambda2, const lr_opts* opts, void* stream);

/* Single-view TSVD, Woolfe variant (Alg. 8, Section 6.5): the sketches of
 * lr_single_pass; Q_c and Q_r are the leading k + l_c left singular vectors
 * of Y_c = A Omega and Y_r = A^T Psi (opts->l_c as in lr_single_pass, minus
 * LR_LC_MINVAR), X^ the least-squares solution of (Psi^T Q_c) X^ =
 * Y_r^T Q_r, U = Q_c U^ and V = Q_r V^ from the SVD of X^.  Arguments,
 * outputs and errors as lr_single_pass; the workspace as lr_workspace_size
 * with ell1, ell2. */
lr_status lr_single_pass_woolfe(lr_handle handle, const lr_mat* A, int k, const lr_mat* Omega, const lr_mat* Psi,
                                lr_mat* U, lr_mat* S, lr_mat* V, const lr_opts* opts, void* stream);

/* Single-view TSVD with the extended sketch of Section 6.7 (the
 * approximation bwz2): Y_c = A Omega, Y_r = A^T Psi and Z = Phi_r^T A Phi_c,
 * all from one pass over A (A Phi_c rides in the range view with Omega);
 * Q_c R_c = Y_c, Q_r R_r = Y_r, U_c T_c = Phi_r^T Q_c, U_r T_r = Phi_c^T Q_r,
 * C = T_c^{-1} U_c^T Z U_r T_r^{-T}, U = Q_c U^, V = Q_r V^ from C's SVD.
 * Omega n x ell, Psi m x ell (l_1 = l_2), Phi_c n x s and Phi_r m x s with
 * ell <= s <= min(m, n) (F32 column-major; lr_srft forms SRFT ones).
 * Outputs and errors as lr_single_pass.  The workspace needs
 * lr_workspace_size(m, n, ell + s, ell + s, 1). */
lr_status lr_single_pass_extended(lr_handle handle, const lr_mat* A, int k, const lr_mat* Omega, const lr_mat* Psi,
                                  const lr_mat* Phi_c, const lr_mat* Phi_r, lr_mat* U, lr_mat* S, lr_mat* V,
                                  const lr_opts* opts, void* stream);

/* The SRFT test matrix of Section 6.7, Phi = D F P (n x s, F32 column-major,
 * written into Phi on the device): D = diag(signs) (n Rademacher signs, F32
 * +-1, device), F the orthonormal DCT-II matrix (columns the cosine basis:
 * F[j, k] = c_k sqrt(2/n) cos(pi (2j+1) k / (2n)), c_0 = 1/sqrt(2), else 1),
 * P the columns cols[0..s) (distinct indices in [0, n), device int32).
 * Asynchronous on `stream`. */
lr_status lr_srft(lr_handle handle, int64_t n, int s, const float* signs, const int* cols, lr_mat* Phi, void* stream);

/* ---------------------------------------------------------------------
 * Row-sharded matrices over several GPUs (one process per GPU).
 * ------------------------------------------------------------------- */

/* The caller's collective: allreduce(ctx, buf, count, dtype, stream) sums
 * `count` elements of the device array buf (dtype LR_F32 or LR_F64) over
 * all ranks, in place, ordered on `stream` (e.g. an NCCL all-reduce on that
 * stream); returns 0 on success.  Every rank calls it the same number of
 * times with the same counts, in the same order. */
typedef int (*lr_allreduce_fn)(void* ctx, void* buf, int64_t count, int dtype, void* stream);
typedef struct {
  int rank, world;
  lr_allreduce_fn allreduce;
  void* ctx;
} lr_comm;

/* Alg. 2 on a matrix whose rows are split over the ranks: rank g holds A_g
 * (m_g x n, the g-th block of rows, any m_g >= 1) and the same Omega
 * (n x (k+p)); it receives U_g (m_g x k, its rows of U), and S and V
 * (replicated).  Range views A_g X are local; each co-range view sums
 * A_g^T W_g over the ranks (one all-reduce of n x (k+p) F32); the thin QR
 * of the row-sharded Q_c all-reduces its (k+p) x (k+p) FP64 Grams (and the
 * block projections) and factors the sum on every rank; the replicated
 * factors (Q_r and R_r, the core SVD) are taken from rank 0 (an all-reduce
 * with zeros elsewhere), so every rank holds the same bits; the sign of each
 * pair is fixed by the largest-magnitude entry of u_i over all ranks (ties
 * to the lowest global row), as in lr_subspace_iter.  Requires
 * k + p <= min(sum m_g, n); the caller checks that the ranks agree on the
 * shapes and arguments.  Otherwise as lr_subspace_iter. */
lr_status lr_subspace_iter_sharded(lr_handle handle, const lr_mat* A_local, int k, int p, int v, const lr_mat* Omega,
                                   lr_mat* U_local, lr_mat* S, lr_mat* V, const lr_comm* comm, const lr_opts* opts,
                                   void* stream);

/* Reverse pass of lr_subspace_iter for the loss L = sum_i dS_i sigma_i
 * (dS: k weights, F32): writes dA = dL/dA (m x n, F32 row-major, same shape
 * as A, overwritten).  The forward views are recomputed, not stored.  A must
 * be F32. */
lr_status lr_subspace_iter_backward(lr_handle handle, const lr_mat* A, int k, int p, int v,
                                    const lr_mat* Omega, const lr_mat* dS, lr_mat* dA,
                                    const lr_opts* opts, void* stream);

/* Reverse pass of lr_subspace_iter for a loss on all three outputs,
 * L = <dU, U> + <dS, S> + <dV, V> (the gradients of any loss at the
 * outputs): writes dA = dL/dA.  dU (m x k) and dV (n x k) are F32
 * column-major, dS k F32 values; any of the three may be NULL (zero), not
 * all.  The reverse of the core SVD couples the k kept singular pairs to the
 * other ell - k of the core through 1 / (s_j^2 - s_i^2) (a pair whose two
 * values coincide contributes nothing), and the sign fix of the forward is
 * applied to dU and dV.  Otherwise as lr_subspace_iter_backward. */
lr_status lr_subspace_iter_backward_uv(lr_handle handle, const lr_mat* A, int k, int p, int v, const lr_mat* Omega,
                                       const lr_mat* dU, const lr_mat* dS, const lr_mat* dV, lr_mat* dA,
                                       const lr_opts* opts, void* stream);

/* ---------------------------------------------------------------------
 * Instrumentation (the paper has no counterpart; used by benchmarks).
 * ------------------------------------------------------------------- */

/* Kernel classes timed by the trace. */
typedef enum {
  LR_TRACE_VIEW_RANGE = 0,   /* Y = A X on the tensor cores (BF16) or SIMT (FP32) */
  LR_TRACE_VIEW_CORANGE = 1, /* Z = A^T W                                          */
  LR_TRACE_ORTH = 2,         /* one lr_orth-equivalent thin QR (all its kernels)    */
  LR_TRACE_CORE_SVD = 3,     /* the small core SVD                                  */
  LR_TRACE_VIEW_DUAL = 4,    /* Y = A X and Z = A^T W in one pass (fused kernel)    */
  LR_TRACE_COUNT = 5
} lr_trace_kind;

/* Turn per-launch CUDA-event timing of the classes above on (1) or off (0).
 * Enabling pre-creates a pool of events (no allocation afterwards); each
 * timed launch records two events on the call's stream. */
lr_status lr_set_trace(lr_handle handle, int on);
/* Synchronise the device, then return the accumulated device time (ms) and
 * the number of timed launches of `kind` since tracing was enabled or last
 * reset (reset != 0 clears the accumulators). */
lr_status lr_trace_read(lr_handle handle, int kind, double* total_ms, int64_t* launches, int reset);
/* Number of CUDA kernels this process has launched through the library. */
lr_status lr_kernel_launches(lr_handle handle, uint64_t* count);

/* Self-test of the bounded waits (no counterpart in the paper).  The
 * cluster kernels (the core SVD) wait on mbarrier phases that their peer
 * CTAs complete, each wait bounded (2 s) so that a lost arrival ends in
 * LR_ERR_TIMEOUT in the device status word instead of a hung GPU.  This call
 * runs that same bounded wait in one CTA on a phase that nothing completes,
 * for timeout_us microseconds (1 .. 1000000), then records LR_ERR_TIMEOUT
 * and returns: read it with lr_get_status.  The kernel ends by itself and
 * the context stays usable.  Asynchronous on `stream`. */
lr_status lr_selftest_bounded_wait(lr_handle handle, int64_t timeout_us, void* stream);

/* ---------------------------------------------------------------------
 * Allocation-free range view (the paper has no counterpart).
 * ------------------------------------------------------------------- */

/* Y = A X as lr_sketch computes it with W = NULL, for callers that cannot
 * call cudaMalloc at all -- e.g. a host program whose own pool has reserved
 * the device's memory, or one that cannot accept the device-wide
 * synchronisation a cudaMalloc may imply -- and therefore cannot create an
 * lr_handle or provide a workspace.  No handle is needed and nothing is
 * allocated: the BF16 copy of X that the tensor-core kernel reads lives in a
 * 4 MiB file-scope device array, so ceil8(n) * ell * 2 bytes must fit in
 * 4 MiB minus 256 bytes (else LR_ERR_UNSUPPORTED), and ell <= 256.  For a
 * BF16 A the view is lr_sketch's own tensor-core kernel.  An F32 A needs no
 * scratch: it runs on the SIMT GEMM and matches lr_sketch (3xTF32) to within
 * the view tolerance, not bit for bit.  Arguments as for lr_sketch; runs on
 * the current device and `stream`.
 * Set-up: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture
 * begins.  Under lazy module loading (the CUDA default) that first call is
 * also when the runtime loads this code and reserves the 4 MiB on the
 * device (held until the process exits), so a caller whose pool will claim
 * the device's memory makes the first call at start-up, or sets
 * CUDA_MODULE_LOADING=EAGER.
 * All calls share the array: calls that overlap on the GPU (other streams
 * or host threads on the same device) race and must be serialised by the
 * caller.  Argument errors are returned synchronously; a device-side
 * failure (a bounded wait that ran out: LR_ERR_TIMEOUT) is kept in the
 * array's status word, which every call clears at its start and
 * lr_sketch_range_static_status reads. */
lr_status lr_sketch_range_static(const lr_mat* A, const lr_mat* X, lr_mat* Y, void* stream);

/* The device status word of the latest lr_sketch_range_static call on the
 * current device (0 or an lr_status code), copied to *device_status after
 * `stream` has finished that call (synchronises `stream`).  Allocates
 * nothing. */
lr_status lr_sketch_range_static_status(void* stream, int* device_status);

#ifdef __cplusplus
}
#endif
#endif /* LOWRANK_H */
