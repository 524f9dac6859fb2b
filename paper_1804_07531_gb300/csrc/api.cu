// C ABI of liblowrank: argument validation, workspace arena and the drivers
// of the paper's view schedules (Bjarkason 2018):
//   lr_subspace_iter        Alg. 2 (generalized subspace iteration, any v >= 2)
//   lr_single_pass          Alg. 7 (1-view, Tropp variant with l_c)
//   lr_block_krylov         Alg. 9 (generalized block Krylov) and, with
//                           opts->enhanced, the row-streamed variant of Sec. 7.3
//   lr_rowwise_single_pass  the one-pass QB of Section 6.8
// plus the building blocks lr_sketch / lr_sketch_chained (views) and lr_orth
// (thin QR by block CholeskyQR2).  Every step runs in this library's kernels.
#include <algorithm>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"

struct lr_trace_rec {
  int kind;
  cudaEvent_t begin, end;
};

struct lr_handle_s {
  int device = 0;
  int* status_dev = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  std::string last_error;
  // instrumentation: a fixed pool of events, filled in order while tracing
  bool trace = false;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  std::vector<lr_trace_rec> recs;
  double acc_ms[LR_TRACE_COUNT] = {};
  int64_t acc_n[LR_TRACE_COUNT] = {};
  // host-streamed sketches: a copy stream and per-buffer events (created on first use)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copied[2] = {nullptr, nullptr};
  cudaEvent_t consumed[2] = {nullptr, nullptr};
};

namespace lr {
std::atomic<uint64_t> g_kernel_launches{0};
}

namespace lr {
namespace {

// FP32 column-major thin matrix; bf (when not null) a BF16 copy of it that a
// thin QR leaves for the BF16 views (column-major, ld ldbf).
struct Mat {
  float* p = nullptr;
  int64_t rows = 0, cols = 0, ld = 0;
  __nv_bfloat16* bf = nullptr;
  int64_t ldbf = 0;
  float* col(int64_t c) const { return p + c * ld; }
};

struct Ctx {
  lr_handle h = nullptr;
  cudaStream_t s = nullptr;
  Arena ar;
  int sms = 1;
  int* status = nullptr;
  lr_opts opt{};
  bool measure = false;
  const lr_comm* comm = nullptr;  // row-sharded runs: the caller's all-reduce
};

// Sum a device buffer over the ranks (no-op without a communicator).
void allreduce(Ctx& c, void* buf, int64_t count, lr_dtype dt) {
  if (c.measure || !c.comm || c.comm->world <= 1 || count <= 0) return;
  const int rc = c.comm->allreduce(c.comm->ctx, buf, count, int(dt), c.s);
  LR_REQUIRE(rc == 0, LR_ERR_INVALID_ARG, "the communicator's all-reduce failed (returned " + std::to_string(rc) + ")");
}
// Every rank takes rank 0's copy of a replicated buffer.
void broadcast0(Ctx& c, void* buf, int64_t count, lr_dtype dt) {
  if (c.measure || !c.comm || c.comm->world <= 1 || count <= 0) return;
  if (c.comm->rank != 0)
    LR_CHECK_CUDA(cudaMemsetAsync(buf, 0, size_t(count) * (dt == LR_F64 ? 8 : 4), c.s));
  allreduce(c, buf, count, dt);
}

// Records a begin/end event pair around a traced region (no-op unless the
// handle traces and events remain in the pool).
struct TraceScope {
  lr_handle h = nullptr;
  cudaStream_t s = nullptr;
  int kind = 0;
  cudaEvent_t end = nullptr;
  TraceScope(const Ctx& c, int k) {
    if (c.measure || !c.h || !c.h->trace || c.h->pool_used + 2 > c.h->pool.size()) return;
    h = c.h;
    s = c.s;
    kind = k;
    cudaEvent_t b = h->pool[h->pool_used++];
    end = h->pool[h->pool_used++];
    cudaEventRecord(b, s);
    h->recs.push_back({kind, b, end});
  }
  ~TraceScope() {
    if (h) cudaEventRecord(end, s);
  }
};

// A as the drivers see it.
struct AMat {
  const void* p = nullptr;
  int64_t m = 0, n = 0, ld = 0;
  bool bf16 = false;
  const __nv_bfloat16* b() const { return static_cast<const __nv_bfloat16*>(p); }
  const float* f() const { return static_cast<const float*>(p); }
  size_t elem() const { return bf16 ? 2 : 4; }
};

constexpr int kMaxBlock = 128;  // column block width of block CholeskyQR2

inline int64_t round8(int64_t x) { return (x + 7) / 8 * 8; }

// ----------------------------------------------------------- thin GEMMs
// C (M x N) = alpha op(A) op(B) + beta C, all FP32 column-major.
inline int64_t round4(int64_t x) { return (x + 3) / 4 * 4; }

inline bool tma_ok(const void* p, int64_t ld) {
  return (reinterpret_cast<uintptr_t>(p) & 15) == 0 && ld % 4 == 0;
}

// C (M x N) = alpha op(A) op(B) + beta C.  Tall products -- the applications
// Q = Y R^{-1} and Y_b -= Q_prev C of the thin QR, the lifts U = Q W -- run
// on the tensor cores as a co-range view of A^T (A^T row-major = A
// col-major; op(B) split into TF32 hi/lo with alpha folded in), in groups of
// at most 256 columns of C; the rest on the SIMT kernel.
void gemm(Ctx& c, int64_t M, int64_t N, int64_t K, bool ta, const float* A, int64_t lda, bool tb, const float* B,
          int64_t ldb, float* C, int64_t ldc, float alpha = 1.f, float beta = 0.f, const int* run_if = nullptr) {
  // (N > 1024 would mean over four launches that each re-read A and cover
  // few output tiles: the SIMT kernel's single launch serves that shape)
  const bool tc = !ta && M >= 2048 && K >= 1 && N <= 1024 && (beta == 0.f || beta == 1.f) && tma_ok(A, lda);
  if (tc) {
    ArenaScope sc(c.ar);
    const int64_t ldw = round4(K);
    float* wh = c.ar.take<float>(size_t(ldw) * N);
    float* wl = c.ar.take<float>(size_t(ldw) * N);
    if (c.measure) return;
    split_tf32(B, ldb, wh, wl, ldw, K, N, c.s, alpha, tb);  // op(B), K x N
    if (beta == 0.f) zero_f32(C, M, N, ldc, c.s, run_if);  // a skipped product leaves C as it was
    for (int64_t g0 = 0; g0 < N; g0 += 256) {
      ViewTf32Args a;
      a.device = c.h->device;
      a.mode = 1;
      a.A = A;
      a.lda = lda;
      a.row0 = 0;
      a.rows = K;
      a.n = M;
      a.Bhi = wh + g0 * ldw;
      a.Blo = wl + g0 * ldw;
      a.ldb = ldw;
      a.ell = int(std::min<int64_t>(256, N - g0));
      a.out = C + g0 * ldc;
      a.ldo = ldc;
      a.status = c.status;
      a.run_if = run_if;
      view_tf32x3(a, c.s);
    }
    return;
  }
  if (c.measure) return;
  GemmArgs g;
  g.run_if = run_if;
  g.M = M; g.N = N; g.K = K; g.ta = ta; g.tb = tb; g.alpha = alpha; g.beta = beta;
  g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C = C; g.ldc = ldc;
  g.mode = GEMM_STORE;
  sgemm(g, c.s);
}

// C64 (M x N, ld ldc) = op(A)^T-style reduction over a long K with FP32
// products and FP64 accumulation across K slices (Grams, cross-Grams).
void gram64(Ctx& c, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B, int64_t ldb,
            double* C64, int64_t ldc, const int* run_if = nullptr) {
  if (c.measure) return;
  LR_CHECK_CUDA(cudaMemsetAsync(C64, 0, size_t(ldc) * N * sizeof(double), c.s));
  if (K >= 1024 && tma_ok(A, lda) && tma_ok(B, ldb)) {
    // tall panels: tensor cores, FP32 products per CTA, FP64 across CTAs, in
    // groups of at most 256 columns of the result
    for (int64_t g0 = 0; g0 < N; g0 += 256) {
      GramTf32Args a;
      a.device = c.h->device;
      a.P = A;
      a.lda = lda;
      a.a = int(M);
      a.Q = B + g0 * ldb;
      a.ldb = ldb;
      a.b = int(std::min<int64_t>(256, N - g0));
      a.m = K;
      a.C64 = C64 + g0 * ldc;
      a.ldc = ldc;
      a.status = c.status;
      a.run_if = run_if;
      gram_tf32x3(a, c.s);
    }
    return;
  }
  GemmArgs g;
  g.M = M; g.N = N; g.K = K; g.ta = true; g.tb = false;
  g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C64 = C64; g.ldc = ldc;
  g.mode = GEMM_ATOMIC_F64;
  g.split_k = split_for(M, N, K, c.sms);
  g.run_if = run_if;
  sgemm(g, c.s);
}

// -------------------------------------------------------------- views
// out (rows_out x ell) = A[r0:r0+rows, :] B (mode 0, out = Y rows r0..) or
// += A[r0:r0+rows, :]^T B[r0:r0+rows, :] (mode 1, out = Z).  The output must
// be zeroed by the caller before the first contribution.
// Pre-converted thin operand (full operand rows; mode 1 offsets by r0):
// BF16 copy for a BF16 A, TF32 hi/lo split for an F32 A.
struct SplitOp {
  const __nv_bfloat16* bf = nullptr;
  const __nv_bfloat16* bf_lo = nullptr;  // BF16 remainder x - bf16(x) (split form), or null
  const float* hi = nullptr;
  const float* lo = nullptr;
  int64_t ld = 0;
};

// Converts the thin operand (rows x ell) into the form the view kernel of
// A's precision reads.  With split (BF16 A only) the operand is also kept as
// a second BF16 term, x = bf16(x) + bf16(x - bf16(x)) to ~2^-16 relative,
// and the view adds both products.
SplitOp convert_operand(Ctx& c, const AMat& A, const float* B, int64_t ldb, int64_t rows, int ell,
                        bool split = false) {
  SplitOp o;
  if (A.bf16) {
    o.ld = round8(rows);
    auto* t = c.ar.take<__nv_bfloat16>(size_t(o.ld) * ell);
    auto* t2 = split ? c.ar.take<__nv_bfloat16>(size_t(o.ld) * ell) : nullptr;
    if (!c.measure) f32_to_bf16(B, ldb, t, t2, o.ld, rows, ell, c.s);
    o.bf = t;
    o.bf_lo = t2;
  } else {
    o.ld = round4(rows);
    float* h = c.ar.take<float>(size_t(o.ld) * ell);
    float* l = c.ar.take<float>(size_t(o.ld) * ell);
    if (!c.measure) split_tf32(B, ldb, h, l, o.ld, rows, ell, c.s);
    o.hi = h;
    o.lo = l;
  }
  return o;
}

void view_band(Ctx& c, const AMat& A, int mode, const float* B, int64_t ldb, int ell, float* out, int64_t ldo,
               int64_t r0, int64_t rows, const SplitOp* pre = nullptr, bool split = false) {
  if (rows <= 0) return;
  {
    ArenaScope sc(c.ar);
    SplitOp op;
    if (pre) {
      op = *pre;
    } else {
      const int64_t orows = (mode == 0) ? A.n : rows;
      op = convert_operand(c, A, mode == 0 ? B : B + r0, ldb, orows, ell, split);
      if (mode == 1) {  // converted from the band's rows: index from row 0
        if (op.bf) op.bf -= r0;
        if (op.bf_lo) op.bf_lo -= r0;
        if (op.hi) {
          op.hi -= r0;
          op.lo -= r0;
        }
      }
    }
    if (c.measure) return;
    TraceScope tr(c, mode == 0 ? LR_TRACE_VIEW_RANGE : LR_TRACE_VIEW_CORANGE);
    for (int g0 = 0; g0 < ell; g0 += 256) {
      const int w = std::min(256, ell - g0);
      if (A.bf16) {
        ViewBf16Args a;
        a.device = c.h->device;
        a.mode = mode;
        a.A = A.b();
        a.lda = A.ld;
        a.row0 = r0;
        a.rows = rows;
        a.n = A.n;
        a.B = op.bf + (mode == 1 ? r0 : 0) + int64_t(g0) * op.ld;
        a.ldb = op.ld;
        a.ell = w;
        a.out = (mode == 0 ? out + r0 : out) + int64_t(g0) * ldo;
        a.ldo = ldo;
        a.status = c.status;
        view_bf16(a, c.s);
        if (op.bf_lo) {  // second term of the split operand, same accumulator
          a.B = op.bf_lo + (mode == 1 ? r0 : 0) + int64_t(g0) * op.ld;
          view_bf16(a, c.s);
        }
      } else {
        ViewTf32Args a;
        a.device = c.h->device;
        a.mode = mode;
        a.A = A.f();
        a.lda = A.ld;
        a.row0 = r0;
        a.rows = rows;
        a.n = A.n;
        a.Bhi = op.hi + (mode == 1 ? r0 : 0) + int64_t(g0) * op.ld;
        a.Blo = op.lo + (mode == 1 ? r0 : 0) + int64_t(g0) * op.ld;
        a.ldb = op.ld;
        a.ell = w;
        a.out = (mode == 0 ? out + r0 : out) + int64_t(g0) * ldo;
        a.ldo = ldo;
        a.status = c.status;
        view_tf32x3(a, c.s);
      }
    }
    return;
  }
}

int64_t band_rows(const AMat& A, int band_mb) {
  // band_mb > 0: bands of that many MiB of A, each read by the range and the
  // co-range products back to back so the second read hits L2 (129 MB).
  // Otherwise (0, -1): one band, i.e. two full passes over A.  Measured on GB300
  // for a 2 GiB A: two full passes (each near the HBM roof) beat every band
  // size, because each band costs two launches and partial-tile atomics
  // that outweigh the HBM bytes saved.
  if (band_mb <= 0) return A.m;
  int64_t r = int64_t(band_mb) * 1024 * 1024 / (A.n * int64_t(A.elem()));
  r = std::max<int64_t>(256, r / 256 * 256);
  return std::min<int64_t>(r, (A.m + 255) / 256 * 256);
}

// Y = A X (X: n x ell).  last: the schedule's final view, whose operand is
// split in two BF16 terms when opts.split_last asks for it.
void view_range(Ctx& c, const AMat& A, const Mat& X, Mat Y, bool last = false) {
  if (!c.measure) zero_f32(Y.p, Y.rows, Y.cols, Y.ld, c.s);
  view_band(c, A, 0, X.p, X.ld, int(X.cols), Y.p, Y.ld, 0, A.m, nullptr, last && c.opt.split_last && A.bf16);
}
// Z = A^T W (W: m x ell).
void view_corange(Ctx& c, const AMat& A, const Mat& W, Mat Z, bool last = false) {
  if (!c.measure) zero_f32(Z.p, Z.rows, Z.cols, Z.ld, c.s);
  view_band(c, A, 1, W.p, W.ld, int(W.cols), Z.p, Z.ld, 0, A.m, nullptr, last && c.opt.split_last && A.bf16);
}

// Y = A X and Z = A^T W (the two sketches of Alg. 7, steps a and b).  The
// operands are converted once.  For a BF16 A the fused kernel reads A once,
// each staged tile feeding both products; it flushes a partial Z^T per tile
// of 256 rows, ell2 / 64 bytes of L2 reductions per element of A, which L2
// absorbs at about the HBM rate (measured), so it wins where that is below
// the 2 bytes of the second read it saves.  Its narrow form (128-column
// k-blocks, ell2 <= 64, or ell2 <= 128 with ell1 <= 64) halves those
// reductions and measured faster than two passes at both widths, so by
// default it runs there; opts.band_mb = -2 forces the fused kernel
// (ell1 <= 128, ell2 <= 256), -1 forces two passes.  Otherwise the range and co-range kernels sweep the
// bands of band_rows() (by default one band: two full passes over A).
void view_dual(Ctx& c, const AMat& A, const Mat& X, Mat Y, const Mat& W, Mat Z) {
  ArenaScope sc(c.ar);
  const SplitOp xo = convert_operand(c, A, X.p, X.ld, A.n, int(X.cols));
  const SplitOp wo = convert_operand(c, A, W.p, W.ld, A.m, int(W.cols));
  if (c.measure) return;
  zero_f32(Y.p, Y.rows, Y.cols, Y.ld, c.s);
  zero_f32(Z.p, Z.rows, Z.cols, Z.ld, c.s);
  const bool fused = A.bf16 && dual_bf16_supported(int(X.cols), int(W.cols)) &&
                     (c.opt.band_mb == -2 ||
                      (c.opt.band_mb == 0 && (W.cols <= 64 || (W.cols <= 128 && X.cols <= 64))));
  if (fused) {
    TraceScope tr(c, LR_TRACE_VIEW_DUAL);
    DualBf16Args d;
    d.device = c.h->device;
    d.A = A.b();
    d.lda = A.ld;
    d.m = A.m;
    d.n = A.n;
    d.X = xo.bf;
    d.ldx = xo.ld;
    d.ell1 = int(X.cols);
    d.W = wo.bf;
    d.ldw = wo.ld;
    d.ell2 = int(W.cols);
    d.Y = Y.p;
    d.ldy = Y.ld;
    d.Z = Z.p;
    d.ldz = Z.ld;
    d.status = c.status;
    view_dual_bf16(d, c.s);
    return;
  }
  const int64_t rb = band_rows(A, c.opt.band_mb);
  for (int64_t r0 = 0; r0 < A.m; r0 += rb) {
    const int64_t rows = std::min(rb, A.m - r0);
    view_band(c, A, 0, X.p, X.ld, int(X.cols), Y.p, Y.ld, r0, rows, &xo);
    view_band(c, A, 1, W.p, W.ld, int(W.cols), Z.p, Z.ld, r0, rows, &wo);
  }
}

// Y = A X and Z = A^T Y (Section 6.8): each band of rows gives its slice of
// Y, which is converted and used for that band's share of A^T Y.
void view_chained(Ctx& c, const AMat& A, const Mat& X, Mat Y, Mat Z) {
  ArenaScope sc(c.ar);
  const SplitOp xo = convert_operand(c, A, X.p, X.ld, A.n, int(X.cols));
  SplitOp yo;
  yo.ld = A.bf16 ? round8(A.m) : round4(A.m);
  if (A.bf16) {
    yo.bf = c.ar.take<__nv_bfloat16>(size_t(yo.ld) * Y.cols);
  } else {
    yo.hi = c.ar.take<float>(size_t(yo.ld) * Y.cols);
    yo.lo = c.ar.take<float>(size_t(yo.ld) * Y.cols);
  }
  if (c.measure) return;
  zero_f32(Y.p, Y.rows, Y.cols, Y.ld, c.s);
  zero_f32(Z.p, Z.rows, Z.cols, Z.ld, c.s);
  const int64_t rb = band_rows(A, c.opt.band_mb);
  for (int64_t r0 = 0; r0 < A.m; r0 += rb) {
    const int64_t rows = std::min(rb, A.m - r0);
    view_band(c, A, 0, X.p, X.ld, int(X.cols), Y.p, Y.ld, r0, rows, &xo);
    if (A.bf16)
      f32_to_bf16(Y.p + r0, Y.ld, const_cast<__nv_bfloat16*>(yo.bf) + r0, nullptr, yo.ld, rows, Y.cols, c.s);
    else
      split_tf32(Y.p + r0, Y.ld, const_cast<float*>(yo.hi) + r0, const_cast<float*>(yo.lo) + r0, yo.ld, rows,
                 Y.cols, c.s);
    view_band(c, A, 1, Y.p, Y.ld, int(Y.cols), Z.p, Z.ld, r0, rows, &yo);
  }
}

// ------------------------------------------------- block CholeskyQR2
// In place thin QR of Y (m x L): column blocks of width <= 128; each block
// is projected out of the previous ones twice (BCGS2, the second pass
// restores the orthogonality lost in the first) and factorised by
// CholeskyQR2 (Gram in FP32 products with FP64 accumulation, Cholesky and
// triangular inverse in one CTA).  R (L x L FP64, ld L) receives the
// triangular factor when non-null: off-diagonal blocks are the summed
// projection coefficients, diagonal blocks R2 R1; ldr is its leading
// dimension (0: L).
// done: leading columns already orthonormal (the output of an earlier thin
// QR, as the first block of a Krylov basis is); they are kept as they are
// and only the remaining columns are projected and factorised.  R's columns
// before done are then the caller's (the earlier thin QR's factor) and are
// left as they are.
// Returns true when Y.bf is set and every factorised block left its BF16
// copy there (the single-kernel thin QR does; the other paths do not).
bool orth(Ctx& c, Mat Y, double* R, int done = 0, bool sharded = false, int ldr = 0) {
  const int64_t m = Y.rows;
  // sharded: Y holds this rank's rows; the caller checks the total
  LR_REQUIRE(sharded || m >= Y.cols, LR_ERR_SHAPE, "orth needs rows >= cols");
  if (ldr == 0) ldr = int(Y.cols);
  LR_REQUIRE(ldr >= Y.cols, LR_ERR_INVALID_ARG, "orth: ldr < columns");
  const int L = int(Y.cols) - done;
  if (L <= 0) return Y.bf != nullptr;
  ArenaScope sc(c.ar);
  const int nb = (L + kMaxBlock - 1) / kMaxBlock;
  const int wmax = (L + nb - 1) / nb;
  float* T = c.ar.take<float>(size_t(m) * wmax);
  double* G64 = c.ar.take<double>(size_t(std::max(L + done, wmax)) * wmax);
  float* C32 = c.ar.take<float>(size_t(L + done) * wmax);
  float* Rinv = c.ar.take<float>(size_t(wmax) * wmax);
  double* R2 = c.ar.take<double>(size_t(wmax) * wmax);  // factor of a later pass
  int* flags = c.ar.take<int>(size_t(nb));
  double* tscratch = c.ar.take<double>(orth_tc_scratch_doubles(wmax));
  if (c.measure) return false;
  bool all_bf = Y.bf != nullptr;
  TraceScope tr(c, LR_TRACE_ORTH);
  if (R) LR_CHECK_CUDA(cudaMemsetAsync(R + int64_t(done) * ldr, 0, size_t(L) * ldr * sizeof(double), c.s));
  LR_CHECK_CUDA(cudaMemsetAsync(flags, 0, sizeof(int) * nb, c.s));
  int c0 = done;
  for (int b = 0; b < nb; ++b) {
    const int w = L / nb + (b < L % nb ? 1 : 0);
    float* Yb = Y.col(c0);
    int* more = flags + b;
    if (c0 > 0) {
      for (int pass = 0; pass < 2; ++pass) {
        gram64(c, c0, w, m, Y.p, Y.ld, Yb, Y.ld, G64, c0);          // C = Q_prev^T Y_b
        if (sharded) allreduce(c, G64, int64_t(c0) * w, LR_F64);    // rows split over the ranks
        f64_to_f32(G64, c0, C32, c0, c0, w, c.s);
        gemm(c, m, w, c0, false, Y.p, Y.ld, false, C32, c0, Yb, Y.ld, -1.f, 1.f);  // Y_b -= Q_prev C
        if (R) add_block_f64(R, ldr, 0, c0, G64, c0, c0, w, c.s);
      }
    }
    // CholeskyQR2 with a breakdown-triggered shift (shifted CholeskyQR3,
    // Fukaya et al. 2020): pass 1 is plain, or shifted when the plain
    // Cholesky breaks down -- which happens in FP32 once kappa(Y_b) nears
    // 1e3 -- and then flags a third pass that the device runs only if set.
    // With opts.shifted_fallback (rank-deficient input: a sketch of a matrix
    // of rank below the block's width) a flagged block takes four passes:
    // shifted, shifted again (the directions outside the column space are
    // still below the FP32 Cholesky's resolution after one shift), then two
    // plain passes that make every column orthonormal; Y_b = Q R holds
    // exactly through shifted passes, so R stays the triangular factor.
    // Passes alternate Y_b -> T -> Y_b -> T (-> Y_b); R_bb = R_last ... R_1.
    const bool robust = c.opt.shifted_fallback != 0;
    double* Rbb = R ? R + c0 + int64_t(c0) * ldr : nullptr;
    if (!sharded && orth_tc_supported(m, w)) {
      // all CholeskyQR passes of the block in one kernel (orth_tc.cu)
      orth_tc(Yb, Y.ld, m, w, Rbb, ldr, tscratch, robust ? 1 : 0, c.status, c.h->device, c.s,
              Y.bf ? Y.bf + int64_t(c0) * Y.ldbf : nullptr, Y.ldbf);
      c0 += w;
      continue;
    }
    all_bf = false;  // this block takes the separate kernels
    // pass 1: Y_b -> T
    gram64(c, w, w, m, Yb, Y.ld, Yb, Y.ld, G64, w);
    if (sharded) allreduce(c, G64, int64_t(w) * w, LR_F64);
    chol_inv(G64, w, Rinv, w, Rbb, ldr, true, CHOL_SHIFT_IF_NEEDED, more, c.status, c.s);
    gemm(c, m, w, w, false, Yb, Y.ld, false, Rinv, w, T, m);
    // pass 2: T -> Y_b (R_bb <- R_2 R_bb by a separate many-CTA product)
    gram64(c, w, w, m, T, m, T, m, G64, w);
    if (sharded) allreduce(c, G64, int64_t(w) * w, LR_F64);
    chol_inv(G64, w, Rinv, w, Rbb ? R2 : nullptr, w, true, robust ? CHOL_SHIFT_IF_FLAGGED : CHOL_PLAIN, more,
             c.status, c.s);
    if (Rbb) upper_product(R2, w, Rbb, ldr, w, nullptr, c.s);
    gemm(c, m, w, w, false, T, m, false, Rinv, w, Yb, Y.ld);
    // pass 3 (only after a shifted pass 1): Y_b -> T -> Y_b
    gram64(c, w, w, m, Yb, Y.ld, Yb, Y.ld, G64, w, more);
    if (sharded) allreduce(c, G64, int64_t(w) * w, LR_F64);
    chol_inv(G64, w, Rinv, w, Rbb ? R2 : nullptr, w, true, CHOL_IF_FLAGGED, more, c.status, c.s);
    if (Rbb) upper_product(R2, w, Rbb, ldr, w, more, c.s);
    gemm(c, m, w, w, false, Yb, Y.ld, false, Rinv, w, T, m, 1.f, 0.f, more);
    if (robust) {
      // pass 4: T -> Y_b
      gram64(c, w, w, m, T, m, T, m, G64, w, more);
      if (sharded) allreduce(c, G64, int64_t(w) * w, LR_F64);
      chol_inv(G64, w, Rinv, w, Rbb ? R2 : nullptr, w, true, CHOL_IF_FLAGGED, more, c.status, c.s);
      if (Rbb) upper_product(R2, w, Rbb, ldr, w, more, c.s);
      gemm(c, m, w, w, false, T, m, false, Rinv, w, Yb, Y.ld, 1.f, 0.f, more);
    } else {
      copy_f32(T, m, Yb, Y.ld, m, w, c.s, more);
    }
    c0 += w;
  }
  return all_bf;
}

// ------------------------------------------------ triangular inverse
// X = R^{-1} (FP32 n x n, ld n) for an upper-triangular FP64 R (ld n) of any
// width: diagonal blocks of <= 128 are inverted in one CTA each, the blocks
// above the diagonal follow from X_IJ = -X_II (sum_{K=I+1..J} R_IK X_KJ),
// computed block column by block column, bottom up, as small GEMMs.
void tri_inv_any(Ctx& c, const double* R, int n, float* X) {
  ArenaScope sc(c.ar);
  const int nb = (n + kMaxBlock - 1) / kMaxBlock;
  const int b = (n + nb - 1) / nb;
  float* R32 = c.ar.take<float>(size_t(n) * n);
  float* T = c.ar.take<float>(size_t(b) * b);
  if (c.measure) return;
  if (nb == 1) {
    tri_inv(R, n, n, X, n, c.status, c.s);
    return;
  }
  auto start = [&](int I) { return I * b; };
  auto size = [&](int I) { return std::min(b, n - I * b); };
  r_to_f32(R, n, n, R32, n, false, c.s);
  LR_CHECK_CUDA(cudaMemsetAsync(X, 0, sizeof(float) * size_t(n) * n, c.s));
  for (int J = 0; J < nb; ++J)
    tri_inv(R + start(J) + int64_t(start(J)) * n, n, size(J), X + start(J) + int64_t(start(J)) * n, n, c.status, c.s);
  for (int J = 1; J < nb; ++J)
    for (int I = J - 1; I >= 0; --I) {
      const int k0 = start(I + 1), kl = start(J) + size(J) - k0;
      // T = R[I, I+1..J] X[I+1..J, J]
      gemm(c, size(I), size(J), kl, false, R32 + start(I) + int64_t(k0) * n, n, false,
           X + k0 + int64_t(start(J)) * n, n, T, size(I));
      // X_IJ = -X_II T
      gemm(c, size(I), size(J), size(I), false, X + start(I) + int64_t(start(I)) * n, n, false, T, size(I),
           X + start(I) + int64_t(start(J)) * n, n, -1.f, 0.f);
    }
}

// --------------------------------------------------------- core SVD
// R (n x n upper, FP64) = Left diag(S) Right^T, outputs FP32 n x n.
// One-sided Jacobi runs on R^T: the rows of R are graded for the bases
// built here (earlier Krylov/subspace directions carry larger norms), which
// makes the columns of R^T converge in fewer sweeps.  R^T = Um S Vm^T gives
// Left = Vm (accumulated rotations) and Right = Um (normalised columns).
void core_svd(Ctx& c, const double* R, int n, float* Left, float* Right, float* S) {
  ArenaScope sc(c.ar);
  float* M = c.ar.take<float>(size_t(n) * n);
  if (c.measure) return;
  TraceScope tr(c, LR_TRACE_CORE_SVD);
  r_to_f32(R, n, n, M, n, true, c.s);
  jacobi_svd(M, n, n, n, Right, n, Left, n, S, nullptr, c.status, c.s);
}

struct Outs {
  Mat U, V;
  void* S = nullptr;
};

void write_outputs(Ctx& c, const Mat& Qleft, const float* Lsel, const Mat& Qright, const float* Rsel, int Lk,
                   const float* Sv, int k, Outs& o) {
  if (c.measure) return;
  gemm(c, o.U.rows, k, Lk, false, Qleft.p, Qleft.ld, false, Lsel, Lk, o.U.p, o.U.ld);
  gemm(c, o.V.rows, k, Lk, false, Qright.p, Qright.ld, false, Rsel, Lk, o.V.p, o.V.ld);
  fix_signs(o.U.p, o.U.ld, o.U.rows, o.V.p, o.V.ld, o.V.rows, k, c.s);
  LR_CHECK_CUDA(cudaMemcpyAsync(o.S, Sv, sizeof(float) * k, cudaMemcpyDeviceToDevice, c.s));
}

// ------------------------------------------------------------ Alg. 2
// The views of A a schedule uses: of a device-resident A by default; the
// host-streamed form supplies its own.
struct Viewer {
  std::function<void(Ctx&, const Mat&, Mat)> range;    // Y = A X
  std::function<void(Ctx&, const Mat&, Mat)> corange;  // Z = A^T W
};

void run_subspace(Ctx& c, const AMat& A, int k, int ell, int v, const Mat& Om, Outs& o, const Viewer* vw = nullptr) {
  ArenaScope sc(c.ar);
  Mat Qc{c.ar.take<float>(size_t(A.m) * ell), A.m, ell, A.m};
  Mat Qr{c.ar.take<float>(size_t(A.n) * ell), A.n, ell, A.n};
  double* Rc = c.ar.take<double>(size_t(ell) * ell);
  double* Rr = c.ar.take<double>(size_t(ell) * ell);
  float* W = c.ar.take<float>(size_t(ell) * ell);
  float* Vj = c.ar.take<float>(size_t(ell) * ell);
  float* Sv = c.ar.take<float>(size_t(ell));
  Mat cur = Om;  // Q_r = Omega (Alg. 2 starts from the raw Gaussian)
  for (int j = 1; j <= v; ++j) {
    if (j % 2 == 1) {
      if (vw) vw->range(c, cur, Qc);
      else view_range(c, A, cur, Qc, j == v);    // A Q_r
      orth(c, Qc, Rc);                           // [Q_c, R_c] = qr(A Q_r)
    } else {
      if (vw) vw->corange(c, Qc, Qr);
      else view_corange(c, A, Qc, Qr, j == v);   // A^T Q_c
      orth(c, Qr, Rr);                           // [Q_r, R_r] = qr(A^T Q_c)
      cur = Qr;
    }
  }
  if (v % 2 == 0) {
    // R_r = V^ L U^T: left vectors of R_r give V, right vectors give U.
    core_svd(c, Rr, ell, W, Vj, Sv);
    write_outputs(c, Qc, Vj, Qr, W, ell, Sv, k, o);
  } else {
    // R_c = U^ L V^T
    core_svd(c, Rc, ell, W, Vj, Sv);
    write_outputs(c, Qc, W, Qr, Vj, ell, Sv, k, o);
  }
}

// ------------------------------------------------ Alg. 2, rows over ranks
// Rank g holds the row block A_g; Q_c is split by rows like A, Q_r (n x ell)
// is replicated.  Range views and every product with Q_c are local; the
// thin QR of Q_c sums its Grams over the ranks (orth's sharded form: the
// sums are identical on every rank, so is each Cholesky factor); a co-range
// view sums the partials A_g^T Q_c,g.  The replicated results of kernels
// that reduce with atomics (the thin QR of Q_r, the product for V) and the
// core SVD are then taken from rank 0, so every rank holds the same bits.
// The sign rule looks at the peak entry of each u_i over all ranks.
void run_subspace_sharded(Ctx& c, const AMat& A, int k, int ell, int v, const Mat& Om, Outs& o) {
  ArenaScope sc(c.ar);
  const int64_t n = A.n;
  Mat Qc{c.ar.take<float>(size_t(A.m) * ell), A.m, ell, A.m};
  Mat Qr{c.ar.take<float>(size_t(n) * ell), n, ell, n};
  float* Vt = c.ar.take<float>(size_t(n) * k);
  double* Rc = c.ar.take<double>(size_t(ell) * ell);
  double* Rr = c.ar.take<double>(size_t(ell) * ell);
  float* W = c.ar.take<float>(size_t(ell) * ell);
  float* Vj = c.ar.take<float>(size_t(ell) * ell);
  float* Sv = c.ar.take<float>(size_t(ell));
  Mat cur = Om;
  for (int j = 1; j <= v; ++j) {
    if (j % 2 == 1) {
      view_range(c, A, cur, Qc, j == v);           // A_g Q_r
      orth(c, Qc, Rc, 0, true);                    // [Q_c, R_c] = qr(A Q_r), Grams summed
    } else {
      view_corange(c, A, Qc, Qr, j == v);          // A_g^T Q_c,g
      allreduce(c, Qr.p, n * ell, LR_F32);         // A^T Q_c = sum_g A_g^T Q_c,g
      orth(c, Qr, Rr);                             // [Q_r, R_r] = qr(A^T Q_c)
      broadcast0(c, Qr.p, n * ell, LR_F32);
      broadcast0(c, Rr, int64_t(ell) * ell, LR_F64);
      cur = Qr;
    }
  }
  core_svd(c, v % 2 == 0 ? Rr : Rc, ell, W, Vj, Sv);
  if (c.measure) return;
  broadcast0(c, W, int64_t(ell) * ell, LR_F32);
  broadcast0(c, Vj, int64_t(ell) * ell, LR_F32);
  broadcast0(c, Sv, ell, LR_F32);
  // v even: R_r = V^ L U^^T (U from the right vectors); v odd: R_c = U^ L V^^T
  const float* Lsel = v % 2 == 0 ? Vj : W;
  const float* Rsel = v % 2 == 0 ? W : Vj;
  gemm(c, o.U.rows, k, ell, false, Qc.p, Qc.ld, false, Lsel, ell, o.U.p, o.U.ld);
  gemm(c, n, k, ell, false, Qr.p, Qr.ld, false, Rsel, ell, Vt, n);
  broadcast0(c, Vt, n * k, LR_F32);
  // Q_r is dead now: its storage holds the world x k peak entries (world <= n)
  const int world = c.comm ? c.comm->world : 1, rank = c.comm ? c.comm->rank : 0;
  float* peaks = Qr.p;
  LR_CHECK_CUDA(cudaMemsetAsync(peaks, 0, sizeof(float) * size_t(world) * k, c.s));
  col_peaks(o.U.p, o.U.ld, o.U.rows, peaks, rank, k, c.s);
  allreduce(c, peaks, int64_t(world) * k, LR_F32);
  flip_by_peaks(o.U.p, o.U.ld, o.U.rows, Vt, n, n, peaks, world, k, c.s);
  copy_f32(Vt, n, o.V.p, o.V.ld, n, k, c.s);
  LR_CHECK_CUDA(cudaMemcpyAsync(o.S, Sv, sizeof(float) * k, cudaMemcpyDeviceToDevice, c.s));
}

// The ranks agree on n, k, p, v and A's type (sum_g x_g = W x and
// sum_g x_g^2 = W x^2 hold for the local x only when every x_g equals it);
// returns the total row count.
int64_t sharded_agree(Ctx& c, const AMat& A, int k, int p, int v) {
  ArenaScope sc(c.ar);
  double* d = c.ar.take<double>(16);
  const double x[5] = {double(A.n), double(k), double(p), double(v), A.bf16 ? 1.0 : 0.0};
  double h[12] = {double(A.m), 1.0};
  for (int i = 0; i < 5; ++i) {
    h[2 + 2 * i] = x[i];
    h[3 + 2 * i] = x[i] * x[i];
  }
  LR_CHECK_CUDA(cudaMemcpyAsync(d, h, sizeof(h), cudaMemcpyHostToDevice, c.s));
  allreduce(c, d, 12, LR_F64);
  LR_CHECK_CUDA(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, c.s));
  LR_CHECK_CUDA(cudaStreamSynchronize(c.s));
  const double W = double(c.comm->world);
  LR_REQUIRE(h[1] == W, LR_ERR_INVALID_ARG, "the communicator's all-reduce does not sum over comm->world ranks");
  for (int i = 0; i < 5; ++i)
    LR_REQUIRE(h[2 + 2 * i] == W * x[i] && h[3 + 2 * i] == W * x[i] * x[i], LR_ERR_INVALID_ARG,
               "the ranks disagree on n, k, p, v or the type of A");
  return int64_t(h[0]);
}

// ---------------------------------------------------- Algs. 3, 4, 5
// An operator J (rows x cols) given by the caller's callback, as the views
// of the schedules see it; transposed when `t` (the views of J^T).
Viewer op_viewer(const lr_operator* J, bool t) {
  auto call = [J](Ctx& c, int transpose, const Mat& X, Mat Y) {
    if (c.measure) return;
    const int rc = J->apply(J->ctx, transpose, X.p, X.ld, X.cols, Y.p, Y.ld, c.s);
    LR_REQUIRE(rc == 0, LR_ERR_INVALID_ARG, "the operator's callback failed (returned " + std::to_string(rc) + ")");
    LR_CHECK_CUDA(cudaGetLastError());
  };
  Viewer vw;
  vw.range = [call, t](Ctx& c, const Mat& X, Mat Y) { call(c, t ? 1 : 0, X, Y); };
  vw.corange = [call, t](Ctx& c, const Mat& W, Mat Z) { call(c, t ? 0 : 1, W, Z); };
  return vw;
}

// Alg. 3 on an operator B (rows_b x cols_b, views vw), v >= 1 views from
// Q_r = Omega (cols_b x ell): odd j Q_c = qr(B Q_r) into Qc (rows_b x ell),
// even j Q_r = qr(B^T Q_c) into Qr (cols_b x ell); returns the last one.
Mat run_qrqc(Ctx& c, const Viewer& vw, const Mat& Om, int v, Mat Qc, Mat Qr) {
  Mat cur = Om;
  for (int j = 1; j <= v; ++j) {
    if (j % 2 == 1) {
      vw.range(c, cur, Qc);
      orth(c, Qc, nullptr);
    } else {
      vw.corange(c, Qc, Qr);
      orth(c, Qr, nullptr);
      cur = Qr;
    }
  }
  return v % 2 == 0 ? Qr : Qc;
}

// The columns of V (n x k) with the sign that makes each one's largest entry positive.
void sign_columns(Ctx& c, Mat V, int k) {
  if (!c.measure) fix_signs(V.p, V.ld, V.rows, V.p, 0, 0, k, c.s);
}

// Alg. 4: J (m x n) by callback; Omega n x ell (v even) or m x ell (v odd).
void run_nystrom(Ctx& c, const lr_operator* J, int k, int ell, int v, const Mat& Om, Mat Vout, float* lam2) {
  ArenaScope sc(c.ar);
  const int64_t m = J->rows, n = J->cols;
  const int64_t mx = std::max(m, n);
  Mat Qa{c.ar.take<float>(size_t(mx) * ell), 0, ell, mx};  // Q_c of the start operator
  Mat Qr{c.ar.take<float>(size_t(n) * ell), n, ell, n};
  Mat Y{c.ar.take<float>(size_t(m) * ell), m, ell, m};
  Mat Yr{c.ar.take<float>(size_t(n) * ell), n, ell, n};
  Mat Ft{c.ar.take<float>(size_t(n) * ell), n, ell, n};
  double* B = c.ar.take<double>(size_t(ell) * ell);
  double* Rf = c.ar.take<double>(size_t(ell) * ell);
  double* ssq = c.ar.take<double>(1);
  float* Rinv = c.ar.take<float>(size_t(ell) * ell);
  float* L = c.ar.take<float>(size_t(ell) * ell);
  float* Rt = c.ar.take<float>(size_t(ell) * ell);
  float* Sv = c.ar.take<float>(size_t(ell));
  const Viewer vj = op_viewer(J, false), vt = op_viewer(J, true);
  if (c.measure) {
    orth(c, Mat{nullptr, mx, ell, mx}, nullptr);
    core_svd(c, nullptr, ell, nullptr, nullptr, nullptr);
    gemm(c, n, ell, ell, false, nullptr, n, false, nullptr, ell, nullptr, n);
    return;
  }
  // Q_r: orth(Omega) (v = 2), Alg. 3 on J (v even) or on J^T (v odd), v - 2 views
  Mat q;
  if (v == 2) {
    copy_f32(Om.p, Om.ld, Qr.p, Qr.ld, n, ell, c.s);
    orth(c, Qr, nullptr);
    q = Qr;
  } else if (v % 2 == 0) {
    Qa.rows = m;
    Qa.ld = m;
    q = run_qrqc(c, vj, Om, v - 2, Qa, Qr);
  } else {  // J^T: its Q_c lives in the n-dimensional space
    Mat qc{Qr.p, n, ell, n};
    Mat qr2{Qa.p, m, ell, m};
    q = run_qrqc(c, vt, Om, v - 2, qc, qr2);
  }
  vj.range(c, q, Y);                                   // J Q_r
  vj.corange(c, Y, Yr);                                // Y_r = J^T (J Q_r)
  constexpr float kEps32 = 1.0f / 8388608.0f;          // 2^-23
  sumsq_f32(Yr.p, Yr.ld, n, ell, ssq, c.s);
  shift_add_f32(Yr.p, Yr.ld, q.p, q.ld, n, ell, ssq, kEps32, c.s);    // Y_r += nu Q_r
  gram64(c, ell, ell, n, q.p, q.ld, Yr.p, Yr.ld, B, ell);            // B = Q_r^T Y_r
  symmetrize_f64(B, ell, c.s);                                         // (B + B^T) / 2
  chol_inv(B, ell, Rinv, ell, nullptr, 0, true, CHOL_PLAIN, nullptr, c.status, c.s);  // C_L = R^T
  gemm(c, n, ell, ell, false, Yr.p, Yr.ld, false, Rinv, ell, Ft.p, Ft.ld);          // F^T = Y_r R^{-1}
  orth(c, Ft, Rf);                                     // F^T = Q_f R_f
  core_svd(c, Rf, ell, L, Rt, Sv);                     // R_f = L diag(S) Rt^T
  gemm(c, n, k, ell, false, Ft.p, Ft.ld, false, L, ell, Vout.p, Vout.ld);  // V = Q_f L_k
  sign_columns(c, Vout, k);
  sq_shift(Sv, k, ssq, kEps32, lam2, c.s);             // max(S^2 - nu, 0)
}

// Alg. 5: Q_r from v - 1 views (Alg. 3 on J^T from an m x ell Omega for
// even v, on J from an n x ell Omega for odd v), B_c = J Q_r, EVD of
// B_c^T B_c through B_c = Q R, R = L diag(S) Rt^T: eigenvectors Q_r Rt.
void run_pinched(Ctx& c, const lr_operator* J, int k, int ell, int v, const Mat& Om, Mat Vout, float* lam2) {
  ArenaScope sc(c.ar);
  const int64_t m = J->rows, n = J->cols;
  const int64_t mx = std::max(m, n);
  Mat Qa{c.ar.take<float>(size_t(mx) * ell), 0, ell, mx};
  Mat Qr{c.ar.take<float>(size_t(n) * ell), n, ell, n};
  Mat Bc{c.ar.take<float>(size_t(m) * ell), m, ell, m};
  double* Rb = c.ar.take<double>(size_t(ell) * ell);
  float* L = c.ar.take<float>(size_t(ell) * ell);
  float* Rt = c.ar.take<float>(size_t(ell) * ell);
  float* Sv = c.ar.take<float>(size_t(ell));
  const Viewer vj = op_viewer(J, false), vt = op_viewer(J, true);
  if (c.measure) {
    orth(c, Mat{nullptr, mx, ell, mx}, nullptr);
    core_svd(c, nullptr, ell, nullptr, nullptr, nullptr);
    return;
  }
  Mat q;
  if (v % 2 == 0) {  // Alg. 3 on J^T, v - 1 (odd) views: its Q_c, n-dimensional
    Mat qc{Qr.p, n, ell, n};
    Mat qr2{Qa.p, m, ell, m};
    q = run_qrqc(c, vt, Om, v - 1, qc, qr2);
  } else {
    Qa.rows = m;
    Qa.ld = m;
    q = run_qrqc(c, vj, Om, v - 1, Qa, Qr);
  }
  vj.range(c, q, Bc);                                  // B_c = J Q_r
  orth(c, Bc, Rb);                                     // B_c = Q R
  core_svd(c, Rb, ell, L, Rt, Sv);                     // R = L diag(S) Rt^T
  gemm(c, n, k, ell, false, q.p, q.ld, false, Rt, ell, Vout.p, Vout.ld);  // V = Q_r Rt_k
  sign_columns(c, Vout, k);
  sq_shift(Sv, k, nullptr, 0.f, lam2, c.s);            // S^2
}

// ------------------------------------------------------------ Alg. 9
// first_range, when given, computes the first view Y = A Omega in place of
// view_range (the host-buffer entry point overlaps it with A's copy).
void run_krylov(Ctx& c, const AMat& A, int k, int ell, int v, const Mat& Om, Outs& o,
                const std::function<void(Ctx&, const Mat&, Mat)>* first_range = nullptr) {
  ArenaScope sc(c.ar);
  const bool even = v % 2 == 0;
  const int nb = even ? v / 2 : (v - 1) / 2;
  const int Lk = nb * ell;
  const int64_t kdim = even ? A.m : A.n, odim = even ? A.n : A.m;
  Mat K{c.ar.take<float>(size_t(kdim) * Lk), kdim, Lk, kdim};
  Mat Tb{c.ar.take<float>(size_t(odim) * ell), odim, ell, odim};
  Mat F{c.ar.take<float>(size_t(odim) * Lk), odim, Lk, odim};  // final view
  double* Rf = c.ar.take<double>(size_t(Lk) * Lk);
  float* W = c.ar.take<float>(size_t(Lk) * Lk);
  float* Vj = c.ar.take<float>(size_t(Lk) * Lk);
  float* Sv = c.ar.take<float>(size_t(Lk));
  if (A.bf16) {
    // the thin QRs leave the BF16 copies the next BF16 views read
    K.ldbf = round8(kdim);
    K.bf = c.ar.take<__nv_bfloat16>(size_t(K.ldbf) * Lk);
    Tb.ldbf = round8(odim);
    Tb.bf = c.ar.take<__nv_bfloat16>(size_t(Tb.ldbf) * ell);
  }
  // a view of A with X: from X's BF16 copy when one is valid
  auto view = [&](const Mat& X, Mat Y, int mode, bool valid_bf, bool last) {
    if (!(A.bf16 && valid_bf && X.bf) || (last && c.opt.split_last)) {
      if (mode == 0) view_range(c, A, X, Y, last);
      else view_corange(c, A, X, Y, last);
      return;
    }
    if (!c.measure) zero_f32(Y.p, Y.rows, Y.cols, Y.ld, c.s);
    SplitOp pre;
    pre.bf = X.bf;
    pre.ld = X.ldbf;
    view_band(c, A, mode, X.p, X.ld, int(X.cols), Y.p, Y.ld, 0, A.m, &pre);
  };
  // The final view multiplies A (or A^T) by the orthonormal basis of K,
  // whose first block is the first inner thin-QR output, kept as it is (the
  // later blocks are projected against it).  Its product with A^T (A) is
  // the next inner view's output, so that view writes F's first block, whose
  // thin QR (with its R factor) then serves both as that inner step's and
  // as the first block of F's; the final view runs over K's other blocks.
  // Not with split_last, whose final view is the more accurate two-term one
  // over all of K.
  const bool reuse = !c.opt.split_last && nb >= 2;
  Mat F0{F.p, odim, ell, odim};  // F's first block
  if (A.bf16 && reuse) {
    F0.ldbf = round8(odim);
    F0.bf = c.ar.take<__nv_bfloat16>(size_t(F0.ldbf) * ell);
  }
  Mat prev = Om;
  bool prev_bf = false;
  bool k0_bf = false;  // K's first block has its BF16 copy
  int blk = 0;
  for (int j = 1; j <= v - 1; ++j) {
    const bool odd = j % 2 == 1;
    const bool in_k = odd == even;
    const bool f_blk = reuse && !in_k && blk == 1;  // A^T (A) times K's first block
    Mat out = in_k ? Mat{K.col(int64_t(blk) * ell), kdim, ell, kdim,
                         K.bf ? K.bf + int64_t(blk) * ell * K.ldbf : nullptr, K.ldbf}
                   : f_blk ? F0 : Tb;
    if (j == 1 && first_range) (*first_range)(c, prev, out);
    else view(prev, out, odd ? 0 : 1, prev_bf, false);
    prev_bf = false;
    if (j < v - 1) prev_bf = orth(c, out, f_blk ? Rf : nullptr, 0, false, Lk);
    if (in_k && blk == 0) k0_bf = prev_bf;
    if (in_k) ++blk;
    prev = out;
  }
  // Q = qr(K); K's first block is already orthonormal (the qr of an inner
  // view) unless it is the raw last block itself
  const bool rest_bf = orth(c, K, nullptr, nb >= 2 ? ell : 0);
  const bool K_bf = rest_bf && (nb < 2 || k0_bf);
  // the final view: all of K, or all but its first block
  const int f0 = reuse ? ell : 0;
  const Mat Kf{K.col(f0), kdim, Lk - f0, kdim, K.bf ? K.bf + int64_t(f0) * K.ldbf : nullptr, K.ldbf};
  const Mat Ff{F.col(f0), odim, Lk - f0, odim};
  const bool Kf_bf = reuse ? rest_bf : K_bf;
  if (even) {
    view(Kf, Ff, 1, Kf_bf, true);        // A^T Q_c
    orth(c, F, Rf, f0);                  // [Q_r, R_r]
    core_svd(c, Rf, Lk, W, Vj, Sv);      // R_r = V^ L U^T
    write_outputs(c, K, Vj, F, W, Lk, Sv, k, o);
  } else {
    view(Kf, Ff, 0, Kf_bf, true);        // A Q_r
    orth(c, F, Rf, f0);                  // [Q_c, R_c]
    core_svd(c, Rf, Lk, W, Vj, Sv);      // R_c = U^ L V^T
    write_outputs(c, F, W, K, Vj, Lk, Sv, k, o);
  }
}

// ------------------------------------------------------- Section 7.3
void run_krylov_rowwise(Ctx& c, const AMat& A, int k, int ell, int v, const Mat& Om, Outs& o) {
  ArenaScope sc(c.ar);
  const int Lk = (v - 1) * ell;
  Mat K{c.ar.take<float>(size_t(A.n) * Lk), A.n, Lk, A.n};
  Mat Y{c.ar.take<float>(size_t(A.m) * ell), A.m, ell, A.m};
  Mat Z{c.ar.take<float>(size_t(A.n) * ell), A.n, ell, A.n};
  double* Rc = c.ar.take<double>(size_t(ell) * ell);
  float* Ri = c.ar.take<float>(size_t(ell) * ell);
  Mat F{c.ar.take<float>(size_t(A.m) * Lk), A.m, Lk, A.m};
  double* Rf = c.ar.take<double>(size_t(Lk) * Lk);
  float* W = c.ar.take<float>(size_t(Lk) * Lk);
  float* Vj = c.ar.take<float>(size_t(Lk) * Lk);
  float* Sv = c.ar.take<float>(size_t(Lk));
  // The last view A Q_r starts with A times K's first block, which the
  // second chained view forms as its Y: that view writes F's first block,
  // whose thin QR (with its R) serves both that step and F's QR, and the
  // last view runs over K's later blocks (not with split_last, whose last
  // view is the more accurate two-term one over all of K).
  const bool reuse = !c.opt.split_last && v >= 3;
  Mat x = Om;
  for (int i = 1; i <= v - 1; ++i) {
    const bool f_blk = reuse && i == 2;  // Y = A K_0, F's first block
    Mat Yi = f_blk ? Mat{F.p, A.m, ell, A.m} : Y;
    view_chained(c, A, x, Yi, Z);        // Y = A X, Z = A^T Y from one read
    orth(c, Yi, f_blk ? Rf : Rc, 0, false, f_blk ? Lk : 0);  // Y = Q_c R_c
    if (f_blk && !c.measure)
      LR_CHECK_CUDA(cudaMemcpy2DAsync(Rc, size_t(ell) * sizeof(double), Rf, size_t(Lk) * sizeof(double),
                                      size_t(ell) * sizeof(double), size_t(ell), cudaMemcpyDeviceToDevice, c.s));
    Mat blk{K.col(int64_t(i - 1) * ell), A.n, ell, A.n};
    tri_inv_any(c, Rc, ell, Ri);
    if (!c.measure) {
      gemm(c, A.n, ell, ell, false, Z.p, Z.ld, false, Ri, ell, blk.p, blk.ld);  // A^T Q_c = Z R_c^{-1}
    }
    if (i < v - 1) orth(c, blk, nullptr);
    x = blk;
  }
  orth(c, K, nullptr, v >= 3 ? ell : 0);  // Q_r = qr(K_r), first block already orthonormal
  const int f0 = reuse ? ell : 0;
  view_range(c, A, Mat{K.col(f0), A.n, Lk - f0, A.n}, Mat{F.col(f0), A.m, Lk - f0, A.m}, true);  // A Q_r
  orth(c, F, Rf, f0);
  core_svd(c, Rf, Lk, W, Vj, Sv);        // R_c = U^ L V^T
  write_outputs(c, F, W, K, Vj, Lk, Sv, k, o);
}

// ------------------------------------------------------- Section 6.8
void run_rowwise_qb(Ctx& c, const AMat& A, int k, int ell, const Mat& Om, Outs& o) {
  ArenaScope sc(c.ar);
  Mat Y{c.ar.take<float>(size_t(A.m) * ell), A.m, ell, A.m};
  Mat Z{c.ar.take<float>(size_t(A.n) * ell), A.n, ell, A.n};
  Mat Bt{c.ar.take<float>(size_t(A.n) * ell), A.n, ell, A.n};
  double* Rc = c.ar.take<double>(size_t(ell) * ell);
  double* Rb = c.ar.take<double>(size_t(ell) * ell);
  float* Ri = c.ar.take<float>(size_t(ell) * ell);
  float* W = c.ar.take<float>(size_t(ell) * ell);
  float* Vj = c.ar.take<float>(size_t(ell) * ell);
  float* Sv = c.ar.take<float>(size_t(ell));
  view_chained(c, A, Om, Y, Z);          // Y_c = A Omega, Y^_r = A^T Y_c
  orth(c, Y, Rc);                        // [Q_c, R_c] = qr(Y_c)
  tri_inv_any(c, Rc, ell, Ri);
  gemm(c, A.n, ell, ell, false, Z.p, Z.ld, false, Ri, ell, Bt.p, Bt.ld);  // B^T = Y^_r R_c^{-1}
  orth(c, Bt, Rb);                       // B^T = Q_b R_b
  core_svd(c, Rb, ell, W, Vj, Sv);       // R_b = V^ L U^T
  write_outputs(c, Y, Vj, Bt, W, ell, Sv, k, o);
}

// ------------------------------------------------------------ Alg. 7
// `sketch` fills Y (m x ell1) = A Omega and Z (n x ell2) = A^T Psi; by
// default from one read of a device-resident A (view_dual), for the
// host-streamed form from column panels copied in from pinned host memory.
using Sketcher = std::function<void(Ctx&, Mat, Mat)>;

// The minimum-variance l_c of Section 6.6 from the sketches Y = A Omega
// (m x ell1) and Z = A^T Psi (n x ell2), left intact.  For every trial
// l_c = 0 .. l1 the leading k singular values of X(l_c) = R^^{-1} Q^^T Z^T
// are found, where Q^ R^ = qr(Psi^T Q_c[:, :k + l_c]) and Q_c holds the left
// singular vectors of Y.  Since Z = Q_z R_z, X(l_c) Q_z = R^^{-1} Q^^T R_z^T
// has the same singular values, so each trial works on small matrices only:
// X^T = R_z Q^ R^^{-T} (ell2 x (k + l_c)).  A small kernel then picks the
// l_c whose locally normalised spectra vary least; the choice sizes the rest
// of Alg. 7, so it is read back (one stream synchronisation).
int minvar_lc(Ctx& c, const AMat& A, int k, const Mat& Y, const Mat& Z, const Mat& Psi) {
  ArenaScope sc(c.ar);
  const int ell1 = int(Y.cols), ell2 = int(Z.cols), l1 = ell1 - k;
  Mat Yc{c.ar.take<float>(size_t(A.m) * ell1), A.m, ell1, A.m};
  Mat Zc{c.ar.take<float>(size_t(A.n) * ell2), A.n, ell2, A.n};
  double* Rc = c.ar.take<double>(size_t(ell1) * ell1);
  double* Rz = c.ar.take<double>(size_t(ell2) * ell2);
  float* Wc = c.ar.take<float>(size_t(ell1) * ell1);
  float* Vc = c.ar.take<float>(size_t(ell1) * ell1);
  float* Sc = c.ar.take<float>(size_t(ell1));
  Mat Qf{c.ar.take<float>(size_t(A.m) * ell1), A.m, ell1, A.m};
  double* B64 = c.ar.take<double>(size_t(ell2) * ell1);
  float* B = c.ar.take<float>(size_t(ell2) * ell1);
  float* Rz32 = c.ar.take<float>(size_t(ell2) * ell2);
  float* Bl = c.ar.take<float>(size_t(ell2) * ell1);
  double* Rl = c.ar.take<double>(size_t(ell1) * ell1);
  float* Ri = c.ar.take<float>(size_t(ell1) * ell1);
  float* M1 = c.ar.take<float>(size_t(ell2) * ell1);
  float* Xt = c.ar.take<float>(size_t(ell2) * ell1);
  float* Uj = c.ar.take<float>(size_t(ell2) * ell1);
  float* Vj = c.ar.take<float>(size_t(ell1) * ell1);
  float* Sj = c.ar.take<float>(size_t(ell1));
  float* sig = c.ar.take<float>(size_t(l1 + 1) * k);
  int* sel = c.ar.take<int>(1);
  if (c.measure) {  // account for the helpers' own temporaries
    orth(c, Mat{nullptr, A.m, ell1, A.m}, nullptr);
    orth(c, Mat{nullptr, A.n, ell2, A.n}, nullptr);
    orth(c, Mat{nullptr, ell2, ell1, ell2}, nullptr);
    core_svd(c, nullptr, ell1, nullptr, nullptr, nullptr);
    tri_inv_any(c, nullptr, ell1, nullptr);
    return l1;
  }
  copy_f32(Y.p, Y.ld, Yc.p, Yc.ld, A.m, ell1, c.s);
  copy_f32(Z.p, Z.ld, Zc.p, Zc.ld, A.n, ell2, c.s);
  orth(c, Yc, Rc);                                   // Y = Q R
  core_svd(c, Rc, ell1, Wc, Vc, Sc);                 // R = W S V^T
  gemm(c, A.m, ell1, ell1, false, Yc.p, Yc.ld, false, Wc, ell1, Qf.p, Qf.ld);  // left singular vectors of Y
  gram64(c, ell2, ell1, A.m, Psi.p, Psi.ld, Qf.p, Qf.ld, B64, ell2);          // Psi^T Q_c (all l_c at once)
  f64_to_f32(B64, ell2, B, ell2, ell2, ell1, c.s);
  orth(c, Zc, Rz);                                   // Z = Q_z R_z
  r_to_f32(Rz, ell2, ell2, Rz32, ell2, false, c.s);
  for (int lc = 0; lc <= l1; ++lc) {
    const int L = k + lc;
    copy_f32(B, ell2, Bl, ell2, ell2, L, c.s);
    orth(c, Mat{Bl, ell2, L, ell2}, Rl);             // [Q^, R^] = qr(Psi^T Q_c)
    tri_inv_any(c, Rl, L, Ri);
    gemm(c, ell2, L, ell2, false, Rz32, ell2, false, Bl, ell2, M1, ell2);   // R_z Q^
    gemm(c, ell2, L, L, false, M1, ell2, true, Ri, L, Xt, ell2);           // X^T = R_z Q^ R^^{-T}
    jacobi_svd(Xt, ell2, ell2, L, Uj, ell2, Vj, L, Sj, nullptr, c.status, c.s);
    LR_CHECK_CUDA(cudaMemcpyAsync(sig + size_t(lc) * k, Sj, sizeof(float) * k, cudaMemcpyDeviceToDevice, c.s));
  }
  minvar_select(sig, l1 + 1, k, sel, c.s);
  int h_sel = l1;
  LR_CHECK_CUDA(cudaMemcpyAsync(&h_sel, sel, sizeof(int), cudaMemcpyDeviceToHost, c.s));
  LR_CHECK_CUDA(cudaStreamSynchronize(c.s));
  return (h_sel >= 0 && h_sel <= l1) ? h_sel : l1;
}

void run_single_pass(Ctx& c, const AMat& A, int k, int l_c, const Mat& Om, const Mat& Psi, Outs& o,
                     const Sketcher& sketch = nullptr) {
  ArenaScope sc(c.ar);
  const int ell1 = int(Om.cols), ell2 = int(Psi.cols);
  const int l1 = ell1 - k;
  Mat Y{c.ar.take<float>(size_t(A.m) * ell1), A.m, ell1, A.m};
  Mat Z{c.ar.take<float>(size_t(A.n) * ell2), A.n, ell2, A.n};
  if (sketch) sketch(c, Y, Z);            // a) Y_c = A Omega_r, b) Y_r = A^T Omega_c
  else view_dual(c, A, Om, Y, Psi, Z);
  const int lc = (l_c == LR_LC_MINVAR) ? minvar_lc(c, A, k, Y, Z, Psi) : (l_c < 0 || l_c > l1) ? l1 : l_c;
  const int Lc = k + lc;
  double* Rc = c.ar.take<double>(size_t(ell1) * ell1);
  Mat Q2{lc < l1 ? c.ar.take<float>(size_t(A.m) * Lc) : nullptr, A.m, Lc, A.m};
  float* Wc = c.ar.take<float>(size_t(ell1) * ell1);
  float* Vc = c.ar.take<float>(size_t(ell1) * ell1);
  float* Sc = c.ar.take<float>(size_t(ell1));
  double* P64 = c.ar.take<double>(size_t(ell2) * Lc);
  Mat P{c.ar.take<float>(size_t(ell2) * Lc), ell2, Lc, ell2};
  double* Rh = c.ar.take<double>(size_t(Lc) * Lc);
  float* Rhi = c.ar.take<float>(size_t(Lc) * Lc);
  Mat Wz{c.ar.take<float>(size_t(A.n) * Lc), A.n, Lc, A.n};
  Mat Xt{c.ar.take<float>(size_t(A.n) * Lc), A.n, Lc, A.n};
  double* Rx = c.ar.take<double>(size_t(Lc) * Lc);
  float* W = c.ar.take<float>(size_t(Lc) * Lc);
  float* Vj = c.ar.take<float>(size_t(Lc) * Lc);
  float* Sv = c.ar.take<float>(size_t(Lc));

  orth(c, Y, Rc);                        // [Q_c, R_c] = qr(Y_c)
  Mat Qc = Y;
  if (lc < l1) {
    core_svd(c, Rc, ell1, Wc, Vc, Sc);   // leading k + l_c left vectors of R_c
    gemm(c, A.m, Lc, ell1, false, Y.p, Y.ld, false, Wc, ell1, Q2.p, Q2.ld);
    Qc = Q2;
  }
  gram64(c, ell2, Lc, A.m, Psi.p, Psi.ld, Qc.p, Qc.ld, P64, ell2);   // Omega_c^T Q_c
  if (!c.measure) f64_to_f32(P64, ell2, P.p, P.ld, ell2, Lc, c.s);
  orth(c, P, Rh);                        // [Q^, R^] = qr(Omega_c^T Q_c)
  gemm(c, A.n, Lc, ell2, false, Z.p, Z.ld, false, P.p, P.ld, Wz.p, Wz.ld);  // Y_r Q^
  tri_inv_any(c, Rh, Lc, Rhi);
  gemm(c, A.n, Lc, Lc, false, Wz.p, Wz.ld, true, Rhi, Lc, Xt.p, Xt.ld);    // X^T = Y_r Q^ R^{-T}
  orth(c, Xt, Rx);                       // X^T = Q_x R_x
  core_svd(c, Rx, Lc, W, Vj, Sv);        // R_x = W S Vj^T, X = Vj S (Q_x W)^T
  write_outputs(c, Qc, Vj, Xt, W, Lc, Sv, k, o);
}

// ------------------------------------------------------------ Alg. 8
// Woolfe variant of the single view: Q_c and Q_r are the leading k + l_c
// left singular vectors of both sketches, X^ the least-squares solution of
// (Psi^T Q_c) X^ = Y_r^T Q_r (through the QR of Psi^T Q_c), U = Q_c U^,
// V = Q_r V^ from the SVD of X^.
void run_woolfe(Ctx& c, const AMat& A, int k, int l_c, const Mat& Om, const Mat& Psi, Outs& o) {
  ArenaScope sc(c.ar);
  const int ell1 = int(Om.cols), ell2 = int(Psi.cols), l1 = ell1 - k;
  const int lc = (l_c < 0 || l_c > l1) ? l1 : l_c, kc = k + lc;
  Mat Y{c.ar.take<float>(size_t(A.m) * ell1), A.m, ell1, A.m};
  Mat Z{c.ar.take<float>(size_t(A.n) * ell2), A.n, ell2, A.n};
  Mat Zq{c.ar.take<float>(size_t(A.n) * ell2), A.n, ell2, A.n};
  Mat Qc{c.ar.take<float>(size_t(A.m) * kc), A.m, kc, A.m};
  Mat Qr{c.ar.take<float>(size_t(A.n) * kc), A.n, kc, A.n};
  double* Rc = c.ar.take<double>(size_t(ell1) * ell1);
  double* Rr = c.ar.take<double>(size_t(ell2) * ell2);
  float* Wc = c.ar.take<float>(size_t(ell1) * ell1);
  float* Vc = c.ar.take<float>(size_t(ell1) * ell1);
  float* Sc = c.ar.take<float>(size_t(ell1));
  float* Wr = c.ar.take<float>(size_t(ell2) * ell2);
  float* Vr = c.ar.take<float>(size_t(ell2) * ell2);
  float* Sr = c.ar.take<float>(size_t(ell2));
  double* P64 = c.ar.take<double>(size_t(ell2) * kc);
  Mat P{c.ar.take<float>(size_t(ell2) * kc), ell2, kc, ell2};
  float* Rhs = c.ar.take<float>(size_t(ell2) * kc);
  double* Rh = c.ar.take<double>(size_t(kc) * kc);
  float* Rhi = c.ar.take<float>(size_t(kc) * kc);
  float* M1 = c.ar.take<float>(size_t(kc) * kc);
  float* X = c.ar.take<float>(size_t(kc) * kc);
  float* Ux = c.ar.take<float>(size_t(kc) * kc);
  float* Vx = c.ar.take<float>(size_t(kc) * kc);
  float* Sx = c.ar.take<float>(size_t(kc));
  view_dual(c, A, Om, Y, Psi, Z);                  // Y_c = A Omega, Y_r = A^T Psi
  if (c.measure) {
    orth(c, Mat{nullptr, std::max(A.m, A.n), std::max(ell1, ell2), std::max(A.m, A.n)}, nullptr);
    core_svd(c, nullptr, std::max(ell1, ell2), nullptr, nullptr, nullptr);
    tri_inv_any(c, nullptr, kc, nullptr);
    return;
  }
  copy_f32(Z.p, Z.ld, Zq.p, Zq.ld, A.n, ell2, c.s);
  orth(c, Y, Rc);                                    // Y_c = Q_c R_c
  core_svd(c, Rc, ell1, Wc, Vc, Sc);                 // leading left vectors of R_c
  gemm(c, A.m, kc, ell1, false, Y.p, Y.ld, false, Wc, ell1, Qc.p, Qc.ld);
  orth(c, Zq, Rr);                                   // Y_r = Q_r R_r
  core_svd(c, Rr, ell2, Wr, Vr, Sr);
  gemm(c, A.n, kc, ell2, false, Zq.p, Zq.ld, false, Wr, ell2, Qr.p, Qr.ld);
  gram64(c, ell2, kc, A.m, Psi.p, Psi.ld, Qc.p, Qc.ld, P64, ell2);     // Psi^T Q_c
  f64_to_f32(P64, ell2, P.p, P.ld, ell2, kc, c.s);
  gram64(c, ell2, kc, A.n, Z.p, Z.ld, Qr.p, Qr.ld, P64, ell2);         // Y_r^T Q_r
  f64_to_f32(P64, ell2, Rhs, ell2, ell2, kc, c.s);
  orth(c, P, Rh);                                    // Psi^T Q_c = Q^ R^
  gemm(c, kc, kc, ell2, true, P.p, P.ld, false, Rhs, ell2, M1, kc);   // Q^^T (Y_r^T Q_r)
  tri_inv_any(c, Rh, kc, Rhi);
  gemm(c, kc, kc, kc, false, Rhi, kc, false, M1, kc, X, kc);          // X^ = R^^{-1} Q^^T Y_r^T Q_r
  jacobi_svd(X, kc, kc, kc, Ux, kc, Vx, kc, Sx, nullptr, c.status, c.s);
  write_outputs(c, Qc, Ux, Qr, Vx, kc, Sx, k, o);
}

// ------------------------------------------------------- Section 6.7
// The extended sketch with SRFT test matrices (the approximation bwz2):
// Y_c = A Omega and A Phi_c from the same range view as Y_r = A^T Psi,
// Z = Phi_r^T (A Phi_c), U_c T_c = Phi_r^T Q_c, U_r T_r = Phi_c^T Q_r,
// C = T_c^{-1} U_c^T Z U_r T_r^{-T}, U = Q_c U^, V = Q_r V^ from C's SVD.
void run_extended(Ctx& c, const AMat& A, int k, const Mat& Om, const Mat& Psi, const Mat& Phc, const Mat& Phr,
                  Outs& o) {
  ArenaScope sc(c.ar);
  const int ell = int(Om.cols), s = int(Phc.cols), w = ell + s;
  Mat Xc{c.ar.take<float>(size_t(A.n) * w), A.n, w, A.n};
  Mat Yc{c.ar.take<float>(size_t(A.m) * w), A.m, w, A.m};
  Mat Yr{c.ar.take<float>(size_t(A.n) * ell), A.n, ell, A.n};
  double* G64 = c.ar.take<double>(size_t(s) * std::max(s, ell));
  float* Zs = c.ar.take<float>(size_t(s) * s);
  Mat Bc{c.ar.take<float>(size_t(s) * ell), s, ell, s};
  Mat Br{c.ar.take<float>(size_t(s) * ell), s, ell, s};
  double* Tc = c.ar.take<double>(size_t(ell) * ell);
  double* Tr = c.ar.take<double>(size_t(ell) * ell);
  float* Tci = c.ar.take<float>(size_t(ell) * ell);
  float* Tri = c.ar.take<float>(size_t(ell) * ell);
  float* M1 = c.ar.take<float>(size_t(ell) * s);
  float* M2 = c.ar.take<float>(size_t(ell) * ell);
  float* C1 = c.ar.take<float>(size_t(ell) * ell);
  float* Cm = c.ar.take<float>(size_t(ell) * ell);
  float* Uc = c.ar.take<float>(size_t(ell) * ell);
  float* Vc = c.ar.take<float>(size_t(ell) * ell);
  float* Sc = c.ar.take<float>(size_t(ell));
  Mat Y{Yc.p, A.m, ell, A.m};
  Mat W{Yc.p + size_t(A.m) * ell, A.m, s, A.m};
  if (c.measure) {
    view_dual(c, A, Xc, Yc, Psi, Yr);
    orth(c, Mat{nullptr, std::max(A.m, A.n), ell, std::max(A.m, A.n)}, nullptr);
    tri_inv_any(c, nullptr, ell, nullptr);
    return;
  }
  copy_f32(Om.p, Om.ld, Xc.p, Xc.ld, A.n, ell, c.s);
  copy_f32(Phc.p, Phc.ld, Xc.p + size_t(A.n) * ell, Xc.ld, A.n, s, c.s);
  view_dual(c, A, Xc, Yc, Psi, Yr);                 // [A Omega, A Phi_c] and A^T Psi, one pass
  gram64(c, s, s, A.m, Phr.p, Phr.ld, W.p, W.ld, G64, s);   // Z = Phi_r^T (A Phi_c)
  f64_to_f32(G64, s, Zs, s, s, s, c.s);
  orth(c, Y, nullptr);                               // Q_c
  orth(c, Yr, nullptr);                              // Q_r
  gram64(c, s, ell, A.m, Phr.p, Phr.ld, Y.p, Y.ld, G64, s);    // Phi_r^T Q_c
  f64_to_f32(G64, s, Bc.p, Bc.ld, s, ell, c.s);
  orth(c, Bc, Tc);                                   // U_c T_c
  gram64(c, s, ell, A.n, Phc.p, Phc.ld, Yr.p, Yr.ld, G64, s);  // Phi_c^T Q_r
  f64_to_f32(G64, s, Br.p, Br.ld, s, ell, c.s);
  orth(c, Br, Tr);                                   // U_r T_r
  gemm(c, ell, s, s, true, Bc.p, Bc.ld, false, Zs, s, M1, ell);         // U_c^T Z
  gemm(c, ell, ell, s, false, M1, ell, false, Br.p, Br.ld, M2, ell);    // (.) U_r
  tri_inv_any(c, Tc, ell, Tci);
  tri_inv_any(c, Tr, ell, Tri);
  gemm(c, ell, ell, ell, false, Tci, ell, false, M2, ell, C1, ell);     // T_c^{-1} (.)
  gemm(c, ell, ell, ell, false, C1, ell, true, Tri, ell, Cm, ell);      // (.) T_r^{-T}
  jacobi_svd(Cm, ell, ell, ell, Uc, ell, Vc, ell, Sc, nullptr, c.status, c.s);
  write_outputs(c, Y, Uc, Yr, Vc, ell, Sc, k, o);
}

// ------------------------------------------------- reverse of Alg. 2
// dA for L = sum_i dS_i sigma_i(R) where R is the last view's triangular
// factor (the core of Alg. 2).  The forward views are recomputed (nothing is
// kept from lr_subspace_iter).  Reverse rules (standard matrix calculus,
// the paper has no derivatives):
//   core:  R = W S Z^T  ->  Rb = W_k diag(dS) Z_k^T;
//   thin QR B = Q R:  M = R Rb^T - Qb^T Q, Bb = (Qb + Q copyltu(M)) R^{-T};
//   view B = A X:  dA += Bb X^T, Xb = A^T Bb;  B = A^T X:  dA += X Bb^T, Xb = A Bb.
// Every dA term is an outer product of two ell-column panels, so dA is
// written once by one GEMM: dA = [L_1 .. L_v] [R_1 .. R_v]^T with
// (L_j, R_j) = (Bb_j, X_j) for odd j and (X_j, Bb_j) for even j.
void run_subspace_backward(Ctx& c, const AMat& A, int k, int ell, int v, const Mat& Om, const float* dS,
                           const Mat* dU, const Mat* dV, float* dA, int64_t ldda) {
  ArenaScope sc(c.ar);
  const int64_t m = A.m, n = A.n;
  Mat Lc{c.ar.take<float>(size_t(m) * v * ell), m, int64_t(v) * ell, m};   // m-side panels
  Mat Rc{c.ar.take<float>(size_t(n) * v * ell), n, int64_t(v) * ell, n};   // n-side panels
  const int64_t rows_v = (v % 2 == 1) ? m : n;
  Mat Qv{c.ar.take<float>(size_t(rows_v) * ell), rows_v, ell, rows_v};      // Q of the last view
  double* Rs = c.ar.take<double>(size_t(v) * ell * ell);
  float* W = c.ar.take<float>(size_t(ell) * ell);
  float* Z = c.ar.take<float>(size_t(ell) * ell);
  float* Sv = c.ar.take<float>(size_t(ell));
  float* Rb = c.ar.take<float>(size_t(ell) * ell);
  float* Rf = c.ar.take<float>(size_t(ell) * ell);
  float* Mm = c.ar.take<float>(size_t(ell) * ell);
  float* Ms = c.ar.take<float>(size_t(ell) * ell);
  float* Ri = c.ar.take<float>(size_t(ell) * ell);
  double* C64 = c.ar.take<double>(size_t(ell) * ell);
  const int64_t mx = std::max(m, n);
  float* rhs = c.ar.take<float>(size_t(mx) * ell);
  float* Qb = c.ar.take<float>(size_t(mx) * ell);
  float* dSd = c.ar.take<float>(size_t(ell));
  // gradients on U and V: [dU; dV] with the forward's sign fix applied, the
  // unfixed U, W^T Wb and Z^T Zb, the middle factor, and the lift term of
  // the second-to-last view's Q
  const int64_t mn = m + n;
  float* DD = c.ar.take<float>(size_t(mn) * k);
  float* Ur = c.ar.take<float>(size_t(m) * k);
  double* X64 = c.ar.take<double>(size_t(ell) * k);
  float* dUh = c.ar.take<float>(size_t(ell) * k);
  float* dVh = c.ar.take<float>(size_t(ell) * k);
  float* Xw = c.ar.take<float>(size_t(ell) * k);
  float* Xz = c.ar.take<float>(size_t(ell) * k);
  float* Inner = c.ar.take<float>(size_t(ell) * ell);
  float* Qp = c.ar.take<float>(size_t(mx) * ell);
  // slot j (1-based) of the panel lists; Q_j of view j lands in the slot of
  // view j + 1 (odd j: Lc, even j: Rc), Omega in Rc slot 1
  auto lslot = [&](int j) { return Mat{Lc.col(int64_t(j - 1) * ell), m, ell, m}; };
  auto rslot = [&](int j) { return Mat{Rc.col(int64_t(j - 1) * ell), n, ell, n}; };
  if (c.measure) {  // account for the helpers' own temporaries
    orth(c, Mat{nullptr, mx, ell, mx}, nullptr);
    core_svd(c, nullptr, ell, nullptr, nullptr, nullptr);
    view_range(c, A, Mat{nullptr, n, ell, n}, Mat{nullptr, m, ell, m});
    view_corange(c, A, Mat{nullptr, m, ell, m}, Mat{nullptr, n, ell, n});
    return;
  }
  copy_f32(Om.p, Om.ld, rslot(1).p, n, n, ell, c.s);
  // ---- forward recomputation: B_j = A Q_{j-1} (odd) or A^T Q_{j-1} (even)
  for (int j = 1; j <= v; ++j) {
    const bool odd = j % 2 == 1;
    Mat in = odd ? rslot(j) : lslot(j);
    Mat out = (j == v) ? Qv : (odd ? lslot(j + 1) : rslot(j + 1));
    if (odd) view_range(c, A, in, out);
    else view_corange(c, A, in, out);
    orth(c, out, Rs + size_t(j - 1) * ell * ell);
  }
  // ---- core: R_v = W S Z^T
  core_svd(c, Rs + size_t(v - 1) * ell * ell, ell, W, Z, Sv);
  const bool uv = dU != nullptr || dV != nullptr;
  bool have_qb = false;
  if (!uv) {
    // sigma only: Rb = W_k diag(dS) Z_k^T
    LR_CHECK_CUDA(cudaMemcpyAsync(dSd, dS, sizeof(float) * k, cudaMemcpyDeviceToDevice, c.s));
    scale_cols_f32(W, ell, ell, k, dSd, c.s);
    gemm(c, ell, ell, k, false, W, ell, true, Z, ell, Rb, ell);
  } else {
    // Outputs (as the forward forms them): v odd R_c = U^ L V^^T, U = Q_v U^_k,
    // V = Q_{v-1} V^_k; v even R_r = V^ L U^^T, U = Q_{v-1} U^_k, V = Q_v V^_k.
    const bool vodd = v % 2 == 1;
    Mat Qprev = vodd ? rslot(v) : lslot(v);            // Q_{v-1} sits in view v's slot
    const Mat Qc = vodd ? Qv : Qprev, Qr = vodd ? Qprev : Qv;
    const float* Uh = vodd ? W : Z;
    const float* Vh = vodd ? Z : W;
    // [dU; dV] with the sign flips of the forward's fix (decided on U = Q_c U^_k)
    LR_CHECK_CUDA(cudaMemsetAsync(DD, 0, sizeof(float) * size_t(mn) * k, c.s));
    if (dU) copy_f32(dU->p, dU->ld, DD, mn, m, k, c.s);
    if (dV) copy_f32(dV->p, dV->ld, DD + m, mn, n, k, c.s);
    gemm(c, m, k, ell, false, Qc.p, Qc.ld, false, Uh, ell, Ur, m);
    fix_signs(Ur, m, m, DD, mn, mn, k, c.s);
    const float* dUr = DD;
    const float* dVr = DD + m;
    // U^b = Q_c^T dU, V^b = Q_r^T dV; lift terms Q_c b = dU U^_k^T, Q_r b = dV V^_k^T
    gram64(c, ell, k, m, Qc.p, Qc.ld, dUr, mn, X64, ell);
    f64_to_f32(X64, ell, dUh, ell, ell, k, c.s);
    gram64(c, ell, k, n, Qr.p, Qr.ld, dVr, mn, X64, ell);
    f64_to_f32(X64, ell, dVh, ell, ell, k, c.s);
    float* q_last = Qb;  // the lift term of Q_v starts the reverse pass
    float* q_prev = Qp;
    gemm(c, m, ell, k, false, dUr, mn, true, Uh, ell, vodd ? q_last : q_prev, m);
    gemm(c, n, ell, k, false, dVr, mn, true, Vh, ell, vodd ? q_prev : q_last, n);
    // the core's left factor carries U^ (v odd) or V^ (v even)
    const float* Wb = vodd ? dUh : dVh;
    const float* Zb = vodd ? dVh : dUh;
    gemm(c, ell, k, ell, true, W, ell, false, Wb, ell, Xw, ell);   // W^T Wb
    gemm(c, ell, k, ell, true, Z, ell, false, Zb, ell, Xz, ell);   // Z^T Zb
    svd_bwd_inner(ell, k, Sv, dS, Xw, Xz, Inner, c.s);
    gemm(c, ell, ell, ell, false, W, ell, false, Inner, ell, Mm, ell);
    gemm(c, ell, ell, ell, false, Mm, ell, true, Z, ell, Rb, ell);  // Rb = W inner Z^T
    have_qb = true;
  }
  // ---- reverse through the views
  for (int j = v; j >= 1; --j) {
    const bool odd = j % 2 == 1;
    const int64_t rows = odd ? m : n;
    Mat Q = (j == v) ? Qv : (odd ? lslot(j + 1) : rslot(j + 1));
    const double* R = Rs + size_t(j - 1) * ell * ell;
    // M = R Rb^T - Qb^T Q  (Rb = 0 below the last view)
    if (j == v) {
      r_to_f32(R, ell, ell, Rf, ell, false, c.s);
      gemm(c, ell, ell, ell, false, Rf, ell, true, Rb, ell, Mm, ell);
    } else {
      LR_CHECK_CUDA(cudaMemsetAsync(Mm, 0, sizeof(float) * ell * ell, c.s));
    }
    if (have_qb) gram64(c, ell, ell, rows, Qb, rows, Q.p, Q.ld, C64, ell);
    qr_bwd_sym(Mm, have_qb ? C64 : nullptr, ell, Ms, c.s);
    // rhs = Qb + Q copyltu(M)
    if (have_qb) copy_f32(Qb, rows, rhs, rows, rows, ell, c.s);
    gemm(c, rows, ell, ell, false, Q.p, Q.ld, false, Ms, ell, rhs, rows, 1.f, have_qb ? 1.f : 0.f);
    // Bb = rhs R^{-T}, written into this view's panel slot
    tri_inv_any(c, R, ell, Ri);
    Mat Bb = odd ? lslot(j) : rslot(j);
    gemm(c, rows, ell, ell, false, rhs, rows, true, Ri, ell, Bb.p, Bb.ld);
    if (j > 1) {
      // Qb_{j-1} = A^T Bb (odd j) or A Bb (even j)
      Mat qb{Qb, odd ? n : m, ell, odd ? n : m};
      if (odd) view_corange(c, A, Bb, qb);
      else view_range(c, A, Bb, qb);
      if (uv && j == v) add_f32(Qb, qb.ld, Qp, qb.ld, qb.rows, ell, c.s);  // Q_{v-1}'s lift term
      have_qb = true;
    }
  }
  // ---- dA = Lc Rc^T, one GEMM (as column-major: dA^T = Rc Lc^T)
  gemm(c, n, m, int64_t(v) * ell, false, Rc.p, Rc.ld, true, Lc.p, Lc.ld, dA, ldda);
}

// ------------------------------------------------- host streaming
// The streaming model of Section 6.1 (A = sum_i H_i, each update seen once)
// with H_i = the i-th column panel of a pinned host A: panel i is copied to
// one of two device panel buffers on the handle's copy stream while the
// previous panel is sketched on the caller's stream; for every panel,
//   Y += A_P Omega[P, :]   and   Z[P, :] = A_P^T Psi,
// so A crosses the host link exactly once.  Events order each buffer's
// reuse after its sketches and each sketch after its copy.
struct HostA {
  const float* p = nullptr;
  int64_t m = 0, n = 0, ld = 0;
  bool panels = false;  // stored as contiguous column panels (lr_opts.host_panels)
};

// Views of a pinned host A streamed in column panels: Y = A X (X: n x ell,
// when Y is given) and/or Z = A^T W (W: m x ell2, when Z is given), with A
// crossing the host link once for both.
void host_views(Ctx& c, const HostA& H, int64_t pc, const Mat* X, Mat* Y, const Mat* W, Mat* Z) {
  ArenaScope sc(c.ar);
  float* buf[2];
  const int64_t ldp = round4(pc);  // panel rows padded to a 16-byte stride (TMA)
  buf[0] = c.ar.take<float>(size_t(H.m) * ldp);
  buf[1] = c.ar.take<float>(size_t(H.m) * ldp);
  AMat shape;  // an F32 A: the co-range operand is split once for all panels
  shape.bf16 = false;
  if (c.measure) {
    if (Z) convert_operand(c, shape, nullptr, 0, H.m, int(W->cols));
    return;
  }
  lr_handle h = c.h;
  if (!h->copy_stream) {
    LR_CHECK_CUDA(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
      LR_CHECK_CUDA(cudaEventCreateWithFlags(&h->copied[i], cudaEventDisableTiming));
      LR_CHECK_CUDA(cudaEventCreateWithFlags(&h->consumed[i], cudaEventDisableTiming));
    }
  }
  if (Y) zero_f32(Y->p, Y->rows, Y->cols, Y->ld, c.s);
  if (Z) zero_f32(Z->p, Z->rows, Z->cols, Z->ld, c.s);
  SplitOp wo;
  if (Z) wo = convert_operand(c, shape, W->p, W->ld, H.m, int(W->cols));
  // the copy stream starts after everything already queued on the caller's stream
  LR_CHECK_CUDA(cudaEventRecord(h->consumed[0], c.s));
  LR_CHECK_CUDA(cudaStreamWaitEvent(h->copy_stream, h->consumed[0], 0));
  LR_CHECK_CUDA(cudaEventRecord(h->consumed[1], c.s));
  const int npan = int((H.n + pc - 1) / pc);
  for (int i = 0; i < npan; ++i) {
    const int b = i & 1;
    const int64_t c0 = int64_t(i) * pc, w = std::min(pc, H.n - c0);
    LR_CHECK_CUDA(cudaStreamWaitEvent(h->copy_stream, h->consumed[b], 0));
    if (H.panels)  // panel i is one contiguous m x pc block
      LR_CHECK_CUDA(cudaMemcpyAsync(buf[b], H.p + int64_t(i) * H.m * pc, size_t(H.m) * size_t(pc) * sizeof(float),
                                    cudaMemcpyHostToDevice, h->copy_stream));
    else
      LR_CHECK_CUDA(cudaMemcpy2DAsync(buf[b], size_t(ldp) * sizeof(float), H.p + c0, size_t(H.ld) * sizeof(float),
                                      size_t(w) * sizeof(float), size_t(H.m), cudaMemcpyHostToDevice,
                                      h->copy_stream));
    LR_CHECK_CUDA(cudaEventRecord(h->copied[b], h->copy_stream));
    LR_CHECK_CUDA(cudaStreamWaitEvent(c.s, h->copied[b], 0));
    AMat P;
    P.p = buf[b];
    P.m = H.m;
    P.n = w;
    P.ld = ldp;
    P.bf16 = false;
    // Y += A_P X[c0 : c0 + w, :]
    if (Y) view_band(c, P, 0, X->p + c0, X->ld, int(X->cols), Y->p, Y->ld, 0, H.m);
    // Z[c0 : c0 + w, :] = A_P^T W
    if (Z) view_band(c, P, 1, W->p, W->ld, int(W->cols), Z->p + c0, Z->ld, 0, H.m, &wo);
    LR_CHECK_CUDA(cudaEventRecord(h->consumed[b], c.s));
  }
}

void sketch_host_panels(Ctx& c, const HostA& H, int64_t pc, const Mat& Om, const Mat& Psi, Mat Y, Mat Z) {
  host_views(c, H, pc, &Om, &Y, &Psi, &Z);
}

// ------------------------------------------------------- validation
AMat check_A(const lr_mat* A) {
  LR_REQUIRE(A && A->data, LR_ERR_INVALID_ARG, "A is NULL");
  LR_REQUIRE(A->dtype == LR_F32 || A->dtype == LR_BF16, LR_ERR_DTYPE, "A must be F32 or BF16");
  LR_REQUIRE(A->col_major == 0, LR_ERR_DTYPE, "A must be row-major");
  LR_REQUIRE(A->rows >= 1 && A->cols >= 1 && A->ld >= A->cols, LR_ERR_SHAPE, "bad A shape");
  AMat a;
  a.p = A->data;
  a.m = A->rows;
  a.n = A->cols;
  a.ld = A->ld;
  a.bf16 = A->dtype == LR_BF16;
  LR_REQUIRE((reinterpret_cast<uintptr_t>(A->data) & 15) == 0, LR_ERR_ALIGNMENT, "A not 16-byte aligned");
  LR_REQUIRE((A->ld * int64_t(a.elem())) % 16 == 0, LR_ERR_ALIGNMENT, "A row stride not a multiple of 16 bytes");
  return a;
}

Mat check_thin(const lr_mat* X, int64_t rows, int64_t cols, const char* name) {
  LR_REQUIRE(X && X->data, LR_ERR_INVALID_ARG, std::string(name) + " is NULL");
  LR_REQUIRE(X->dtype == LR_F32, LR_ERR_DTYPE, std::string(name) + " must be F32");
  LR_REQUIRE(X->col_major == 1, LR_ERR_DTYPE, std::string(name) + " must be column-major");
  LR_REQUIRE(X->rows == rows && (cols < 0 || X->cols == cols) && X->ld >= X->rows, LR_ERR_SHAPE,
             std::string(name) + " has the wrong shape");
  return Mat{static_cast<float*>(X->data), X->rows, X->cols, X->ld};
}

Outs check_outs(const AMat& A, int k, lr_mat* U, lr_mat* S, lr_mat* V) {
  Outs o;
  o.U = check_thin(U, A.m, k, "U");
  o.V = check_thin(V, A.n, k, "V");
  LR_REQUIRE(S && S->data, LR_ERR_INVALID_ARG, "S is NULL");
  LR_REQUIRE(S->dtype == LR_F32, LR_ERR_DTYPE, "S must be F32");
  LR_REQUIRE(S->rows * S->cols >= k, LR_ERR_SHAPE, "S too short");
  o.S = S->data;
  return o;
}

lr_status finish(lr_handle h, const Error& e) {
  if (h) h->last_error = e.msg;
  return e.st;
}

Ctx make_ctx(lr_handle h, const lr_opts* opts, void* stream) {
  Ctx c;
  c.h = h;
  c.s = static_cast<cudaStream_t>(stream);
  c.ar.base = static_cast<char*>(h->ws);
  c.ar.cap = h->ws_bytes;
  c.sms = dev_info(h->device).sms;
  c.status = h->status_dev;
  if (opts) c.opt = *opts;
  else c.opt.l_c = -1;
  LR_CHECK_CUDA(cudaSetDevice(h->device));
  return c;
}

template <class F>
lr_status guarded(lr_handle h, F&& f) {
  if (!h) return LR_ERR_INVALID_ARG;
  try {
    h->last_error.clear();
    f();
    return LR_OK;
  } catch (const Error& e) {
    return finish(h, e);
  } catch (const std::exception& e) {
    return finish(h, Error{LR_ERR_INVALID_ARG, e.what()});
  }
}

void check_kpv(const AMat& A, int k, int p, int v, int vmin) {
  LR_REQUIRE(k >= 1 && p >= 0, LR_ERR_INVALID_ARG, "need k >= 1 and p >= 0");
  LR_REQUIRE(k + p <= std::min(A.m, A.n), LR_ERR_INVALID_ARG, "need k + p <= min(m, n)");
  LR_REQUIRE(v >= vmin, LR_ERR_INVALID_ARG, "too few views");
}

}  // namespace
}  // namespace lr

using namespace lr;

namespace lr {
namespace {
void check_op(const lr_operator* J) {
  LR_REQUIRE(J && J->apply, LR_ERR_INVALID_ARG, "operator (or its callback) is NULL");
  LR_REQUIRE(J->rows >= 1 && J->cols >= 1, LR_ERR_SHAPE, "bad operator shape");
}
}  // namespace
}  // namespace lr

extern "C" {

lr_status lr_create(lr_handle* handle, int device) {
  if (!handle) return LR_ERR_INVALID_ARG;
  *handle = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return LR_ERR_INVALID_ARG;
  auto* h = new lr_handle_s();
  h->device = device;
  if (cudaSetDevice(device) != cudaSuccess || cudaMalloc(&h->status_dev, sizeof(int)) != cudaSuccess ||
      cudaMemset(h->status_dev, 0, sizeof(int)) != cudaSuccess) {
    delete h;
    return LR_ERR_CUDA;
  }
  *handle = h;
  return LR_OK;
}

lr_status lr_destroy(lr_handle h) {
  if (!h) return LR_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  cudaFree(h->status_dev);
  for (cudaEvent_t e : h->pool) cudaEventDestroy(e);
  for (int i = 0; i < 2; ++i) {
    if (h->copied[i]) cudaEventDestroy(h->copied[i]);
    if (h->consumed[i]) cudaEventDestroy(h->consumed[i]);
  }
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  delete h;
  return LR_OK;
}

const char* lr_status_string(lr_status st) {
  switch (st) {
    case LR_OK: return "ok";
    case LR_ERR_INVALID_ARG: return "invalid argument";
    case LR_ERR_SHAPE: return "inconsistent shape";
    case LR_ERR_DTYPE: return "unsupported dtype or layout";
    case LR_ERR_ALIGNMENT: return "misaligned pointer or stride";
    case LR_ERR_BREAKDOWN: return "Cholesky breakdown (rank-deficient sketch)";
    case LR_ERR_NONFINITE: return "non-finite value";
    case LR_ERR_TIMEOUT: return "device-side wait timed out";
    case LR_ERR_CUDA: return "CUDA error";
    case LR_ERR_NOMEM: return "workspace missing or too small";
    case LR_ERR_UNSUPPORTED: return "unsupported by this build";
  }
  return "unknown status";
}

const char* lr_last_error(lr_handle h) { return h ? h->last_error.c_str() : ""; }

lr_status lr_set_workspace(lr_handle h, void* ptr, size_t bytes) {
  if (!h) return LR_ERR_INVALID_ARG;
  if (bytes && (!ptr || (reinterpret_cast<uintptr_t>(ptr) & 255))) return LR_ERR_ALIGNMENT;
  h->ws = ptr;
  h->ws_bytes = bytes;
  return LR_OK;
}

lr_status lr_get_status(lr_handle h, void* stream, int* device_status) {
  return guarded(h, [&] {
    LR_REQUIRE(device_status, LR_ERR_INVALID_ARG, "device_status is NULL");
    LR_CHECK_CUDA(cudaSetDevice(h->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int v = 0;
    LR_CHECK_CUDA(cudaMemcpyAsync(&v, h->status_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    LR_CHECK_CUDA(cudaStreamSynchronize(s));
    LR_CHECK_CUDA(cudaMemsetAsync(h->status_dev, 0, sizeof(int), s));
    LR_CHECK_CUDA(cudaStreamSynchronize(s));
    *device_status = v;
  });
}

lr_status lr_workspace_size(lr_handle h, int64_t m, int64_t n, int ell1, int ell2, int v, size_t* bytes) {
  return guarded(h, [&] {
    LR_REQUIRE(bytes && m > 0 && n > 0 && ell1 > 0 && v >= 1, LR_ERR_INVALID_ARG, "bad workspace query");
    size_t best = 0;
    const int vv = std::max(v, 2);
    for (int bf = 0; bf < 2; ++bf) {
      AMat A;
      A.m = m; A.n = n; A.ld = n; A.bf16 = bf == 1;
      // Each schedule's allocation sequence is replayed without launches;
      // schedules these sizes cannot run (e.g. widths over a limit) are
      // skipped rather than failing the query.
      auto measure = [&](auto&& body) {
        Ctx c;
        c.h = h;
        c.measure = true;
        c.ar.measure = true;
        c.sms = 1;
        c.opt.shifted_fallback = 1;
        c.opt.split_last = 1;  // size for the split form too
        try {
          body(c);
        } catch (const Error&) {
        }
        best = std::max(best, c.ar.peak);
      };
      Mat Om{nullptr, n, ell1, n};
      Outs o;
      const int k = 1;
      measure([&](Ctx& c) { run_subspace(c, A, k, ell1, vv, Om, o); });
      measure([&](Ctx& c) { run_subspace_sharded(c, A, ell1, ell1, vv, Om, o); });  // (m = the local rows)
      measure([&](Ctx& c) { run_krylov(c, A, k, ell1, vv, Om, o); });
      measure([&](Ctx& c) { run_krylov_rowwise(c, A, k, ell1, vv, Om, o); });
      measure([&](Ctx& c) { run_rowwise_qb(c, A, k, ell1, Om, o); });
      if (ell2 >= ell1) {
        Mat Ps{nullptr, m, ell2, m};
        measure([&](Ctx& c) { run_woolfe(c, A, std::max(1, ell1 - 1), -1, Om, Ps, o); });
      }
      if (!A.bf16 && ell1 <= 128) {  // the operator forms (shapes only: no callback in measuring mode)
        lr_operator op{m, n, nullptr, nullptr};
        measure([&](Ctx& c) { run_nystrom(c, &op, k, ell1, vv, Om, Mat{nullptr, n, k, n}, nullptr); });
        measure([&](Ctx& c) { run_pinched(c, &op, k, ell1, vv, Om, Mat{nullptr, n, k, n}, nullptr); });
      }
      if (!A.bf16) measure([&](Ctx& c) { run_subspace_backward(c, A, ell1, ell1, vv, Om, nullptr, nullptr, nullptr, nullptr, 0); });  // k <= ell
      if (ell2 >= ell1) {
        Mat Ps{nullptr, m, ell2, m};
        measure([&](Ctx& c) { run_single_pass(c, A, std::max(1, ell1 - 1), -1, Om, Ps, o); });
      }
      measure([&](Ctx& c) {
        Mat Y{nullptr, m, std::max(ell1, ell2), m};
        orth(c, Y, nullptr);
        Mat Zm{nullptr, n, ell2 > 0 ? ell2 : ell1, n};
        view_dual(c, A, Om, Y, Y, Zm);
        view_chained(c, A, Om, Y, Zm);
      });
    }
    *bytes = best + 4096;
  });
}

lr_status lr_sketch(lr_handle h, const lr_mat* A, const lr_mat* X, const lr_mat* W, lr_mat* Y, lr_mat* Z,
                    const lr_opts* opts, void* stream) {
  return guarded(h, [&] {
    AMat a = check_A(A);
    Ctx c = make_ctx(h, opts, stream);
    LR_REQUIRE(X || W, LR_ERR_INVALID_ARG, "need X or W");
    Mat x, y, w, z;
    if (X) {
      x = check_thin(X, a.n, -1, "X");
      y = check_thin(Y, a.m, x.cols, "Y");
    }
    if (W) {
      w = check_thin(W, a.m, -1, "W");
      z = check_thin(Z, a.n, w.cols, "Z");
    }
    if (X && W) view_dual(c, a, x, y, w, z);
    else if (X) view_range(c, a, x, y);
    else view_corange(c, a, w, z);
  });
}

lr_status lr_sketch_chained(lr_handle h, const lr_mat* A, const lr_mat* X, lr_mat* Y, lr_mat* Z, const lr_opts* opts,
                            void* stream) {
  return guarded(h, [&] {
    AMat a = check_A(A);
    Ctx c = make_ctx(h, opts, stream);
    Mat x = check_thin(X, a.n, -1, "X");
    Mat y = check_thin(Y, a.m, x.cols, "Y");
    Mat z = check_thin(Z, a.n, x.cols, "Z");
    view_chained(c, a, x, y, z);
  });
}

lr_status lr_orth(lr_handle h, lr_mat* Y, lr_mat* R, const lr_opts* opts, void* stream) {
  return guarded(h, [&] {
    LR_REQUIRE(Y, LR_ERR_INVALID_ARG, "Y is NULL");
    Mat y = check_thin(Y, Y->rows, -1, "Y");
    LR_REQUIRE(y.rows >= y.cols && y.cols >= 1, LR_ERR_SHAPE, "orth needs rows >= cols >= 1");
    double* r = nullptr;
    if (R) {
      LR_REQUIRE(R->data && R->dtype == LR_F64 && R->rows == y.cols && R->cols == y.cols && R->ld == y.cols,
                 LR_ERR_SHAPE, "R must be a dense ell x ell F64 matrix");
      r = static_cast<double*>(R->data);
    }
    Ctx c = make_ctx(h, opts, stream);
    orth(c, y, r);
  });
}

lr_status lr_subspace_iter(lr_handle h, const lr_mat* A, int k, int p, int v, const lr_mat* Omega, lr_mat* U,
                           lr_mat* S, lr_mat* V, const lr_opts* opts, void* stream) {
  return guarded(h, [&] {
    AMat a = check_A(A);
    check_kpv(a, k, p, v, 2);
    Mat om = check_thin(Omega, a.n, k + p, "Omega");
    Outs o = check_outs(a, k, U, S, V);
    Ctx c = make_ctx(h, opts, stream);
    run_subspace(c, a, k, k + p, v, om, o);
  });
}

lr_status lr_subspace_iter_sharded(lr_handle h, const lr_mat* A_local, int k, int p, int v, const lr_mat* Omega,
                                   lr_mat* U_local, lr_mat* S, lr_mat* V, const lr_comm* comm, const lr_opts* opts,
                                   void* stream) {
  return guarded(h, [&] {
    LR_REQUIRE(comm && comm->allreduce && comm->world >= 1 && comm->rank >= 0 && comm->rank < comm->world,
               LR_ERR_INVALID_ARG, "bad communicator");
    AMat a = check_A(A_local);
    LR_REQUIRE(k >= 1 && p >= 0 && v >= 2, LR_ERR_INVALID_ARG, "need k >= 1, p >= 0 and v >= 2");
    LR_REQUIRE(k + p <= a.n, LR_ERR_INVALID_ARG, "need k + p <= n");
    LR_REQUIRE(comm->world <= a.n, LR_ERR_INVALID_ARG, "at most n ranks");
    Mat om = check_thin(Omega, a.n, k + p, "Omega");
    Outs o = check_outs(a, k, U_local, S, V);
    Ctx c = make_ctx(h, opts, stream);
    c.comm = comm;
    const int64_t m = sharded_agree(c, a, k, p, v);
    LR_REQUIRE(k + p <= m, LR_ERR_INVALID_ARG, "need k + p <= the total number of rows");
    run_subspace_sharded(c, a, k, k + p, v, om, o);
  });
}

lr_status lr_block_krylov(lr_handle h, const lr_mat* A, int k, int p, int v, const lr_mat* Omega, lr_mat* U,
                          lr_mat* S, lr_mat* V, const lr_opts* opts, void* stream) {
  return guarded(h, [&] {
    AMat a = check_A(A);
    check_kpv(a, k, p, v, 2);
    Mat om = check_thin(Omega, a.n, k + p, "Omega");
    Outs o = check_outs(a, k, U, S, V);
    Ctx c = make_ctx(h, opts, stream);
    const bool enhanced = opts && opts->enhanced;
    const int ell = k + p;
    if (enhanced) {
      LR_REQUIRE(int64_t(v - 1) * ell <= std::min(a.m, a.n), LR_ERR_INVALID_ARG, "Krylov basis wider than A");
      run_krylov_rowwise(c, a, k, ell, v, om, o);
    } else {
      const int nb = (v % 2 == 0) ? v / 2 : (v - 1) / 2;
      LR_REQUIRE(int64_t(nb) * ell <= std::min(a.m, a.n), LR_ERR_INVALID_ARG, "Krylov basis wider than A");
      run_krylov(c, a, k, ell, v, om, o);
    }
  });
}

lr_status lr_rowwise_single_pass(lr_handle h, const lr_mat* A, int k, const lr_mat* Omega, lr_mat* U, lr_mat* S,
                                 lr_mat* V, const lr_opts* opts, void* stream) {
  return guarded(h, [&] {
    AMat a = check_A(A);
    LR_REQUIRE(Omega, LR_ERR_INVALID_ARG, "Omega is NULL");
    const int ell = int(Omega->cols);
    check_kpv(a, k, ell - k, 1, 1);
    Mat om = check_thin(Omega, a.n, ell, "Omega");
    Outs o = check_outs(a, k, U, S, V);
    Ctx c = make_ctx(h, opts, stream);
    run_rowwise_qb(c, a, k, ell, om, o);
  });
}

lr_status lr_single_pass(lr_handle h, const lr_mat* A, int k, const lr_mat* Omega, const lr_mat* Psi, lr_mat* U,
                         lr_mat* S, lr_mat* V, const lr_opts* opts, void* stream) {
  return guarded(h, [&] {
    AMat a = check_A(A);
    LR_REQUIRE(Omega && Psi, LR_ERR_INVALID_ARG, "Omega and Psi are required");
    Mat om = check_thin(Omega, a.n, -1, "Omega");
    Mat ps = check_thin(Psi, a.m, -1, "Psi");
    LR_REQUIRE(k >= 1 && om.cols > k, LR_ERR_INVALID_ARG, "need ell1 > k");
    LR_REQUIRE(ps.cols >= om.cols, LR_ERR_INVALID_ARG, "need ell2 >= ell1 (l_2 >= l_1)");
    LR_REQUIRE(ps.cols <= std::min(a.m, a.n), LR_ERR_INVALID_ARG, "ell2 larger than min(m, n)");
    const int lc = opts ? opts->l_c : -1;
    Outs o = check_outs(a, k, U, S, V);
    Ctx c = make_ctx(h, opts, stream);
    run_single_pass(c, a, k, lc, om, ps, o);
  });
}

lr_status lr_single_pass_host(lr_handle h, const lr_mat* A_host, int64_t panel_cols, int k, const lr_mat* Omega,
                              const lr_mat* Psi, lr_mat* U, lr_mat* S, lr_mat* V, const lr_opts* opts, void* stream) {
  return guarded(h, [&] {
    LR_REQUIRE(A_host && A_host->data, LR_ERR_INVALID_ARG, "A_host is NULL");
    LR_REQUIRE(A_host->dtype == LR_F32 && A_host->col_major == 0, LR_ERR_DTYPE, "A_host must be F32 row-major");
    LR_REQUIRE(A_host->rows >= 1 && A_host->cols >= 1 &&
                   (A_host->ld >= A_host->cols || (opts && opts->host_panels)),
               LR_ERR_SHAPE, "bad A_host");
    LR_REQUIRE(panel_cols >= 1, LR_ERR_INVALID_ARG, "panel_cols must be positive");
    cudaPointerAttributes pa{};
    LR_CHECK_CUDA(cudaPointerGetAttributes(&pa, A_host->data));
    LR_REQUIRE(pa.type == cudaMemoryTypeHost, LR_ERR_INVALID_ARG, "A_host must be pinned (page-locked) host memory");
    AMat a;  // shapes only; the data stays on the host
    a.m = A_host->rows;
    a.n = A_host->cols;
    a.ld = A_host->ld;
    a.bf16 = false;
    LR_REQUIRE(Omega && Psi, LR_ERR_INVALID_ARG, "Omega and Psi are required");
    Mat om = check_thin(Omega, a.n, -1, "Omega");
    Mat ps = check_thin(Psi, a.m, -1, "Psi");
    LR_REQUIRE(k >= 1 && om.cols > k && ps.cols >= om.cols && ps.cols <= std::min(a.m, a.n), LR_ERR_INVALID_ARG,
               "need ell2 >= ell1 > k and ell2 <= min(m, n)");
    Outs o = check_outs(a, k, U, S, V);
    Ctx c = make_ctx(h, opts, stream);
    const bool panels = opts && opts->host_panels;
    LR_REQUIRE(!panels || (panel_cols % 4 == 0 && A_host->ld == panel_cols), LR_ERR_SHAPE,
               "panel layout: panel_cols must be a multiple of 4 and A_host->ld == panel_cols");
    HostA H{static_cast<const float*>(A_host->data), a.m, a.n, A_host->ld, panels};
    const int64_t pc = panels ? panel_cols : std::min<int64_t>(panel_cols, a.n);
    run_single_pass(c, a, k, opts ? opts->l_c : -1, om, ps, o,
                    [&](Ctx& cc, Mat Y, Mat Z) { sketch_host_panels(cc, H, pc, om, ps, Y, Z); });
  });
}

lr_status lr_subspace_iter_host(lr_handle h, const lr_mat* A_host, int64_t panel_cols, int k, int p, int v,
                                const lr_mat* Omega, lr_mat* U, lr_mat* S, lr_mat* V, const lr_opts* opts,
                                void* stream) {
  return guarded(h, [&] {
    LR_REQUIRE(A_host && A_host->data, LR_ERR_INVALID_ARG, "A_host is NULL");
    LR_REQUIRE(A_host->dtype == LR_F32 && A_host->col_major == 0, LR_ERR_DTYPE, "A_host must be F32 row-major");
    LR_REQUIRE(A_host->rows >= 1 && A_host->cols >= 1 &&
                   (A_host->ld >= A_host->cols || (opts && opts->host_panels)),
               LR_ERR_SHAPE, "bad A_host");
    LR_REQUIRE(panel_cols >= 1, LR_ERR_INVALID_ARG, "panel_cols must be positive");
    cudaPointerAttributes pa{};
    LR_CHECK_CUDA(cudaPointerGetAttributes(&pa, A_host->data));
    LR_REQUIRE(pa.type == cudaMemoryTypeHost, LR_ERR_INVALID_ARG, "A_host must be pinned (page-locked) host memory");
    AMat a;  // shapes only; the data stays on the host
    a.m = A_host->rows;
    a.n = A_host->cols;
    a.ld = A_host->ld;
    a.bf16 = false;
    check_kpv(a, k, p, v, 2);
    const int ell = k + p;
    Mat om = check_thin(Omega, a.n, ell, "Omega");
    Outs o = check_outs(a, k, U, S, V);
    Ctx c = make_ctx(h, opts, stream);
    const bool panels = opts && opts->host_panels;
    LR_REQUIRE(!panels || (panel_cols % 4 == 0 && A_host->ld == panel_cols), LR_ERR_SHAPE,
               "panel layout: panel_cols must be a multiple of 4 and A_host->ld == panel_cols");
    HostA H{static_cast<const float*>(A_host->data), a.m, a.n, A_host->ld, panels};
    const int64_t pc = panels ? panel_cols : std::min<int64_t>(panel_cols, a.n);
    Viewer vw;
    vw.range = [&](Ctx& cc, const Mat& X, Mat Y) { host_views(cc, H, pc, &X, &Y, nullptr, nullptr); };
    vw.corange = [&](Ctx& cc, const Mat& W, Mat Z) { host_views(cc, H, pc, nullptr, nullptr, &W, &Z); };
    run_subspace(c, a, k, ell, v, om, o, &vw);
  });
}

lr_status lr_block_krylov_host(lr_handle h, const lr_mat* A_host, int k, int p, int v, const lr_mat* Omega_host,
                               lr_mat* U_host, lr_mat* S_host, lr_mat* V_host, const lr_opts* opts, void* stream) {
  return guarded(h, [&] {
    LR_REQUIRE(A_host && A_host->data, LR_ERR_INVALID_ARG, "A_host is NULL");
    LR_REQUIRE(A_host->dtype == LR_F32 || A_host->dtype == LR_BF16, LR_ERR_DTYPE, "A_host must be F32 or BF16");
    LR_REQUIRE(A_host->col_major == 0, LR_ERR_DTYPE, "A_host must be row-major");
    LR_REQUIRE(A_host->rows >= 1 && A_host->cols >= 1 && A_host->ld >= A_host->cols, LR_ERR_SHAPE, "bad A_host");
    auto pinned = [](const void* ptr) {
      cudaPointerAttributes pa{};
      return ptr && cudaPointerGetAttributes(&pa, ptr) == cudaSuccess && pa.type == cudaMemoryTypeHost;
    };
    AMat a;  // shapes; the data moves to the workspace below
    a.m = A_host->rows;
    a.n = A_host->cols;
    a.ld = A_host->ld;
    a.bf16 = A_host->dtype == LR_BF16;
    LR_REQUIRE((A_host->ld * int64_t(a.elem())) % 16 == 0, LR_ERR_ALIGNMENT, "A row stride not a multiple of 16 bytes");
    check_kpv(a, k, p, v, 2);
    const int ell = k + p;
    const int nb = (v % 2 == 0) ? v / 2 : (v - 1) / 2;
    LR_REQUIRE(int64_t(nb) * ell <= std::min(a.m, a.n), LR_ERR_INVALID_ARG, "Krylov basis wider than A");
    Mat om_h = check_thin(Omega_host, a.n, ell, "Omega_host");
    Outs oh = check_outs(a, k, U_host, S_host, V_host);
    LR_REQUIRE(pinned(A_host->data) && pinned(om_h.p) && pinned(oh.U.p) && pinned(oh.V.p) && pinned(oh.S),
               LR_ERR_INVALID_ARG, "host buffers must be pinned (page-locked)");
    Ctx c = make_ctx(h, opts, stream);
    ArenaScope sc(c.ar);
    char* a_dev = c.ar.take<char>(size_t(a.m) * size_t(a.ld) * a.elem());
    Mat om{c.ar.take<float>(size_t(a.n) * ell), a.n, ell, a.n};
    Outs o;
    o.U = Mat{c.ar.take<float>(size_t(a.m) * k), a.m, k, a.m};
    o.V = Mat{c.ar.take<float>(size_t(a.n) * k), a.n, k, a.n};
    o.S = c.ar.take<float>(size_t(k));
    LR_CHECK_CUDA(cudaMemcpy2DAsync(om.p, size_t(om.ld) * 4, om_h.p, size_t(om_h.ld) * 4, size_t(a.n) * 4, size_t(ell),
                                    cudaMemcpyHostToDevice, c.s));
    a.p = a_dev;
    // A crosses the host link in row blocks on the handle's copy stream; the
    // first view (Y = A Omega, rows r0 .. of Y from rows r0 .. of A) runs on
    // each block as soon as it has landed, so it hides under the copy of the
    // later blocks; the other views start once all of A is on the device.
    const std::function<void(Ctx&, const Mat&, Mat)> first = [&](Ctx& cc, const Mat& X, Mat Y) {
      ArenaScope fs(cc.ar);
      SplitOp pre = convert_operand(cc, a, X.p, X.ld, a.n, int(X.cols));
      if (cc.measure) return;
      lr_handle hh = cc.h;
      if (!hh->copy_stream) {
        LR_CHECK_CUDA(cudaStreamCreateWithFlags(&hh->copy_stream, cudaStreamNonBlocking));
        for (int i = 0; i < 2; ++i) {
          LR_CHECK_CUDA(cudaEventCreateWithFlags(&hh->copied[i], cudaEventDisableTiming));
          LR_CHECK_CUDA(cudaEventCreateWithFlags(&hh->consumed[i], cudaEventDisableTiming));
        }
      }
      zero_f32(Y.p, Y.rows, Y.cols, Y.ld, cc.s);
      // the copies start after everything already queued on the caller's stream
      LR_CHECK_CUDA(cudaEventRecord(hh->consumed[0], cc.s));
      LR_CHECK_CUDA(cudaStreamWaitEvent(hh->copy_stream, hh->consumed[0], 0));
      const int64_t rb = std::max<int64_t>(256, (a.m / 8 + 255) / 256 * 256);
      const size_t row_bytes = size_t(a.ld) * a.elem();
      for (int64_t r0 = 0, b = 0; r0 < a.m; r0 += rb, ++b) {
        const int64_t rows = std::min(rb, a.m - r0);
        LR_CHECK_CUDA(cudaMemcpyAsync(a_dev + size_t(r0) * row_bytes,
                                      static_cast<const char*>(A_host->data) + size_t(r0) * row_bytes,
                                      size_t(rows) * row_bytes, cudaMemcpyHostToDevice, hh->copy_stream));
        LR_CHECK_CUDA(cudaEventRecord(hh->copied[b & 1], hh->copy_stream));
        LR_CHECK_CUDA(cudaStreamWaitEvent(cc.s, hh->copied[b & 1], 0));
        view_band(cc, a, 0, X.p, X.ld, int(X.cols), Y.p, Y.ld, r0, rows, &pre);
      }
    };
    run_krylov(c, a, k, ell, v, om, o, &first);
    LR_CHECK_CUDA(cudaMemcpy2DAsync(oh.U.p, size_t(oh.U.ld) * 4, o.U.p, size_t(o.U.ld) * 4, size_t(a.m) * 4, size_t(k),
                                    cudaMemcpyDeviceToHost, c.s));
    LR_CHECK_CUDA(cudaMemcpy2DAsync(oh.V.p, size_t(oh.V.ld) * 4, o.V.p, size_t(o.V.ld) * 4, size_t(a.n) * 4, size_t(k),
                                    cudaMemcpyDeviceToHost, c.s));
    LR_CHECK_CUDA(cudaMemcpyAsync(oh.S, o.S, sizeof(float) * k, cudaMemcpyDeviceToHost, c.s));
  });
}

lr_status lr_subspace_iter_op(lr_handle h, const lr_operator* J, int k, int p, int v, const lr_mat* Omega, lr_mat* U,
                              lr_mat* S, lr_mat* V, const lr_opts* opts, void* stream) {
  return guarded(h, [&] {
    check_op(J);
    AMat a;  // shapes only
    a.m = J->rows;
    a.n = J->cols;
    a.ld = J->cols;
    check_kpv(a, k, p, v, 2);
    Mat om = check_thin(Omega, a.n, k + p, "Omega");
    Outs o = check_outs(a, k, U, S, V);
    Ctx c = make_ctx(h, opts, stream);
    const Viewer vw = op_viewer(J, false);
    run_subspace(c, a, k, k + p, v, om, o, &vw);
  });
}

lr_status lr_nystrom_tevd(lr_handle h, const lr_operator* J, int k, int p, int v, const lr_mat* Omega, lr_mat* V,
                          lr_mat* Lambda2, const lr_opts* opts, void* stream) {
  return guarded(h, [&] {
    check_op(J);
    AMat a;
    a.m = J->rows;
    a.n = J->cols;
    check_kpv(a, k, p, v, 2);
    LR_REQUIRE(k + p <= 128, LR_ERR_UNSUPPORTED, "lr_nystrom_tevd: k + p <= 128");
    Mat om = check_thin(Omega, v % 2 == 0 ? a.n : a.m, k + p, "Omega");
    Mat vo = check_thin(V, a.n, k, "V");
    LR_REQUIRE(Lambda2 && Lambda2->data && Lambda2->dtype == LR_F32 && Lambda2->rows * Lambda2->cols >= k,
               LR_ERR_SHAPE, "Lambda2 must hold k F32 values");
    Ctx c = make_ctx(h, opts, stream);
    run_nystrom(c, J, k, k + p, v, om, vo, static_cast<float*>(Lambda2->data));
  });
}

lr_status lr_pinched_tevd(lr_handle h, const lr_operator* J, int k, int p, int v, const lr_mat* Omega, lr_mat* V,
                          lr_mat* Lambda2, const lr_opts* opts, void* stream) {
  return guarded(h, [&] {
    check_op(J);
    AMat a;
    a.m = J->rows;
    a.n = J->cols;
    check_kpv(a, k, p, v, 2);
    Mat om = check_thin(Omega, v % 2 == 0 ? a.m : a.n, k + p, "Omega");
    Mat vo = check_thin(V, a.n, k, "V");
    LR_REQUIRE(Lambda2 && Lambda2->data && Lambda2->dtype == LR_F32 && Lambda2->rows * Lambda2->cols >= k,
               LR_ERR_SHAPE, "Lambda2 must hold k F32 values");
    Ctx c = make_ctx(h, opts, stream);
    run_pinched(c, J, k, k + p, v, om, vo, static_cast<float*>(Lambda2->data));
  });
}

lr_status lr_single_pass_woolfe(lr_handle h, const lr_mat* A, int k, const lr_mat* Omega, const lr_mat* Psi,
                                lr_mat* U, lr_mat* S, lr_mat* V, const lr_opts* opts, void* stream) {
  return guarded(h, [&] {
    AMat a = check_A(A);
    LR_REQUIRE(Omega && Psi, LR_ERR_INVALID_ARG, "Omega and Psi are required");
    Mat om = check_thin(Omega, a.n, -1, "Omega");
    Mat ps = check_thin(Psi, a.m, -1, "Psi");
    LR_REQUIRE(k >= 1 && om.cols > k, LR_ERR_INVALID_ARG, "need ell1 > k");
    LR_REQUIRE(ps.cols >= om.cols, LR_ERR_INVALID_ARG, "need ell2 >= ell1 (l_2 >= l_1)");
    LR_REQUIRE(ps.cols <= std::min(a.m, a.n), LR_ERR_INVALID_ARG, "ell2 larger than min(m, n)");
    Outs o = check_outs(a, k, U, S, V);
    Ctx c = make_ctx(h, opts, stream);
    run_woolfe(c, a, k, opts ? opts->l_c : -1, om, ps, o);
  });
}

lr_status lr_single_pass_extended(lr_handle h, const lr_mat* A, int k, const lr_mat* Omega, const lr_mat* Psi,
                                  const lr_mat* Phi_c, const lr_mat* Phi_r, lr_mat* U, lr_mat* S, lr_mat* V,
                                  const lr_opts* opts, void* stream) {
  return guarded(h, [&] {
    AMat a = check_A(A);
    LR_REQUIRE(Omega && Psi && Phi_c && Phi_r, LR_ERR_INVALID_ARG, "Omega, Psi, Phi_c and Phi_r are required");
    Mat om = check_thin(Omega, a.n, -1, "Omega");
    Mat ps = check_thin(Psi, a.m, om.cols, "Psi");
    Mat pc = check_thin(Phi_c, a.n, -1, "Phi_c");
    Mat pr = check_thin(Phi_r, a.m, pc.cols, "Phi_r");
    LR_REQUIRE(k >= 1 && om.cols > k, LR_ERR_INVALID_ARG, "need ell > k");
    LR_REQUIRE(pc.cols >= om.cols, LR_ERR_INVALID_ARG, "need s >= ell");
    LR_REQUIRE(pc.cols <= std::min(a.m, a.n), LR_ERR_INVALID_ARG, "s larger than min(m, n)");
    Outs o = check_outs(a, k, U, S, V);
    Ctx c = make_ctx(h, opts, stream);
    run_extended(c, a, k, om, ps, pc, pr, o);
  });
}

lr_status lr_srft(lr_handle h, int64_t n, int s, const float* signs, const int* cols, lr_mat* Phi, void* stream) {
  return guarded(h, [&] {
    LR_REQUIRE(signs && cols, LR_ERR_INVALID_ARG, "signs and cols are required");
    LR_REQUIRE(n >= 1 && s >= 1 && s <= n, LR_ERR_SHAPE, "need 1 <= s <= n");
    Mat phi = check_thin(Phi, n, s, "Phi");
    Ctx c = make_ctx(h, nullptr, stream);
    srft(n, s, signs, cols, phi.p, phi.ld, c.s);
  });
}

lr_status lr_subspace_iter_backward_uv(lr_handle h, const lr_mat* A, int k, int p, int v, const lr_mat* Omega,
                                       const lr_mat* dU, const lr_mat* dS, const lr_mat* dV, lr_mat* dA,
                                       const lr_opts* opts, void* stream) {
  return guarded(h, [&] {
    AMat a = check_A(A);
    LR_REQUIRE(!a.bf16, LR_ERR_DTYPE, "the reverse pass needs an F32 A");
    check_kpv(a, k, p, v, 2);
    Mat om = check_thin(Omega, a.n, k + p, "Omega");
    LR_REQUIRE(dU || dS || dV, LR_ERR_INVALID_ARG, "need at least one of dU, dS, dV");
    LR_REQUIRE(!dS || (dS->data && dS->dtype == LR_F32 && dS->rows * dS->cols >= k), LR_ERR_SHAPE,
               "dS must hold k F32 weights");
    Mat du, dv;
    if (dU) du = check_thin(dU, a.m, k, "dU");
    if (dV) dv = check_thin(dV, a.n, k, "dV");
    LR_REQUIRE(dA && dA->data && dA->dtype == LR_F32 && dA->col_major == 0 && dA->rows == a.m && dA->cols == a.n &&
                   dA->ld >= a.n,
               LR_ERR_SHAPE, "dA must be an F32 row-major m x n matrix");
    Ctx c = make_ctx(h, opts, stream);
    run_subspace_backward(c, a, k, k + p, v, om, dS ? static_cast<const float*>(dS->data) : nullptr,
                          dU ? &du : nullptr, dV ? &dv : nullptr, static_cast<float*>(dA->data), dA->ld);
  });
}

lr_status lr_subspace_iter_backward(lr_handle h, const lr_mat* A, int k, int p, int v, const lr_mat* Omega,
                                    const lr_mat* dS, lr_mat* dA, const lr_opts* opts, void* stream) {
  if (!dS) return h ? LR_ERR_INVALID_ARG : LR_ERR_INVALID_ARG;
  return lr_subspace_iter_backward_uv(h, A, k, p, v, Omega, nullptr, dS, nullptr, dA, opts, stream);
}

lr_status lr_set_trace(lr_handle h, int on) {
  return guarded(h, [&] {
    LR_CHECK_CUDA(cudaSetDevice(h->device));
    if (on && h->pool.empty()) {
      h->pool.resize(8192);
      for (auto& e : h->pool) LR_CHECK_CUDA(cudaEventCreate(&e));
      h->recs.reserve(4096);
    }
    h->trace = on != 0;
  });
}

lr_status lr_trace_read(lr_handle h, int kind, double* total_ms, int64_t* launches, int reset) {
  return guarded(h, [&] {
    LR_REQUIRE(kind >= 0 && kind < LR_TRACE_COUNT && total_ms && launches, LR_ERR_INVALID_ARG, "bad trace query");
    LR_CHECK_CUDA(cudaSetDevice(h->device));
    LR_CHECK_CUDA(cudaDeviceSynchronize());
    for (const auto& r : h->recs) {
      float ms = 0.f;
      LR_CHECK_CUDA(cudaEventElapsedTime(&ms, r.begin, r.end));
      h->acc_ms[r.kind] += ms;
      h->acc_n[r.kind] += 1;
    }
    h->recs.clear();
    h->pool_used = 0;
    *total_ms = h->acc_ms[kind];
    *launches = h->acc_n[kind];
    if (reset) {
      for (int i = 0; i < LR_TRACE_COUNT; ++i) {
        h->acc_ms[i] = 0.0;
        h->acc_n[i] = 0;
      }
    }
  });
}

lr_status lr_kernel_launches(lr_handle h, uint64_t* count) {
  if (!h || !count) return LR_ERR_INVALID_ARG;
  *count = g_kernel_launches.load();
  return LR_OK;
}

lr_status lr_selftest_bounded_wait(lr_handle h, int64_t timeout_us, void* stream) {
  return guarded(h, [&] {
    LR_REQUIRE(timeout_us >= 1 && timeout_us <= 1000000, LR_ERR_INVALID_ARG, "timeout_us must be in 1..1000000");
    LR_CHECK_CUDA(cudaSetDevice(h->device));
    selftest_bounded_wait(h->status_dev, uint64_t(timeout_us) * 1000u, static_cast<cudaStream_t>(stream));
  });
}

}  // extern "C"
