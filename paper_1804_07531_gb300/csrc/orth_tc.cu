// CholeskyQR2 of one column block of a tall panel (the thin QR between the
// views of Alg. 2 / Alg. 9, the paper's qr) in one cooperative persistent
// kernel whose row products run on the 5th-generation tensor cores.
//
// Each CTA owns the 128-row chunks ch = blockIdx.x, blockIdx.x + grid, ...
// of the m x w panel Y (w <= 128).  A pass stages a chunk in shared memory
// as three BF16 terms, x = h + m + l (each the rounding of what the previous
// terms leave, so the three carry ~24 bits, FP32 accuracy), and multiplies:
//   Gram   G += Y_ch^T Y_ch : S = H^T H + M^T M and X = H^T M + H^T L in
//          TMEM (M = N = 128, K = the chunk's 128 rows), G = S + X + X^T;
//   apply  Q_ch^T = R^{-T} Y_ch^T in TMEM (M = 128 output columns, N = two
//          halves of 64 rows, K = w): the six products of order <= 2 of
//          the terms of R^{-T} and of the chunk.
// The staged chunk is one layout for both: per 64-row half, 128 lines (one
// per column) of 64 BF16 rows, 128-byte swizzled -- the K-major operand of
// the Gram and, through an MN-major descriptor, the B operand of the apply.
// After an apply the epilogue writes the new rows back to Y (in place: rows
// never move between CTAs) and restages them for the next pass's Gram.
//
//   G1 = Y^T Y | R1 = chol(G1): Y <- Y R1^{-1}, G2 = Y^T Y | R2 = chol(G2): Y <- Y R2^{-1}
//   (after a shifted R1: a third pass, and the robust form: a shifted R2 and a fourth pass)
//
// The partial Grams meet in FP64 global buffers (red.add) behind a grid
// barrier; every CTA then factors the same Gram itself (chol_cta.cuh, FP32)
// so the factor never travels back.  One launch per block, one barrier per
// pass.  All waits are bounded (2 s): mbarrier waits on the MMAs and the grid
// barriers record LR_ERR_TIMEOUT and the CTAs return after freeing TMEM.
#include "chol_cta.cuh"
#include "grid_sync.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace lr {
namespace {

using namespace tc;

constexpr int kThreadsT = 256;
constexpr int kRows = 128;                   // rows per chunk
constexpr int kW = 128;                      // widest block
constexpr uint32_t kBox = 16384;             // 64 rows x 128 lines of BF16
constexpr uint32_t kTerm = 2 * kBox;         // one term of a 128 x 128 operand
constexpr int kLd = chol::ld_of(kW);         // 132
// Shared-memory map (bytes from the 1024-aligned base): the three terms of
// R^{-T} at [0, 3 kTerm), the three terms of the staged chunk at
// [3 kTerm, 6 kTerm).  While a Gram is factored the same bytes hold the
// factorisation's arrays: L (and the diagonal blocks of L^{-1}) in the R^{-T}
// part, R^{-1} and the inverse's scratch in the chunk part.
constexpr size_t kOffCH = 3 * size_t(kTerm);
constexpr size_t kOffXd = size_t(kW) * kLd * 4;
constexpr size_t kOffXt = kOffCH;
constexpr size_t kOffT = kOffCH + size_t(kW) * kLd * 4;
constexpr size_t kSmemT = 6 * size_t(kTerm) + 1024;
static_assert(kOffXd + size_t(kW) * chol::kDld * 4 <= kOffCH, "L^{-1} diagonal blocks fit beside L");
static_assert(kOffT + (size_t(chol::kB) * chol::t_ld(kW) + kW + 2 * chol::kB) * 4 <= 6 * size_t(kTerm),
              "the inverse's scratch fits beside R^{-1}");
// TMEM columns: Q^T of a chunk (two halves of 64), then S and X of the Gram
constexpr uint32_t kColQ = 0, kColS = 128, kColX = 256;

struct TcArgs {
  float* Y;           // m x w block (column-major, ld ldy), in place -> Q
  int64_t ldy;
  int64_t m;
  int w;
  double* R;          // the block's triangular factor (w x w, ld ldr), or null
  int ldr;
  float* G;           // Gram buffers G1..G4 (FP32, row-major 128 x 128 each, lower part), zero at launch
  unsigned* ctr;      // grid-barrier counter, zero at launch
  int* gabort;        // raised when a barrier timed out, zero at launch
  int* status;
  int robust;
  int vec;            // Y allows float4 access (16-byte aligned, ld % 4 == 0)
  __nv_bfloat16* ybf; // when not null: BF16 copy of the final Q (ld ldbf, a multiple of 8, 16-byte aligned)
  int64_t ldbf;
};

// x = h + m + l in BF16, each term the rounding of the remainder.
__device__ __forceinline__ void split3(float x, uint32_t& h, uint32_t& m, uint32_t& l) {
  const __nv_bfloat16 bh = __float2bfloat16_rn(x);
  float r = x - __bfloat162float(bh);
  const __nv_bfloat16 bm = __float2bfloat16_rn(r);
  r -= __bfloat162float(bm);
  const __nv_bfloat16 bl = __float2bfloat16_rn(r);
  h = __bfloat16_as_ushort(bh);
  m = __bfloat16_as_ushort(bm);
  l = __bfloat16_as_ushort(bl);
}
// Eight consecutive values (one 16-byte unit of a line) -> the unit in each
// of the three term buffers at byte offset off.
__device__ __forceinline__ void store_unit3(uint8_t* base, uint32_t off, const float (&v)[8]) {
  uint32_t h[8], m[8], l[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) split3(v[j], h[j], m[j], l[j]);
  *reinterpret_cast<uint4*>(base + off) =
      make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
  *reinterpret_cast<uint4*>(base + kTerm + off) =
      make_uint4(m[0] | (m[1] << 16), m[2] | (m[3] << 16), m[4] | (m[5] << 16), m[6] | (m[7] << 16));
  *reinterpret_cast<uint4*>(base + 2 * kTerm + off) =
      make_uint4(l[0] | (l[1] << 16), l[2] | (l[3] << 16), l[4] | (l[5] << 16), l[6] | (l[7] << 16));
}
// Byte offset of unit u (elements 8u .. 8u + 7 along the 128-element K or
// row direction) of line c in an operand term: two boxes of 64, 128-byte
// lines, 16-byte units swizzled by the line index.
__device__ __forceinline__ uint32_t unit_off(int u, int c) {
  return uint32_t(u >> 3) * kBox + uint32_t(c) * 128u + (uint32_t((u & 7) ^ (c & 7)) << 4);
}

// A chunk's rows in flight: each thread loads the eight rows of unit u of
// column c for items it = tid, tid + 256, ... (2048 items, 8 per thread).
struct ChunkRegs {
  float4 v[8][2];
};
__device__ __forceinline__ void chunk_load(const TcArgs& a, int64_t row0, ChunkRegs& cr) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int it = threadIdx.x + i * kThreadsT, u = it & 15, c = it >> 4;
    const int64_t r = row0 + 8 * u;
    float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
    if (c < a.w && r < a.m) {
      const float* p = a.Y + r + int64_t(c) * a.ldy;
      if (a.vec && r + 8 <= a.m) {
        lo = *reinterpret_cast<const float4*>(p);
        hi = *reinterpret_cast<const float4*>(p + 4);
      } else {
        float t[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) t[j] = (r + j < a.m) ? p[j] : 0.f;
        lo = make_float4(t[0], t[1], t[2], t[3]);
        hi = make_float4(t[4], t[5], t[6], t[7]);
      }
    }
    cr.v[i][0] = lo;
    cr.v[i][1] = hi;
  }
}
__device__ __forceinline__ void chunk_stage(uint8_t* ch, const ChunkRegs& cr) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int it = threadIdx.x + i * kThreadsT, u = it & 15, c = it >> 4;
    const float v[8] = {cr.v[i][0].x, cr.v[i][0].y, cr.v[i][0].z, cr.v[i][0].w,
                        cr.v[i][1].x, cr.v[i][1].y, cr.v[i][1].z, cr.v[i][1].w};
    store_unit3(ch, unit_off(u, c), v);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Gram of the staged chunk into S and X (thread 0 issues).  K-major
// operands: line = column (M or N index), 64 rows per line and box.
__device__ __forceinline__ void issue_gram(uint32_t tmem, uint32_t ch, bool accumulate) {
  constexpr uint32_t kId = idesc_bf16(128, false);
  const uint64_t dh0 = sw128_desc(ch, 16, 1024);
#pragma unroll 1
  for (int s = 0; s < 8; ++s) {
    const uint32_t off = uint32_t(s >> 2) * kBox + uint32_t(s & 3) * 32u;
    const uint64_t dh = desc_at(dh0, off);
    const uint64_t dm = desc_at(dh0, kTerm + off);
    const uint64_t dl = desc_at(dh0, 2 * kTerm + off);
    const uint32_t acc = (accumulate || s > 0) ? 1u : 0u;
    umma_bf16(tmem + kColS, dh, dh, kId, acc);  // H^T H
    umma_bf16(tmem + kColS, dm, dm, kId, 1u);   // M^T M
    umma_bf16(tmem + kColX, dh, dm, kId, acc);  // H^T M
    umma_bf16(tmem + kColX, dh, dl, kId, 1u);   // H^T L
  }
}

// kind::f16 instruction descriptor with B MN-major (bit 16), M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16_bmn(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((uint32_t(n) >> 3) << 17) | ((128u >> 4) << 24);
}

// Q_ch^T = R^{-T} Y_ch^T (thread 0 issues): A = R^{-T} (K-major: line = output
// column, K = the block's columns), B = the staged chunk, MN-major (N = its
// 128 rows: the two 64-row halves, one box apart as the leading offset;
// K = 16 columns per step = 16 lines).  One MMA per product and step.
__device__ __forceinline__ void issue_apply(uint32_t tmem, uint32_t rt, uint32_t ch, int ksteps) {
  constexpr uint32_t kId = idesc_bf16_bmn(128);
  const uint64_t da0 = sw128_desc(rt, 16, 1024);    // R^{-T} terms, K-major
  const uint64_t db0 = sw128_desc(ch, kBox, 1024);  // chunk terms, MN-major, halves kBox apart
  const uint32_t d = tmem + kColQ;
#pragma unroll 1
  for (int s = 0; s < ksteps; ++s) {
    const uint32_t aoff = uint32_t(s >> 2) * kBox + uint32_t(s & 3) * 32u;
    const uint64_t ah = desc_at(da0, aoff);
    const uint64_t am = desc_at(da0, kTerm + aoff);
    const uint64_t al = desc_at(da0, 2 * kTerm + aoff);
    const uint32_t boff = uint32_t(s) * 2048u;
    const uint64_t bh = desc_at(db0, boff);
    const uint64_t bm = desc_at(db0, kTerm + boff);
    const uint64_t bl = desc_at(db0, 2 * kTerm + boff);
    umma_bf16(d, ah, bh, kId, s > 0 ? 1u : 0u);
    umma_bf16(d, ah, bm, kId, 1u);
    umma_bf16(d, am, bh, kId, 1u);
    umma_bf16(d, ah, bl, kId, 1u);
    umma_bf16(d, al, bh, kId, 1u);
    umma_bf16(d, am, bm, kId, 1u);
  }
}

struct Sync {
  uint64_t* mbar;
  uint32_t phase;
  volatile int* abort_flag;
  int* status;
};
// thread 0 commits the MMAs issued so far; every thread waits for them.
__device__ __forceinline__ bool mma_done(Sync& s) {
  if (threadIdx.x == 0) umma_commit(s.mbar);
  const bool ok = mbar_wait_warp(s.mbar, s.phase, s.abort_flag, s.status);
  s.phase ^= 1u;
  tc_fence_after();
  return __syncthreads_and(ok) != 0;
}

__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

// S, X (this CTA's Gram partial) -> the lower part of the row-major FP32
// buffer g (ld kW): G(i, j) = S_ij + X_ij + X_ji for j <= i, four entries of a
// row per vector reduction (entries above the diagonal in the last group
// receive zeros and are never read).  X goes through shared memory (xs: 128 x
// 129 floats, free once the pass's last MMA has completed) so that thread i
// also sees column i.  The FP32 sum over the CTAs is far below the rounding
// of the FP32 Cholesky that reads it.  Warp w reads lane quarter w % 4 (Gram
// row i) and column half w / 4.
__device__ __noinline__ void flush_gram(const TcArgs& a, uint32_t tmem, float* g, float* xs) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = (warp & 3) * 32 + lane, j0 = (warp >> 2) * 64;
  const uint32_t lb = tmem + (uint32_t((warp & 3) * 32) << 16);
  float s[64];
#pragma unroll
  for (int gq = 0; gq < 4; ++gq) {
    float x[16], t[16];
    tmem_ld16(lb + kColX + uint32_t(j0 + 16 * gq), x);
#pragma unroll
    for (int u = 0; u < 16; ++u) xs[i * 129 + j0 + 16 * gq + u] = x[u];
    tmem_ld16(lb + kColS + uint32_t(j0 + 16 * gq), t);
#pragma unroll
    for (int u = 0; u < 16; ++u) s[16 * gq + u] = t[u] + x[u];
  }
  __syncthreads();
  if (i >= a.w) return;
#pragma unroll
  for (int t = 0; t < 64; t += 4) {
    const int j = j0 + t;
    if (j > i) break;
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = (j + u <= i) ? s[t + u] + xs[(j + u) * 129 + i] : 0.f;
    red_add_v4(g + i * kW + j, v[0], v[1], v[2], v[3]);
  }
}

// Epilogue of an apply: Q_ch^T from TMEM (lane = output column n, columns =
// rows) -> Y rows (FP32) and, for the next pass's Gram, the staged chunk.
// Warp w: output columns 32 (w % 4) .. + 31, rows of half w / 4.
__device__ __noinline__ void apply_epilogue(const TcArgs& a, uint32_t tmem, int64_t row0, uint8_t* ch,
                                               bool restage) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = (warp & 3) * 32 + lane, half = warp >> 2;
  const uint32_t lb = tmem + (uint32_t((warp & 3) * 32) << 16) + kColQ + uint32_t(half) * 64u;
  float v[64];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    float t[16];
    tmem_ld16(lb + uint32_t(16 * g), t);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[16 * g + j] = t[j];
  }
  const int64_t r0 = row0 + half * 64;
  if (n < a.w && r0 < a.m) {
    float* p = a.Y + r0 + int64_t(n) * a.ldy;
    if (a.vec && r0 + 64 <= a.m) {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        *reinterpret_cast<float4*>(p + 4 * j) = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    } else {
      for (int j = 0; j < 64; ++j)
        if (r0 + j < a.m) p[j] = v[j];
    }
  }
  if (!restage && a.ybf && n < a.w && r0 < a.m) {
    // the last pass also leaves the BF16 copy that a BF16 view of Q reads
    __nv_bfloat16* q = a.ybf + r0 + int64_t(n) * a.ldbf;
    if (r0 + 64 <= a.m) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        uint32_t w4[4];
#pragma unroll
        for (int t = 0; t < 4; ++t)
          w4[t] = uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(v[8 * u + 2 * t]))) |
                  (uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(v[8 * u + 2 * t + 1]))) << 16);
        *reinterpret_cast<uint4*>(q + 8 * u) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
      }
    } else {
      for (int j = 0; j < 64; ++j)
        if (r0 + j < a.m) q[j] = __float2bfloat16_rn(v[j]);
    }
  }
  if (restage) {
    // rows beyond m and columns beyond w stay out of the next Gram
    const bool live = n < a.w;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      float t[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) t[j] = (live && r0 + 8 * u + j < a.m) ? v[8 * u + j] : 0.f;
      store_unit3(ch, unit_off(half * 8 + u, n), t);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
}

// The Gram of one pass (FP32, row-major ld 128, lower part) -> L and R^{-1}
// in shared memory.  Returns 0, LR_ERR_NONFINITE or LR_ERR_BREAKDOWN (the
// same in every CTA: every CTA reads the same Gram).
__device__ __noinline__ int factor(const TcArgs& a, const float* g, int N, bool shift, uint8_t* base, int* sh, double* tr) {
  float* A = reinterpret_cast<float*>(base);
  float* Xd = reinterpret_cast<float*>(base + kOffXd);
  float* Xt = reinterpret_cast<float*>(base + kOffXt);
  float* T = reinterpret_cast<float*>(base + kOffT);
  float* dinv = T + chol::kB * chol::t_ld(N);
  float* colbuf = dinv + N;
  const int tid = threadIdx.x, w = a.w;
  if (tid == 0) *sh = 0;
  __syncthreads();
  bool bad = false;
  // four entries of row r of the lower part per load; consecutive threads
  // take consecutive rows, so the column-major stores into A and Xt fall in
  // distinct banks
  for (int base_i = tid; base_i < N * (N / 4); base_i += 16 * kThreadsT) {
    float4 gv[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int idx = base_i + u * kThreadsT, r = idx % N, c = 4 * (idx / N);
      gv[u] = (idx < N * (N / 4) && r < w && c <= r) ? __ldcg(reinterpret_cast<const float4*>(g + r * kW + c))
                                                      : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int idx = base_i + u * kThreadsT, r = idx % N, c = 4 * (idx / N);
      if (idx >= N * (N / 4)) continue;
      const float e[4] = {gv[u].x, gv[u].y, gv[u].z, gv[u].w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int cc = c + q;
        float v = e[q];
        if (!(r < w && cc < w && cc <= r)) v = (r == cc) ? 1.f : 0.f;  // identity padding, upper part zero
        if (!isfinite(v)) bad = true;
        A[r + cc * kLd] = v;
        Xt[r + cc * kLd] = 0.f;
      }
    }
  }
  if (bad) *sh = 1;
  if (tid < 32) {
    float d[kW / 32];
#pragma unroll
    for (int q = 0; q < kW / 32; ++q) {
      const int i = tid + 32 * q;
      d[q] = i < w ? __ldcg(g + i * kW + i) : 0.f;
    }
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < kW / 32; ++q) t += double(d[q]);
    t = warp_sum(t);
    if (tid == 0) *tr = t;
  }
  __syncthreads();
  if (*sh) return LR_ERR_NONFINITE;
  if (shift) {
    const float s = float(1e-5 * (*tr));
    for (int i = tid; i < w; i += kThreadsT) A[i + i * kLd] += s;
    __syncthreads();
  }
  if (chol::block_chol(A, N, kLd, dinv, colbuf, sh)) return LR_ERR_BREAKDOWN;
  chol::block_inverse(A, Xt, Xd, T, dinv, N, kLd);
  return 0;
}

// R <- R_p R (R = R_1 after the first pass) for columns b = blockIdx.x,
// blockIdx.x + grid, ...; R_p = L^T with L at the start of shared memory.
// Written R + (R_p - I) R, FP32 products, FP64 sum.  stage: 128 floats.
__device__ void update_r(const TcArgs& a, const float* L, bool first, float* stage) {
  const int w = a.w, tid = threadIdx.x;
  for (int b = blockIdx.x; b < w; b += gridDim.x) {
    double* col = a.R + int64_t(b) * a.ldr;
    if (first) {
      for (int r = tid; r < w; r += kThreadsT) col[r] = (r <= b) ? double(L[b + r * kLd]) : 0.0;
      continue;
    }
    for (int k = tid; k <= b; k += kThreadsT) stage[k] = float(col[k]);
    __syncthreads();
    if (tid <= b) {
      float s = 0.f;
      for (int k = tid; k <= b; ++k) s = fmaf(L[k + tid * kLd] - (k == tid ? 1.f : 0.f), stage[k], s);
      col[tid] += double(s);
    }
    __syncthreads();
  }
}

// R^{-1} (FP32, column-major Xt, N x N) -> the three terms of R^{-T}: line n
// holds column n of R^{-1} (K = k), zero beyond N.
__device__ __forceinline__ void stage_rinv(uint8_t* rt, const float* Xt, int N) {
  for (int it = threadIdx.x; it < 16 * kW; it += kThreadsT) {
    const int u = it & 15, n = it >> 4;
    float v[8];
    if (n < N && 8 * u < N) {
      const float4 x0 = *reinterpret_cast<const float4*>(Xt + 8 * u + n * kLd);
      const float4 x1 = *reinterpret_cast<const float4*>(Xt + 8 * u + 4 + n * kLd);
      v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
      v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = 0.f;
    }
    store_unit3(rt, unit_off(u, n), v);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ void run(const TcArgs& a, uint8_t* smem, uint32_t tmem, Sync& sy, int* sh, double* tr) {
  const int tid = threadIdx.x, w = a.w, G = gridDim.x;
  const int N = (w + 31) / 32 * 32;
  const int ksteps = N / 16;
  const int64_t nchunks = (a.m + kRows - 1) / kRows;
  uint8_t* ch = smem + kOffCH;
  const uint32_t ch_s = smem_u32(ch), rt_s = smem_u32(smem);
  unsigned bar = 0;
  ChunkRegs cr;

  // pass 0: G1 = Y^T Y
  {
    int64_t c = blockIdx.x;
    chunk_load(a, c * kRows, cr);
    for (bool first = true; c < nchunks; c += G, first = false) {
      chunk_stage(ch, cr);
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        issue_gram(tmem, ch_s, !first);
      }
      if (c + G < nchunks) chunk_load(a, (c + G) * kRows, cr);  // overlaps the MMAs
      if (!mma_done(sy)) return;
    }
    flush_gram(a, tmem, a.G, reinterpret_cast<float*>(ch));
  }
  if (!gridsync::sync(a.ctr, a.gabort, a.status, bar++, sh)) return;

  int npass = 2;
  bool shifted = false;
  for (int pass = 0; pass < npass; ++pass) {
    const float* g = a.G + pass * kW * kW;
    int err;
    if (pass == 0) {
      err = factor(a, g, N, false, smem, sh, tr);
      if (err == LR_ERR_BREAKDOWN) {
        err = factor(a, g, N, true, smem, sh, tr);
        shifted = true;
        npass = a.robust ? 4 : 3;
      }
    } else {
      err = factor(a, g, N, pass == 1 && shifted && a.robust, smem, sh, tr);
    }
    if (err) {
      if (tid == 0 && blockIdx.x == 0) set_status(a.status, err);
      return;  // every CTA takes the same decision
    }
    if (a.R) update_r(a, reinterpret_cast<const float*>(smem), pass == 0, reinterpret_cast<float*>(smem + kOffXd));
    __syncthreads();
    stage_rinv(smem, reinterpret_cast<const float*>(smem + kOffXt), N);
    __syncthreads();
    const bool gram_next = pass + 1 < npass;
    int64_t c = blockIdx.x;
    chunk_load(a, c * kRows, cr);
    for (bool first = true; c < nchunks; c += G, first = false) {
      chunk_stage(ch, cr);
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        issue_apply(tmem, rt_s, ch_s, ksteps);
      }
      if (!mma_done(sy)) return;
      apply_epilogue(a, tmem, c * kRows, ch, gram_next);
      tc_fence_before();
      __syncthreads();
      if (gram_next && tid == 0) {
        tc_fence_after();
        issue_gram(tmem, ch_s, !first);
      }
      // the next chunk's rows (other rows than this chunk's) load while the
      // Gram MMAs run
      if (c + G < nchunks) chunk_load(a, (c + G) * kRows, cr);
      if (gram_next && !mma_done(sy)) return;
    }
    if (gram_next) {
      flush_gram(a, tmem, a.G + (pass + 1) * kW * kW, reinterpret_cast<float*>(ch));
      if (!gridsync::sync(a.ctr, a.gabort, a.status, bar++, sh)) return;
    }
  }
}

__global__ void __launch_bounds__(kThreadsT, 1) orth_tc_kernel(TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag, sh;
  __shared__ double tr;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    mbar_init(&mbar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  Sync sy{&mbar, 0u, &abort_flag, a.status};
  run(a, smem, tmem_slot, sy, &sh, &tr);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_slot), "r"(512));
  }
}

}  // namespace

bool orth_tc_supported(int64_t m, int w) { return m >= 1 && w >= 1 && w <= kW; }

size_t orth_tc_scratch_doubles(int) { return 4 * size_t(kW) * kW / 2 + 64; }

void orth_tc(float* Y, int64_t ldy, int64_t m, int w, double* R, int ldr, double* scratch, int robust, int* status,
             int device, cudaStream_t s, __nv_bfloat16* ybf, int64_t ldbf) {
  LR_REQUIRE(orth_tc_supported(m, w), LR_ERR_UNSUPPORTED, "orth_tc: block wider than 128");
  static std::atomic<int> grid_cap[64];  // co-resident CTAs, per device
  int cap = grid_cap[device & 63].load();
  if (cap == 0) {
    LR_CHECK_CUDA(cudaFuncSetAttribute(orth_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmemT)));
    int per_sm = 0;
    LR_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, orth_tc_kernel, kThreadsT, kSmemT));
    cap = per_sm * dev_info(device).sms;
    LR_REQUIRE(cap >= 1, LR_ERR_CUDA, "orth_tc: kernel does not fit on an SM");
    grid_cap[device & 63].store(cap);
  }
  const size_t red = orth_tc_scratch_doubles(w);
  LR_CHECK_CUDA(cudaMemsetAsync(scratch, 0, red * sizeof(double), s));
  TcArgs a;
  a.Y = Y;
  a.ldy = ldy;
  a.m = m;
  a.w = w;
  a.R = R;
  a.ldr = ldr;
  a.G = reinterpret_cast<float*>(scratch);
  a.ctr = reinterpret_cast<unsigned*>(scratch + red - 64);
  a.gabort = reinterpret_cast<int*>(scratch + red - 32);
  a.status = status;
  a.robust = robust;
  a.vec = (reinterpret_cast<uintptr_t>(Y) & 15) == 0 && ldy % 4 == 0;
  LR_REQUIRE(!ybf || ((reinterpret_cast<uintptr_t>(ybf) & 15) == 0 && ldbf % 8 == 0 && ldbf >= m), LR_ERR_ALIGNMENT,
             "orth_tc: BF16 copy not 16-byte aligned or its ld not a multiple of 8");
  a.ybf = ybf;
  a.ldbf = ldbf;
  const int64_t nchunks = (m + kRows - 1) / kRows;
  const int grid = int(std::min<int64_t>(cap, nchunks));
  void* args[] = {&a};
  LR_CHECK_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(orth_tc_kernel), dim3(grid),
                                            dim3(kThreadsT), args, kSmemT, s));
  LR_LAUNCH_CHECK();
}

}  // namespace lr
