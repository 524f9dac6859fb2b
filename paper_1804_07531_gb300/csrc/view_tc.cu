// BF16 views of A on the 5th-generation tensor cores (tcgen05 + TMA).
//
// A view multiplies the m x n matrix A by a tall thin matrix (the products
// with A and A^T in Alg. 2, Alg. 7 and Alg. 9 of Bjarkason 2018):
//   range view     Y = A X     (mode 0; output rows = rows of A, K = n)
//   co-range view  Z = A^T W   (mode 1; output rows = cols of A, K = rows)
// The path is HBM-bound for the widths the method uses (2 ell / sizeof(bf16)
// flop per byte of A), so the kernel's job is to stream A exactly once at
// full bandwidth while the tensor cores keep up:
//   * persistent grid, one CTA per SM, stream-K split of the flattened
//     (output tile, k-block) iteration space, so every SM gets the same
//     number of A tiles;
//   * warp 0 issues TMA loads of 128-byte-swizzled A tiles and thin-operand
//     tiles into a STAGES-deep shared-memory ring (mbarrier full/empty);
//   * warp 1 issues tcgen05.mma (M = 128, N = padded ell, K = 16) into a
//     TMEM accumulator per 128-row strip; the same swizzled A tile serves as
//     a K-major operand (range) or an MN-major operand (co-range, the
//     transpose is free);
//   * warps 2-5 drain TMEM (tcgen05.ld) and add the partial tile into the
//     FP32 output with atomics (partial tiles exist only where stream-K
//     ranges cut a tile, at most two per CTA).
// Every mbarrier wait is bounded (about 2 s of %globaltimer); on expiry the
// kernel records LR_ERR_TIMEOUT, lets in-flight copies and MMAs finish,
// frees its TMEM and returns.
#include <algorithm>

#include "kernels.h"
#include "tc_common.cuh"

namespace lr {
namespace {

using namespace tc;
constexpr int kThreads = 192;

struct ViewParams {
  int64_t m_out;        // valid output rows
  int ell;              // valid output columns
  int kblocks;          // ceil(K / 64)
  int64_t iters_total;  // tiles * kblocks
  float* out;
  double* out64;        // FP64 output (products accumulated in FP64 across CTAs)
  int64_t ldo;
  int* status;
  const int* run_if;    // the launch is a no-op when *run_if == 0
};

template <int MODE, int NS, int NCOL, int STAGES>
struct Cfg {
  static constexpr uint32_t kABytes = NS * 16384u;       // NS strips of 128 x 64 bf16
  static constexpr uint32_t kBBytes = NCOL * 128u;       // NCOL rows x 64 bf16
  static constexpr uint32_t kStage = kABytes + kBBytes;  // multiple of 1024
  static constexpr uint32_t kTmemCols = (NS * NCOL <= 32) ? 32 : (NS * NCOL <= 64) ? 64 : (NS * NCOL <= 128) ? 128
                                        : (NS * NCOL <= 256) ? 256 : 512;
  static constexpr size_t kSmem = size_t(STAGES) * kStage + 1024 + 256;
  static_assert(NS * NCOL <= 512, "TMEM holds 512 FP32 columns");
  static_assert(NCOL % 16 == 0 && NCOL >= 16 && NCOL <= 256, "M=128 MMA needs N % 16 == 0, N <= 256");
};

template <int MODE, int NS, int NCOL, int STAGES>
__global__ void __launch_bounds__(kThreads, 1)
    view_bf16_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, ViewParams p) {
  using C = Cfg<MODE, NS, NCOL, STAGES>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * C::kStage);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* drain = acc_empty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t G = gridDim.x;
  const int64_t it_begin = p.iters_total * blockIdx.x / G;
  const int64_t it_end = p.iters_total * (blockIdx.x + 1) / G;
  const int kb_n = p.kblocks;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 4);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(C::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
      uint32_t stage = 0, phase = 0;
      for (int64_t it = it_begin; it < it_end; ++it) {
        const int tile = int(it / kb_n);
        const int kb = int(it % kb_n);
        if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, p.status)) break;
        uint8_t* sa = smem + stage * C::kStage;
        uint8_t* sb = sa + C::kABytes;
        mbar_expect_tx(&full[stage], C::kStage);
        if (MODE == 0) {
#pragma unroll
          for (int s = 0; s < NS; ++s) tma_load_2d(sa + s * 16384, &tmA, &full[stage], kb * 64, tile * 128 * NS + s * 128);
        } else {
#pragma unroll
          for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int h = 0; h < 2; ++h)
              tma_load_2d(sa + s * 16384 + h * 8192, &tmA, &full[stage], tile * 128 * NS + s * 128 + h * 64, kb * 64);
        }
        tma_load_2d(sb, &tmB, &full[stage], kb * 64, 0);
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (*abort_flag) {  // let copies already issued land before the CTA exits
        const uint64_t t0 = globaltimer();
        while (globaltimer() - t0 < 10000000ull) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t kIdesc = idesc_bf16(NCOL, MODE == 1);
      uint32_t stage = 0, phase = 0, acc_phase = 0;
      int64_t it = it_begin;
      bool ok = true;
      while (ok && it < it_end) {
        const int tile = int(it / kb_n);
        const int64_t seg_end = (it_end < int64_t(tile + 1) * kb_n) ? it_end : int64_t(tile + 1) * kb_n;
        if (!mbar_wait(acc_empty, acc_phase ^ 1u, abort_flag, p.status)) break;
        tc_fence_after();
        bool first = true;
        for (; it < seg_end; ++it) {
          if (!mbar_wait(&full[stage], phase, abort_flag, p.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_base = smem_u32(smem + stage * C::kStage);
          const uint64_t da = (MODE == 0) ? sw128_desc(a_base, 16, 1024) : sw128_desc(a_base, 8192, 1024);
          const uint64_t db = sw128_desc(a_base + C::kABytes, 16, 1024);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t bdesc = desc_at(db, kk * 32);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
              const uint64_t adesc = desc_at(da, s * 16384 + (MODE == 0 ? kk * 32 : kk * 2048));
              umma_bf16(tmem_base + uint32_t(s * NCOL), adesc, bdesc, kIdesc, (first && kk == 0) ? 0u : 1u);
            }
          }
          first = false;
          umma_commit(&empty[stage]);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        umma_commit(acc_full);
        acc_phase ^= 1u;
      }
      // All MMAs issued by this thread must complete before TMEM is freed.
      umma_commit(drain);
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < kTimeoutNs) {
      }
    }
  } else {
    // Epilogue: warps 2..5 own TMEM lane quarters (warp % 4).
    const int q = warp & 3;
    uint32_t acc_phase = 0;
    int64_t it = it_begin;
    while (it < it_end) {
      const int tile = int(it / kb_n);
      const int64_t seg_end = (it_end < int64_t(tile + 1) * kb_n) ? it_end : int64_t(tile + 1) * kb_n;
      if (!mbar_wait_warp(acc_full, acc_phase, abort_flag, p.status)) break;
      tc_fence_after();
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const int64_t row = int64_t(tile) * 128 * NS + s * 128 + q * 32 + lane;
        const bool row_ok = row < p.m_out;
        float* orow = p.out + row;
#pragma unroll 1
        for (int c0 = 0; c0 < NCOL; c0 += 16) {
          float v[16];
          tmem_ld16(tmem_base + (uint32_t(q * 32) << 16) + uint32_t(s * NCOL + c0), v);
          if (row_ok) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (c0 + j < p.ell) atomicAdd(orow + int64_t(c0 + j) * p.ldo, v[j]);
          }
        }
      }
      tc_fence_before();
      if (lane == 0) mbar_arrive(acc_empty);
      acc_phase ^= 1u;
      it = seg_end;
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(C::kTmemCols));
  }
}

// --------------------------------------------------- FP32 form (3xTF32)
// FP32 views on the tensor cores with FP32-level accuracy: every operand is
// split as x = hi + lo with hi = x truncated to TF32 (low 13 mantissa bits
// cleared) and lo = x - hi (exact in FP32), and the product is
// hi*hi + hi*lo + lo*hi (the dropped lo*lo and the TF32 rounding of lo are
// ~2^-21 relative).  A arrives by TMA as raw FP32 and is split in shared
// memory by four converter warps (hi in place, lo into a twin buffer, then
// fence.proxy.async so the tensor cores see the generic-proxy writes); the
// thin operand comes pre-split.  A 128-byte swizzled row holds 32 FP32
// values, so the descriptors and the 32-byte k-step offsets follow the BF16
// kernel with K = 8 per tcgen05.mma.  Both operands are K-major: for the
// co-range view the converter warps also transpose the staged tile (the
// MN-major operand form the BF16 kernel uses for the co-range view gave
// wrong products with TF32 operands on this GPU).
//
// Accumulation in chunks: the tensor core's FP32 accumulation into TMEM loses
// a little in every MMA (measured: a bias of about -9e-8 of the result per
// 32 K-elements, so -5e-5 at K = 20000), which would exceed the FP32 form's
// error budget on long views.  The MMAs therefore accumulate at most
// kChunkKb k-blocks (256 K-elements) in TMEM; the epilogue warps add each
// chunk into a running sum kept in a second TMEM region with ordinary
// round-to-nearest FP32 additions, and add the running sum into the output
// at the end of the work segment.  The bias is then bounded by one chunk's.
constexpr int kThreadsT = 320;  // TMA, MMA, 4 epilogue, 4 converter warps
constexpr int kChunkKb = 8;     // k-blocks of 32 accumulated in TMEM per chunk

template <int MODE, int NCOL, int STAGES>
struct CfgT {
  static constexpr uint32_t kABytes = 16384u;            // 128 x 32 FP32
  static constexpr uint32_t kBBytes = NCOL * 128u;       // NCOL rows x 32 FP32
  static constexpr uint32_t kStage = 2 * kABytes + 2 * kBBytes;
  // TMEM: the chunk accumulator (NCOL columns) and the running sum (NCOL)
  static constexpr uint32_t kTmemCols = NCOL <= 16 ? 32 : NCOL <= 32 ? 64 : NCOL <= 64 ? 128 : NCOL <= 128 ? 256 : 512;
  static constexpr size_t kSmem = size_t(STAGES) * kStage + 1024 + 256;
  static_assert(NCOL % 16 == 0 && NCOL >= 16 && NCOL <= 256, "M=128 MMA needs N % 16 == 0, N <= 256");
};

// SPLITB: the thin operand arrives raw (one FP32 tile through tmBhi) and the
// converter warps split it in shared memory as well; OUT64: the partial
// products are added into an FP64 output.  Both serve the tall-skinny
// products of the thin QR (Grams P^T Q of long FP32 panels).
template <int MODE, int NCOL, int STAGES, bool SPLITB, bool OUT64>
__global__ void __launch_bounds__(kThreadsT, 1)
    view_tf32x3_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBhi,
                       const __grid_constant__ CUtensorMap tmBlo, ViewParams p) {
  if (p.run_if && *p.run_if == 0) return;
  using C = CfgT<MODE, NCOL, STAGES>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * C::kStage);
  uint64_t* conv = full + STAGES;
  uint64_t* empty = conv + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* drain = acc_empty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t G = gridDim.x;
  const int64_t it_begin = p.iters_total * blockIdx.x / G;
  const int64_t it_end = p.iters_total * (blockIdx.x + 1) / G;
  const int kb_n = p.kblocks;
  // stage s: [A hi | A lo | B hi | B lo]
  auto a_hi = [&](int s) { return smem + s * C::kStage; };
  auto a_lo = [&](int s) { return smem + s * C::kStage + C::kABytes; };
  auto b_hi = [&](int s) { return smem + s * C::kStage + 2 * C::kABytes; };
  auto b_lo = [&](int s) { return smem + s * C::kStage + 2 * C::kABytes + C::kBBytes; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 4);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 4);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(C::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      uint32_t stage = 0, phase = 0;
      for (int64_t it = it_begin; it < it_end; ++it) {
        const int tile = int(it / kb_n);
        const int kb = int(it % kb_n);
        if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, p.status)) break;
        mbar_expect_tx(&full[stage], C::kABytes + (SPLITB ? 1u : 2u) * C::kBBytes);
        if (MODE == 0) {
          tma_load_2d(a_hi(stage), &tmA, &full[stage], kb * 32, tile * 128);
        } else {
#pragma unroll
          for (int h = 0; h < 4; ++h) tma_load_2d(a_hi(stage) + h * 4096, &tmA, &full[stage], tile * 128 + h * 32, kb * 32);
        }
        tma_load_2d(b_hi(stage), &tmBhi, &full[stage], kb * 32, 0);
        if (!SPLITB) tma_load_2d(b_lo(stage), &tmBlo, &full[stage], kb * 32, 0);
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (*abort_flag) {
        const uint64_t t0 = globaltimer();
        while (globaltimer() - t0 < 10000000ull) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t kIdesc = idesc_tf32(NCOL, false);  // both operands K-major
      uint32_t stage = 0, phase = 0, acc_phase = 0;
      int64_t it = it_begin;
      bool ok = true;
      while (ok && it < it_end) {
        const int tile = int(it / kb_n);
        const int64_t seg_end = (it_end < int64_t(tile + 1) * kb_n) ? it_end : int64_t(tile + 1) * kb_n;
        const int64_t chunk_end = (seg_end < it + kChunkKb) ? seg_end : it + kChunkKb;
        if (!mbar_wait(acc_empty, acc_phase ^ 1u, abort_flag, p.status)) break;
        tc_fence_after();
        bool first = true;
        for (; it < chunk_end; ++it) {
          if (!mbar_wait(&conv[stage], phase, abort_flag, p.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t dah0 = sw128_desc(smem_u32(a_hi(stage)), 16, 1024);
          const uint64_t dal0 = sw128_desc(smem_u32(a_lo(stage)), 16, 1024);
          const uint64_t dbh0 = sw128_desc(smem_u32(b_hi(stage)), 16, 1024);
          const uint64_t dbl0 = sw128_desc(smem_u32(b_lo(stage)), 16, 1024);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t dbh = desc_at(dbh0, kk * 32);
            const uint64_t dbl = desc_at(dbl0, kk * 32);
            const uint64_t dah = desc_at(dah0, kk * 32);
            const uint64_t dal = desc_at(dal0, kk * 32);
            umma_tf32(tmem_base, dah, dbh, kIdesc, (first && kk == 0) ? 0u : 1u);
            umma_tf32(tmem_base, dah, dbl, kIdesc, 1u);
            umma_tf32(tmem_base, dal, dbh, kIdesc, 1u);
          }
          first = false;
          umma_commit(&empty[stage]);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        umma_commit(acc_full);
        acc_phase ^= 1u;
      }
      umma_commit(drain);
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < kTimeoutNs) {
      }
    }
  } else if (warp >= 6) {
    // converters: A tile -> hi (in place) and lo
    const int ct = threadIdx.x - 6 * 32;  // 0..127
    uint32_t stage = 0, phase = 0;
    for (int64_t it = it_begin; it < it_end; ++it) {
      if (!mbar_wait_warp(&full[stage], phase, abort_flag, p.status)) break;
      if (MODE == 0) {
        // K-major tile as loaded: split in place, elementwise
        float4* hi = reinterpret_cast<float4*>(a_hi(stage));
        float4* lo = reinterpret_cast<float4*>(a_lo(stage));
#pragma unroll 4
        for (int i = ct; i < int(C::kABytes / 16); i += 128) {
          float4 v = hi[i], h, l;
          h.x = __uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u);
          h.y = __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u);
          h.z = __uint_as_float(__float_as_uint(v.z) & 0xFFFFE000u);
          h.w = __uint_as_float(__float_as_uint(v.w) & 0xFFFFE000u);
          l.x = v.x - h.x;
          l.y = v.y - h.y;
          l.z = v.z - h.z;
          l.w = v.w - h.w;
          hi[i] = h;
          lo[i] = l;
        }
      } else {
        // Co-range: the tile arrives as 4 boxes of [32 K-rows x 32 M-cols]
        // (K = rows of A), 4 KB each.  Box hb holds output rows
        // M = 32 hb .. 32 hb + 31, and those rows of the K-major operand
        // occupy the same 4 KB, so converter warp hb transposes box hb in
        // place: lane mc gathers the 32 K values of column mc (the warp reads
        // one 128-byte source row per step, conflict-free), then writes row
        // M = 32 hb + mc of hi in place and of lo into the twin buffer, in
        // the 128-byte-swizzled K-major layout the MMA reads.
        const float* src = reinterpret_cast<const float*>(a_hi(stage));
        const int mm = ct, hb = mm >> 5, mc = mm & 31;
        float v[32];
#pragma unroll
        for (int k = 0; k < 32; ++k)
          v[k] = src[(hb * 4096 + k * 128 + ((((mc >> 2) ^ (k & 7)) << 4)) + ((mc & 3) << 2)) >> 2];
        __syncwarp();
        float* dhi = reinterpret_cast<float*>(a_hi(stage));
        float* dlo = reinterpret_cast<float*>(a_lo(stage));
#pragma unroll
        for (int kc = 0; kc < 8; ++kc) {
          float4 h, l;
          h.x = __uint_as_float(__float_as_uint(v[4 * kc + 0]) & 0xFFFFE000u);
          h.y = __uint_as_float(__float_as_uint(v[4 * kc + 1]) & 0xFFFFE000u);
          h.z = __uint_as_float(__float_as_uint(v[4 * kc + 2]) & 0xFFFFE000u);
          h.w = __uint_as_float(__float_as_uint(v[4 * kc + 3]) & 0xFFFFE000u);
          l.x = v[4 * kc + 0] - h.x;
          l.y = v[4 * kc + 1] - h.y;
          l.z = v[4 * kc + 2] - h.z;
          l.w = v[4 * kc + 3] - h.w;
          const int off = (mm * 128 + ((kc ^ (mm & 7)) << 4)) >> 2;
          *reinterpret_cast<float4*>(dhi + off) = h;
          *reinterpret_cast<float4*>(dlo + off) = l;
        }
      }
      if (SPLITB) {
        // the thin operand's tile is K-major as loaded: split in place
        float4* hi = reinterpret_cast<float4*>(b_hi(stage));
        float4* lo = reinterpret_cast<float4*>(b_lo(stage));
#pragma unroll 4
        for (int i = ct; i < int(C::kBBytes / 16); i += 128) {
          float4 v = hi[i], h, l;
          h.x = __uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u);
          h.y = __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u);
          h.z = __uint_as_float(__float_as_uint(v.z) & 0xFFFFE000u);
          h.w = __uint_as_float(__float_as_uint(v.w) & 0xFFFFE000u);
          l.x = v.x - h.x;
          l.y = v.y - h.y;
          l.z = v.z - h.z;
          l.w = v.w - h.w;
          hi[i] = h;
          lo[i] = l;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&conv[stage]);
      if (++stage == STAGES) {
        stage = 0;
        phase ^= 1u;
      }
    }
  } else {
    // Epilogue: warps 2..5 own TMEM lane quarters (warp % 4).  Per chunk:
    // running (+)= chunk; at the segment's last chunk the sum goes out.
    const int q = warp & 3;
    const uint32_t lane_base = tmem_base + (uint32_t(q * 32) << 16);
    uint32_t acc_phase = 0;
    int64_t it = it_begin;
    bool first_chunk = true;
    while (it < it_end) {
      const int tile = int(it / kb_n);
      const int64_t seg_end = (it_end < int64_t(tile + 1) * kb_n) ? it_end : int64_t(tile + 1) * kb_n;
      const int64_t chunk_end = (seg_end < it + kChunkKb) ? seg_end : it + kChunkKb;
      const bool last_chunk = chunk_end == seg_end;
      if (!mbar_wait_warp(acc_full, acc_phase, abort_flag, p.status)) break;
      tc_fence_after();
      const int64_t row = int64_t(tile) * 128 + q * 32 + lane;
      const bool row_ok = row < p.m_out;
#pragma unroll 1
      for (int c0 = 0; c0 < NCOL; c0 += 16) {
        float v[16];
        tmem_ld16(lane_base + uint32_t(c0), v);
        if (!first_chunk) {
          float r[16];
          tmem_ld16(lane_base + uint32_t(NCOL + c0), r);
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] += r[j];
        }
        if (!last_chunk) {
          tmem_st16(lane_base + uint32_t(NCOL + c0), v);
        } else if (row_ok) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c0 + j < p.ell) {
              if (OUT64) atomicAdd(p.out64 + row + int64_t(c0 + j) * p.ldo, double(v[j]));
              else atomicAdd(p.out + row + int64_t(c0 + j) * p.ldo, v[j]);
            }
        }
      }
      if (!last_chunk) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      tc_fence_before();
      if (lane == 0) mbar_arrive(acc_empty);
      acc_phase ^= 1u;
      first_chunk = last_chunk;
      it = chunk_end;
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(C::kTmemCols));
  }
}

__global__ void split_tf32_kernel(const float* __restrict__ src, int64_t lds, float* __restrict__ hi,
                                  float* __restrict__ lo, int64_t ldd, int64_t rows, int64_t cols, float scale,
                                  int trans) {
  for (int64_t c = blockIdx.y; c < cols; c += gridDim.y)
    for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < rows; r += int64_t(gridDim.x) * blockDim.x) {
      const float x = scale * (trans ? src[c + r * lds] : src[r + c * lds]);
      const float h = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
      hi[r + c * ldd] = h;
      lo[r + c * ldd] = x - h;
    }
}

// ------------------------------------------------------------------ host
// Grid of a view launch.  Stream-K by default: min(SMs, iterations), each
// CTA a contiguous range of (tile, k-block) iterations.  When the thin
// operand is larger than L2 and there are fewer output tiles than SMs (the
// co-range view of a tall panel), the CTAs that share a tile start at
// different k-blocks under stream-K, so every CTA streams its own rows of the
// operand from HBM (about one full read of it per tile).  There the grid is
// tiles x floor(SMs / tiles) instead: each CTA takes one K slice of one tile,
// the CTAs of a slice start at the same k-block and advance together, and
// each block of operand rows is read from HBM once and from L2 by the others.
inline int view_grid(int64_t iters_total, int tiles, int sms, double b_bytes) {
  if (b_bytes > 48.0 * 1024 * 1024 && tiles > 0 && tiles < sms) return tiles * (sms / tiles);
  return int(std::min<int64_t>(sms, iters_total));
}

template <int MODE, int NCOL>
void launch_ncol(const CUtensorMap& ma, const CUtensorMap& mb, ViewParams p, int tiles, int sms, cudaStream_t s,
                 double b_bytes = 0) {
  constexpr int NS = 2;
  constexpr int STAGES = (NCOL <= 128) ? 4 : 3;
  using C = Cfg<MODE, NS, NCOL, STAGES>;
  auto kern = view_bf16_kernel<MODE, NS, NCOL, STAGES>;
  static std::atomic<bool> attr_set[64];  // attributes set, per device
  int dev = 0;
  LR_CHECK_CUDA(cudaGetDevice(&dev));
  if (!attr_set[dev & 63]) {
    LR_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::kSmem)));
    attr_set[dev & 63] = true;
  }
  p.iters_total = int64_t(tiles) * p.kblocks;
  int grid = view_grid(p.iters_total, tiles, sms, b_bytes);
  if (grid <= 0) return;
  kern<<<grid, kThreads, C::kSmem, s>>>(ma, mb, p);
  LR_LAUNCH_CHECK();
}

}  // namespace

int view_bf16_ncol(int ell) {
  return ell <= 32 ? 32 : ell <= 64 ? 64 : ell <= 128 ? 128 : 256;
}

void view_bf16(const ViewBf16Args& a, cudaStream_t s) {
  LR_REQUIRE(a.ell >= 1 && a.ell <= 256, LR_ERR_UNSUPPORTED, "bf16 view handles ell <= 256 per call");
  if (a.rows <= 0 || a.n <= 0) return;
  const int sms = dev_info(a.device).sms;
  const __nv_bfloat16* abase = a.A + a.row0 * a.lda;
  ViewParams p{};
  p.ell = a.ell;
  p.out = a.out;
  p.ldo = a.ldo;
  p.status = a.status;
  const int ncol = view_bf16_ncol(a.ell);
  if (a.mode == 0) {
    // Y[row0 : row0+rows] += A[row0 : row0+rows, :] X ; X col-major n x ell (ld ldb)
    CUtensorMap ma = make_map_bf16(abase, a.n, a.rows, a.lda, 64, 128);
    CUtensorMap mb = make_map_bf16(a.B, a.n, a.ell, a.ldb, 64, ncol);
    p.m_out = a.rows;
    p.kblocks = ceil_div(a.n, 64);
    const int tiles = ceil_div(a.rows, 256);
    switch (ncol) {
      case 32: launch_ncol<0, 32>(ma, mb, p, tiles, sms, s); break;
      case 64: launch_ncol<0, 64>(ma, mb, p, tiles, sms, s); break;
      case 128: launch_ncol<0, 128>(ma, mb, p, tiles, sms, s); break;
      default: launch_ncol<0, 256>(ma, mb, p, tiles, sms, s); break;
    }
  } else {
    // Z += A[row0 : row0+rows, :]^T W_band ; W_band col-major (rows x ell,
    // ld ldb) holds the operand rows of this band.
    CUtensorMap ma = make_map_bf16(abase, a.n, a.rows, a.lda, 64, 64);
    CUtensorMap mb = make_map_bf16(a.B, a.rows, a.ell, a.ldb, 64, ncol);
    p.m_out = a.n;
    p.kblocks = ceil_div(a.rows, 64);
    const int tiles = ceil_div(a.n, 256);
    const double bb = double(a.rows) * ncol * 2;  // the BF16 operand rows this launch reads
    switch (ncol) {
      case 32: launch_ncol<1, 32>(ma, mb, p, tiles, sms, s, bb); break;
      case 64: launch_ncol<1, 64>(ma, mb, p, tiles, sms, s, bb); break;
      case 128: launch_ncol<1, 128>(ma, mb, p, tiles, sms, s, bb); break;
      default: launch_ncol<1, 256>(ma, mb, p, tiles, sms, s, bb); break;
    }
  }
}


namespace {
template <int MODE, int NCOL, bool SPLITB = false, bool OUT64 = false>
void launch_tf32(const CUtensorMap& ma, const CUtensorMap& mbh, const CUtensorMap& mbl, ViewParams p, int tiles,
                 int sms, cudaStream_t s, double b_bytes = 0) {
  constexpr int STAGES = (NCOL <= 64) ? 4 : (NCOL <= 128) ? 3 : 2;
  using C = CfgT<MODE, NCOL, STAGES>;
  auto kern = view_tf32x3_kernel<MODE, NCOL, STAGES, SPLITB, OUT64>;
  static std::atomic<bool> attr_set[64];  // attributes set, per device
  int dev = 0;
  LR_CHECK_CUDA(cudaGetDevice(&dev));
  if (!attr_set[dev & 63]) {
    LR_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::kSmem)));
    attr_set[dev & 63] = true;
  }
  p.iters_total = int64_t(tiles) * p.kblocks;
  const int grid = view_grid(p.iters_total, tiles, sms, b_bytes);
  if (grid <= 0) return;
  kern<<<grid, kThreadsT, C::kSmem, s>>>(ma, mbh, mbl, p);
  LR_LAUNCH_CHECK();
}
}  // namespace

void split_tf32(const float* src, int64_t lds, float* hi, float* lo, int64_t ldd, int64_t rows, int64_t cols,
                cudaStream_t s, float scale, bool trans) {
  if (rows <= 0 || cols <= 0) return;
  split_tf32_kernel<<<grid_2d(rows, cols), 256, 0, s>>>(src, lds, hi, lo, ldd, rows, cols, scale, trans ? 1 : 0);
  LR_LAUNCH_CHECK();
}

void gram_tf32x3(const GramTf32Args& a, cudaStream_t s) {
  LR_REQUIRE(a.b >= 1 && a.b <= 256, LR_ERR_UNSUPPORTED, "tensor-core Gram handles b <= 256 per call");
  if (a.a <= 0 || a.m <= 0) return;
  const int sms = dev_info(a.device).sms;
  ViewParams p{};
  p.ell = a.b;
  p.out64 = a.C64;
  p.ldo = a.ldc;
  p.status = a.status;
  p.run_if = a.run_if;
  p.m_out = a.a;
  p.kblocks = ceil_div(a.m, 32);
  const int ncol = view_bf16_ncol(a.b);
  // A = P^T (a x m row-major, row stride lda); B = Q (m x b col-major), raw
  CUtensorMap ma = make_map_f32(a.P, a.m, a.a, a.lda, 32, 128);
  CUtensorMap mb = make_map_f32(a.Q, a.m, a.b, a.ldb, 32, ncol);
  const int tiles = ceil_div(a.a, 128);
  switch (ncol) {
    case 32: launch_tf32<0, 32, true, true>(ma, mb, mb, p, tiles, sms, s); break;
    case 64: launch_tf32<0, 64, true, true>(ma, mb, mb, p, tiles, sms, s); break;
    case 128: launch_tf32<0, 128, true, true>(ma, mb, mb, p, tiles, sms, s); break;
    default: launch_tf32<0, 256, true, true>(ma, mb, mb, p, tiles, sms, s); break;
  }
}

void view_tf32x3(const ViewTf32Args& a, cudaStream_t s) {
  LR_REQUIRE(a.ell >= 1 && a.ell <= 256, LR_ERR_UNSUPPORTED, "tf32 view handles ell <= 256 per call");
  if (a.rows <= 0 || a.n <= 0) return;
  const int sms = dev_info(a.device).sms;
  const float* abase = a.A + a.row0 * a.lda;
  ViewParams p{};
  p.ell = a.ell;
  p.out = a.out;
  p.ldo = a.ldo;
  p.status = a.status;
  p.run_if = a.run_if;
  const int ncol = view_bf16_ncol(a.ell);
  if (a.mode == 0) {
    CUtensorMap ma = make_map_f32(abase, a.n, a.rows, a.lda, 32, 128);
    CUtensorMap mh = make_map_f32(a.Bhi, a.n, a.ell, a.ldb, 32, ncol);
    CUtensorMap ml = make_map_f32(a.Blo, a.n, a.ell, a.ldb, 32, ncol);
    p.m_out = a.rows;
    p.kblocks = ceil_div(a.n, 32);
    const int tiles = ceil_div(a.rows, 128);
    switch (ncol) {
      case 32: launch_tf32<0, 32>(ma, mh, ml, p, tiles, sms, s); break;
      case 64: launch_tf32<0, 64>(ma, mh, ml, p, tiles, sms, s); break;
      case 128: launch_tf32<0, 128>(ma, mh, ml, p, tiles, sms, s); break;
      default: launch_tf32<0, 256>(ma, mh, ml, p, tiles, sms, s); break;
    }
  } else {
    CUtensorMap ma = make_map_f32(abase, a.n, a.rows, a.lda, 32, 32);
    CUtensorMap mh = make_map_f32(a.Bhi, a.rows, a.ell, a.ldb, 32, ncol);
    CUtensorMap ml = make_map_f32(a.Blo, a.rows, a.ell, a.ldb, 32, ncol);
    p.m_out = a.n;
    p.kblocks = ceil_div(a.rows, 32);
    const int tiles = ceil_div(a.n, 128);
    const double bb = double(a.rows) * ncol * 8;  // the TF32 hi + lo operand rows this launch reads
    switch (ncol) {
      case 32: launch_tf32<1, 32>(ma, mh, ml, p, tiles, sms, s, bb); break;
      case 64: launch_tf32<1, 64>(ma, mh, ml, p, tiles, sms, s, bb); break;
      case 128: launch_tf32<1, 128>(ma, mh, ml, p, tiles, sms, s, bb); break;
      default: launch_tf32<1, 256>(ma, mh, ml, p, tiles, sms, s, bb); break;
    }
  }
}

}  // namespace lr
