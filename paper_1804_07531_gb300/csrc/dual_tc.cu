// The one-read dual sketch of Alg. 7 (Bjarkason 2018, Sec. 6.5, steps a and
// b, which the paper notes are independent): Y = A Omega and Z = A^T Psi from
// ONE pass over a BF16 A on the 5th-generation tensor cores.
//
// Each staged A tile feeds both products before its stage is released:
//   * a CTA owns a strip of 256 rows of A and walks its columns in 64-column
//     k-blocks (persistent grid, stream-K over (strip, k-block));
//   * range:    Y[strip] (256 x ell1, two M = 128 accumulators resident in
//     TMEM for the whole strip) += A_tile (K-major) Omega[k-block];
//   * co-range: Z[k-block]^T (ell2 x 64) = Psi[strip]^T A_tile, the same tile
//     read as an MN-major B operand (N = the tile's 64 columns, K = its 256
//     rows) against Psi's strip (ell2 x 256, K-major), which stays in shared
//     memory for the whole strip;
//   * the Z^T partial of each k-block (double-buffered in TMEM) is added into
//     Z by the epilogue warps with vector reductions (red.global.add.v4.f32);
//     Z (n x ell2 FP32) is small enough to stay in L2, so the partials are
//     reduced there and A is the only operand streamed from HBM.
// That form serves the widths the narrow form below cannot hold (ell2 > 128,
// or ell2 > 64 with ell1 > 64); the narrow form takes 128-column k-blocks and
// the tile as the co-range's M operand.
// Warp roles: 0 TMA producer, 1 MMA issuer (single thread), 2-9 epilogue
// (two warps per TMEM lane quarter).
// Every mbarrier wait is bounded (about 2 s): on expiry the kernel records
// LR_ERR_TIMEOUT, lets issued copies and MMAs finish, frees its TMEM and
// returns.
#include <algorithm>

#include "kernels.h"
#include "tc_common.cuh"

namespace lr {
namespace {

using namespace tc;

constexpr int kThreadsD = 320;               // TMA, MMA, 8 epilogue warps
constexpr int kEpiWarps = 8;
constexpr uint32_t kATile = 32768u;          // 256 rows x 64 BF16
constexpr uint32_t kPsiHalf = 16384u;        // 128 ell2-rows x 64 BF16 (one K chunk)
constexpr size_t kSmemMaxD = 227u * 1024u;   // dynamic shared memory per CTA

// kind::f16 instruction descriptor with B MN-major (bit 16).
__host__ __device__ constexpr uint32_t idesc_bf16_bmn(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((uint32_t(n) >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

template <int NCY, int NH>
struct DCfg {
  static constexpr uint32_t kXBytes = NCY * 128u;              // NCY rows x 64 BF16
  static constexpr uint32_t kStage = kATile + kXBytes;          // multiple of 1024
  static constexpr uint32_t kPsiBytes = 4u * NH * kPsiHalf;     // 4 K chunks of 64 strip rows
  static constexpr int kStages =
      int(std::min<size_t>(4, (kSmemMaxD - kPsiBytes - 2048) / kStage));
  static constexpr size_t kSmem = size_t(kPsiBytes) + size_t(kStages) * kStage + 1024 + 256;
  static constexpr uint32_t kZCol = 2 * NCY;                    // TMEM column of Z^T buffer 0
  static constexpr uint32_t kZBuf = NH * 64;                    // TMEM columns per Z^T buffer
  static_assert(kStages >= 2, "at least a double-buffered ring");
  static_assert(kZCol + 2 * kZBuf <= 512, "TMEM holds 512 FP32 columns");
  static_assert(kSmem <= kSmemMaxD, "shared memory");
};

struct DualParams {
  int64_t m, n;
  int ell1, ell2;
  int kblocks;           // ceil(n / 64)
  int64_t iters_total;   // strips * kblocks
  float* Y;
  int64_t ldy;
  float* Z;
  int64_t ldz;
  int z_vec;             // Z and ldz allow 16-byte vector reductions
  int* status;
};

template <int NCY, int NH>
__global__ void __launch_bounds__(kThreadsD, 1)
    dual_bf16_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX,
                     const __grid_constant__ CUtensorMap tmP, DualParams p) {
  using C = DCfg<NCY, NH>;
  constexpr int S = C::kStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* psi = smem;                                    // [4 chunks][NH halves] 128 x 64 BF16
  uint8_t* ring = smem + C::kPsiBytes;                    // S stages of [A tile | X tile]
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + S * C::kStage);
  uint64_t* empty = full + S;
  uint64_t* psi_full = empty + S;
  uint64_t* psi_empty = psi_full + 1;
  uint64_t* y_full = psi_empty + 1;
  uint64_t* y_empty = y_full + 1;
  uint64_t* z_full = y_empty + 1;   // [2]
  uint64_t* z_empty = z_full + 2;   // [2]
  uint64_t* drain = z_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t G = gridDim.x;
  const int64_t it_begin = p.iters_total * blockIdx.x / G;
  const int64_t it_end = p.iters_total * (blockIdx.x + 1) / G;
  const int kb_n = p.kblocks;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(psi_full, 1);
    mbar_init(psi_empty, 1);
    mbar_init(y_full, 1);
    mbar_init(y_empty, kEpiWarps);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&z_full[b], 1);
      mbar_init(&z_empty[b], kEpiWarps);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------- producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmX)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmP)) : "memory");
      uint32_t stage = 0, phase = 0, psi_phase = 0;
      int64_t it = it_begin;
      bool ok = true;
      while (ok && it < it_end) {
        const int strip = int(it / kb_n);
        const int64_t seg_end = std::min<int64_t>(it_end, int64_t(strip + 1) * kb_n);
        // Psi's strip: 4 chunks of 64 rows x NH halves of 128 columns
        if (!mbar_wait(psi_empty, psi_phase ^ 1u, abort_flag, p.status)) break;
        mbar_expect_tx(psi_full, C::kPsiBytes);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int h = 0; h < NH; ++h)
            tma_load_2d(psi + (q * NH + h) * kPsiHalf, &tmP, psi_full, strip * 256 + q * 64, h * 128);
        psi_phase ^= 1u;
        for (; it < seg_end; ++it) {
          const int kb = int(it % kb_n);
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, p.status)) {
            ok = false;
            break;
          }
          uint8_t* sa = ring + stage * C::kStage;
          mbar_expect_tx(&full[stage], C::kStage);
          tma_load_2d(sa, &tmA, &full[stage], kb * 64, strip * 256);
          tma_load_2d(sa + 16384, &tmA, &full[stage], kb * 64, strip * 256 + 128);
          tma_load_2d(sa + kATile, &tmX, &full[stage], kb * 64, 0);
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (*abort_flag) {  // let copies already issued land before the CTA exits
        const uint64_t t0 = globaltimer();
        while (globaltimer() - t0 < 10000000ull) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t kIdY = idesc_bf16(NCY, false);
      constexpr uint32_t kIdZ = idesc_bf16_bmn(64);
      uint32_t stage = 0, phase = 0, psi_phase = 0, y_phase = 0;
      uint32_t zb = 0, zph = 0;  // Z^T buffer, and the phase bit of each buffer
      int64_t it = it_begin;
      bool ok = true;
      while (ok && it < it_end) {
        const int strip = int(it / kb_n);
        const int64_t seg_end = std::min<int64_t>(it_end, int64_t(strip + 1) * kb_n);
        if (!mbar_wait(psi_full, psi_phase, abort_flag, p.status)) break;
        psi_phase ^= 1u;
        if (!mbar_wait(y_empty, y_phase ^ 1u, abort_flag, p.status)) break;
        tc_fence_after();
        const uint64_t dpsi = sw128_desc(smem_u32(psi), 16, 1024);
        bool first = true;
        for (; it < seg_end; ++it) {
          if (!mbar_wait(&full[stage], phase, abort_flag, p.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_base = smem_u32(ring + stage * C::kStage);
          const uint64_t da = sw128_desc(a_base, 16, 1024);           // A tile, K-major
          const uint64_t dx = sw128_desc(a_base + kATile, 16, 1024);  // X tile
          const uint64_t dam = sw128_desc(a_base, 8192, 1024);        // A tile, MN-major
          // range: Y[s] += A[s] X, K = 64 columns of A in 4 steps of 16
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t bdesc = desc_at(dx, kk * 32);
#pragma unroll
            for (int s = 0; s < 2; ++s)
              umma_bf16(tmem_base + uint32_t(s * NCY), desc_at(da, s * 16384 + kk * 32), bdesc, kIdY,
                        (first && kk == 0) ? 0u : 1u);
          }
          first = false;
          // co-range: Z^T[zb][h] = Psi[strip][h]^T A, K = the 256 rows in 16 steps
          if (!mbar_wait(&z_empty[zb], ((zph >> zb) & 1u) ^ 1u, abort_flag, p.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t zcol = C::kZCol + zb * C::kZBuf;
#pragma unroll
          for (int kk = 0; kk < 16; ++kk) {
            const uint64_t bdesc = desc_at(dam, kk * 2048);
#pragma unroll
            for (int h = 0; h < NH; ++h)
              umma_bf16(tmem_base + zcol + uint32_t(h * 64),
                        desc_at(dpsi, ((kk >> 2) * NH + h) * kPsiHalf + (kk & 3) * 32), bdesc, kIdZ,
                        kk == 0 ? 0u : 1u);
          }
          umma_commit(&z_full[zb]);
          zph ^= 1u << zb;
          zb ^= 1u;
          umma_commit(&empty[stage]);
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        umma_commit(y_full);
        y_phase ^= 1u;
        umma_commit(psi_empty);
      }
      umma_commit(drain);
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < kTimeoutNs) {
      }
    }
  } else {
    // --------------------------------------------------------- epilogue
    // Warps 2..9: warp w reads TMEM lane quarter q = w % 4 (rows q*32 ..
    // q*32+31 of every M = 128 accumulator); the two warps of a quarter split
    // the work: Z^T halves (NH = 2) or column halves (NH = 1), and the two
    // 128-row halves of Y.
    const int q = warp & 3, part = (warp - 2) >> 2;
    const uint32_t lane_base = tmem_base + (uint32_t(q * 32) << 16);
    constexpr int kZCols = NH == 2 ? 64 : 32;  // Z^T columns this warp drains per k-block
    const int zh = NH == 2 ? part : 0;
    const int zc0 = NH == 2 ? 0 : part * 32;
    uint32_t y_phase = 0, zb = 0, zph = 0;
    int64_t it = it_begin;
    bool ok = true;
    while (ok && it < it_end) {
      const int strip = int(it / kb_n);
      const int64_t seg_end = std::min<int64_t>(it_end, int64_t(strip + 1) * kb_n);
      for (; it < seg_end; ++it) {
        const int64_t j0 = int64_t(it % kb_n) * 64 + zc0;  // first column of A this warp reduces
        if (!mbar_wait_warp(&z_full[zb], (zph >> zb) & 1u, abort_flag, p.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        uint32_t r[kZCols / 16][16];
        const uint32_t zaddr = lane_base + C::kZCol + zb * C::kZBuf + uint32_t(zh * 64 + zc0);
#pragma unroll
        for (int g = 0; g < kZCols / 16; ++g) tmem_ld16_nowait(zaddr + uint32_t(g * 16), r[g]);
        tmem_wait_ld();
        tc_fence_before();
        if (lane == 0) mbar_arrive(&z_empty[zb]);  // the accumulator is in registers now
        const int l = zh * 128 + q * 32 + lane;     // the column of Z (index into ell2)
        if (l < p.ell2) {
          float* zl = p.Z + int64_t(l) * p.ldz;
#pragma unroll
          for (int g = 0; g < kZCols / 16; ++g) {
            const int64_t j = j0 + g * 16;
            if (p.z_vec && j + 16 <= p.n) {
#pragma unroll
              for (int u = 0; u < 4; ++u)
                red_add_v4(zl + j + 4 * u, __uint_as_float(r[g][4 * u]), __uint_as_float(r[g][4 * u + 1]),
                           __uint_as_float(r[g][4 * u + 2]), __uint_as_float(r[g][4 * u + 3]));
            } else {
#pragma unroll
              for (int u = 0; u < 16; ++u)
                if (j + u < p.n) atomicAdd(zl + j + u, __uint_as_float(r[g][u]));
            }
          }
        }
        zph ^= 1u << zb;
        zb ^= 1u;
      }
      if (!ok) break;
      // the strip's Y partial (the whole strip when the segment covers all
      // k-blocks): this warp drains the 128-row half `part`
      if (!mbar_wait_warp(y_full, y_phase, abort_flag, p.status)) break;
      tc_fence_after();
      {
        const int s = part;
        const int64_t row = int64_t(strip) * 256 + s * 128 + q * 32 + lane;
        const bool row_ok = row < p.m;
#pragma unroll 1
        for (int c0 = 0; c0 < NCY; c0 += 16) {
          float v[16];
          tmem_ld16(lane_base + uint32_t(s * NCY + c0), v);
          if (row_ok) {
#pragma unroll
            for (int u = 0; u < 16; ++u)
              if (c0 + u < p.ell1) atomicAdd(p.Y + row + int64_t(c0 + u) * p.ldy, v[u]);
          }
        }
      }
      tc_fence_before();
      if (lane == 0) mbar_arrive(y_empty);
      y_phase ^= 1u;
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512));
  }
}

// ------------------------------------------------------------------------
// Narrow co-range sketches (ell2 <= 64, or ell2 <= 128 with ell1 <= 64, so
// that Psi's strip and two stages fit shared memory): 128-column k-blocks,
// and the co-range product with the roles swapped, Z[k-block] (128 columns
// of A x ell2) = A_tile^T Psi[strip]: the staged tile is the MN-major A
// operand (M = its 128 columns, two 64-column boxes LBO apart; K = the
// strip's 256 rows) and Psi's strip the K-major B operand (N = NZ = 64 or
// 128 lines).  One MMA then covers twice the columns of the Psi-as-A form
// (M = 128 lines, N = 64 columns), so a k-block of 128 columns takes 16
// range and 16 co-range MMAs where the 64-column form takes 48 (ell2 <= 64):
// the single issuing thread, not HBM, bounded that form.  TMEM lane = column of A, so
// each epilogue lane adds its column's partials and a warp's reduction
// instruction covers 32 consecutive floats of a column of Z.
constexpr uint32_t kAWide = 65536u;     // 256 rows x 128 columns: boxes (r, c) of 128 x 64 at (2r + c) x 16 KB

// NZ: Psi lines held (the co-range MMA's N), 64 or 128.
template <int NCY, int NZ>
struct WCfg {
  static constexpr uint32_t kXBytes = 2u * NCY * 128u;       // two boxes of NCY lines x 64 BF16
  static constexpr uint32_t kStage = kAWide + kXBytes;       // multiple of 1024
  static constexpr uint32_t kPsiChunk = NZ * 128u;           // 64 strip rows x NZ lines BF16
  static constexpr uint32_t kPsiBytes = 4u * kPsiChunk;      // 4 K chunks of 64 strip rows
  static constexpr int kStages = int(std::min<size_t>(4, (kSmemMaxD - kPsiBytes - 2048) / kStage));
  static constexpr size_t kSmem = size_t(kPsiBytes) + size_t(kStages) * kStage + 1024 + 256;
  static constexpr uint32_t kZCol = 2 * NCY;                 // TMEM column of Z buffer 0
  static constexpr uint32_t kZBuf = NZ;                      // TMEM columns per Z buffer
  static_assert(kStage % 1024 == 0, "stages keep the 1024-byte swizzle alignment");
  static_assert(kStages >= 2, "at least a double-buffered ring");
  static_assert(kZCol + 2 * kZBuf <= 512, "TMEM holds 512 FP32 columns");
  static_assert(kSmem <= kSmemMaxD, "shared memory");
};

template <int NCY, int NZ>
__global__ void __launch_bounds__(kThreadsD, 1)
    dual_wide_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX,
                     const __grid_constant__ CUtensorMap tmP, DualParams p) {
  using C = WCfg<NCY, NZ>;
  constexpr int S = C::kStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* psi = smem;                  // [4 chunks] NZ lines x 64 BF16
  uint8_t* ring = smem + C::kPsiBytes;  // S stages of [A boxes | X boxes]
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + S * C::kStage);
  uint64_t* empty = full + S;
  uint64_t* psi_full = empty + S;
  uint64_t* psi_empty = psi_full + 1;
  uint64_t* y_full = psi_empty + 1;
  uint64_t* y_empty = y_full + 1;
  uint64_t* z_full = y_empty + 1;  // [2]
  uint64_t* z_empty = z_full + 2;  // [2]
  uint64_t* drain = z_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t G = gridDim.x;
  const int64_t it_begin = p.iters_total * blockIdx.x / G;
  const int64_t it_end = p.iters_total * (blockIdx.x + 1) / G;
  const int kb_n = p.kblocks;  // 128-column k-blocks

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(psi_full, 1);
    mbar_init(psi_empty, 1);
    mbar_init(y_full, 1);
    mbar_init(y_empty, kEpiWarps);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&z_full[b], 1);
      mbar_init(&z_empty[b], kEpiWarps);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------- producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmX)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmP)) : "memory");
      uint32_t stage = 0, phase = 0, psi_phase = 0;
      int64_t it = it_begin;
      bool ok = true;
      while (ok && it < it_end) {
        const int strip = int(it / kb_n);
        const int64_t seg_end = std::min<int64_t>(it_end, int64_t(strip + 1) * kb_n);
        // Psi's strip: 4 chunks of 64 rows x NZ lines
        if (!mbar_wait(psi_empty, psi_phase ^ 1u, abort_flag, p.status)) break;
        mbar_expect_tx(psi_full, C::kPsiBytes);
#pragma unroll
        for (int q = 0; q < 4; ++q) tma_load_2d(psi + q * C::kPsiChunk, &tmP, psi_full, strip * 256 + q * 64, 0);
        psi_phase ^= 1u;
        for (; it < seg_end; ++it) {
          const int kb = int(it % kb_n);
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, p.status)) {
            ok = false;
            break;
          }
          uint8_t* sa = ring + stage * C::kStage;
          mbar_expect_tx(&full[stage], C::kStage);
#pragma unroll
          for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 2; ++c)
              tma_load_2d(sa + (2 * r + c) * 16384, &tmA, &full[stage], kb * 128 + c * 64, strip * 256 + r * 128);
#pragma unroll
          for (int c = 0; c < 2; ++c)
            tma_load_2d(sa + kAWide + c * (NCY * 128), &tmX, &full[stage], kb * 128 + c * 64, 0);
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (*abort_flag) {  // let copies already issued land before the CTA exits
        const uint64_t t0 = globaltimer();
        while (globaltimer() - t0 < 10000000ull) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t kIdY = idesc_bf16(NCY, false);
      constexpr uint32_t kIdZ = idesc_bf16(NZ, true);  // A (the tile) MN-major, N = NZ lines of Psi
      uint32_t stage = 0, phase = 0, psi_phase = 0, y_phase = 0;
      uint32_t zb = 0, zph = 0;  // Z buffer, and the phase bit of each buffer
      int64_t it = it_begin;
      bool ok = true;
      while (ok && it < it_end) {
        const int strip = int(it / kb_n);
        const int64_t seg_end = std::min<int64_t>(it_end, int64_t(strip + 1) * kb_n);
        if (!mbar_wait(psi_full, psi_phase, abort_flag, p.status)) break;
        psi_phase ^= 1u;
        if (!mbar_wait(y_empty, y_phase ^ 1u, abort_flag, p.status)) break;
        tc_fence_after();
        const uint64_t dpsi = sw128_desc(smem_u32(psi), 16, 1024);
        bool first = true;
        for (; it < seg_end; ++it) {
          if (!mbar_wait(&full[stage], phase, abort_flag, p.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_base = smem_u32(ring + stage * C::kStage);
          const uint64_t da = sw128_desc(a_base, 16, 1024);            // A boxes, K-major
          const uint64_t dx = sw128_desc(a_base + kAWide, 16, 1024);   // X boxes
          const uint64_t dam = sw128_desc(a_base, 16384, 1024);        // A boxes, MN-major: c = 1 box LBO on
          // range: Y[r] += A[r] X, K = 128 columns in 8 steps of 16
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            const uint32_t c = uint32_t(kk >> 2), ko = uint32_t(kk & 3) * 32u;
            const uint64_t bdesc = desc_at(dx, c * (NCY * 128u) + ko);
#pragma unroll
            for (int r = 0; r < 2; ++r)
              umma_bf16(tmem_base + uint32_t(r * NCY), desc_at(da, (2u * r + c) * 16384u + ko), bdesc, kIdY,
                        (first && kk == 0) ? 0u : 1u);
          }
          first = false;
          // co-range: Z[zb] (128 columns x NZ lines) = A_tile^T Psi[strip], K = 256 rows in 16 steps
          if (!mbar_wait(&z_empty[zb], ((zph >> zb) & 1u) ^ 1u, abort_flag, p.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t zcol = C::kZCol + zb * C::kZBuf;
#pragma unroll
          for (int kk = 0; kk < 16; ++kk)
            umma_bf16(tmem_base + zcol, desc_at(dam, uint32_t(kk >> 3) * 32768u + uint32_t(kk & 7) * 2048u),
                      desc_at(dpsi, uint32_t(kk >> 2) * C::kPsiChunk + uint32_t(kk & 3) * 32u), kIdZ,
                      kk == 0 ? 0u : 1u);
          umma_commit(&z_full[zb]);
          zph ^= 1u << zb;
          zb ^= 1u;
          umma_commit(&empty[stage]);
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        umma_commit(y_full);
        y_phase ^= 1u;
        umma_commit(psi_empty);
      }
      umma_commit(drain);
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < kTimeoutNs) {
      }
    }
  } else {
    // --------------------------------------------------------- epilogue
    // Warps 2..9: warp w reads TMEM lane quarter q = w % 4; the two warps of
    // a quarter take Z lines 0-31 and 32-63 (part), and the two 128-row
    // halves of Y.
    const int q = warp & 3, part = (warp - 2) >> 2;
    const uint32_t lane_base = tmem_base + (uint32_t(q * 32) << 16);
    uint32_t y_phase = 0, zb = 0, zph = 0;
    int64_t it = it_begin;
    bool ok = true;
    while (ok && it < it_end) {
      const int strip = int(it / kb_n);
      const int64_t seg_end = std::min<int64_t>(it_end, int64_t(strip + 1) * kb_n);
      for (; it < seg_end; ++it) {
        const int64_t j = int64_t(it % kb_n) * 128 + q * 32 + lane;  // the column of A this lane adds
        if (!mbar_wait_warp(&z_full[zb], (zph >> zb) & 1u, abort_flag, p.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        constexpr int kG = NZ / 32;  // 16-line groups this warp drains
        uint32_t r[kG][16];
        const uint32_t zaddr = lane_base + C::kZCol + zb * C::kZBuf + uint32_t(part * (NZ / 2));
#pragma unroll
        for (int g = 0; g < kG; ++g) tmem_ld16_nowait(zaddr + uint32_t(16 * g), r[g]);
        tmem_wait_ld();
        tc_fence_before();
        if (lane == 0) mbar_arrive(&z_empty[zb]);  // the accumulator is in registers now
        if (j < p.n) {
          float* zj = p.Z + j;
#pragma unroll
          for (int g = 0; g < kG; ++g)
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              const int l = part * (NZ / 2) + g * 16 + u;
              if (l < p.ell2) atomicAdd(zj + int64_t(l) * p.ldz, __uint_as_float(r[g][u]));
            }
        }
        zph ^= 1u << zb;
        zb ^= 1u;
      }
      if (!ok) break;
      // the strip's Y partial: this warp drains the 128-row half `part`
      if (!mbar_wait_warp(y_full, y_phase, abort_flag, p.status)) break;
      tc_fence_after();
      {
        const int s = part;
        const int64_t row = int64_t(strip) * 256 + s * 128 + q * 32 + lane;
        const bool row_ok = row < p.m;
#pragma unroll 1
        for (int c0 = 0; c0 < NCY; c0 += 16) {
          float v[16];
          tmem_ld16(lane_base + uint32_t(s * NCY + c0), v);
          if (row_ok) {
#pragma unroll
            for (int u = 0; u < 16; ++u)
              if (c0 + u < p.ell1) atomicAdd(p.Y + row + int64_t(c0 + u) * p.ldy, v[u]);
          }
        }
      }
      tc_fence_before();
      if (lane == 0) mbar_arrive(y_empty);
      y_phase ^= 1u;
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512));
  }
}

template <int NCY, int NZ>
void launch_wide(const CUtensorMap& ma, const CUtensorMap& mx, const CUtensorMap& mp, DualParams p, int sms,
                 cudaStream_t s) {
  using C = WCfg<NCY, NZ>;
  auto kern = dual_wide_kernel<NCY, NZ>;
  static std::atomic<bool> attr_set[64];  // attributes set, per device
  int dev = 0;
  LR_CHECK_CUDA(cudaGetDevice(&dev));
  if (!attr_set[dev & 63]) {
    LR_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::kSmem)));
    attr_set[dev & 63] = true;
  }
  const int grid = int(std::min<int64_t>(sms, p.iters_total));
  if (grid <= 0) return;
  kern<<<grid, kThreadsD, C::kSmem, s>>>(ma, mx, mp, p);
  LR_LAUNCH_CHECK();
}

template <int NCY, int NH>
void launch_dual(const CUtensorMap& ma, const CUtensorMap& mx, const CUtensorMap& mp, DualParams p, int sms,
                 cudaStream_t s) {
  using C = DCfg<NCY, NH>;
  auto kern = dual_bf16_kernel<NCY, NH>;
  static std::atomic<bool> attr_set[64];  // attributes set, per device
  int dev = 0;
  LR_CHECK_CUDA(cudaGetDevice(&dev));
  if (!attr_set[dev & 63]) {
    LR_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::kSmem)));
    attr_set[dev & 63] = true;
  }
  const int grid = int(std::min<int64_t>(sms, p.iters_total));
  if (grid <= 0) return;
  kern<<<grid, kThreadsD, C::kSmem, s>>>(ma, mx, mp, p);
  LR_LAUNCH_CHECK();
}

}  // namespace

bool dual_bf16_supported(int ell1, int ell2) { return ell1 >= 1 && ell1 <= 128 && ell2 >= 1 && ell2 <= 256; }

void view_dual_bf16(const DualBf16Args& a, cudaStream_t s) {
  LR_REQUIRE(dual_bf16_supported(a.ell1, a.ell2), LR_ERR_UNSUPPORTED, "fused dual sketch: ell1 <= 128, ell2 <= 256");
  if (a.m <= 0 || a.n <= 0) return;
  DualParams p{};
  p.m = a.m;
  p.n = a.n;
  p.ell1 = a.ell1;
  p.ell2 = a.ell2;
  p.kblocks = ceil_div(a.n, 64);
  p.iters_total = int64_t(ceil_div(a.m, 256)) * p.kblocks;
  p.Y = a.Y;
  p.ldy = a.ldy;
  p.Z = a.Z;
  p.ldz = a.ldz;
  p.z_vec = (reinterpret_cast<uintptr_t>(a.Z) % 16 == 0) && (a.ldz % 4 == 0);
  p.status = a.status;
  const int ncy = a.ell1 <= 32 ? 32 : a.ell1 <= 64 ? 64 : 128;
  const int nh = a.ell2 <= 128 ? 1 : 2;
  // A: m x n row-major; X: n x ell1 column-major (rows = X columns, ld ldx);
  // Psi: m x ell2 column-major (ld ldw)
  CUtensorMap ma = make_map_bf16(a.A, a.n, a.m, a.lda, 64, 128);
  CUtensorMap mx = make_map_bf16(a.X, a.n, a.ell1, a.ldx, 64, ncy);
  CUtensorMap mp = make_map_bf16(a.W, a.m, a.ell2, a.ldw, 64, 128);
  const int sms = dev_info(a.device).sms;
  if (a.ell2 <= 64 || (a.ell2 <= 128 && ncy <= 64)) {
    // 128-column k-blocks, co-range with the tile as the M operand
    p.kblocks = ceil_div(a.n, 128);
    p.iters_total = int64_t(ceil_div(a.m, 256)) * p.kblocks;
    const int nz = a.ell2 <= 64 ? 64 : 128;
    CUtensorMap mpw = make_map_bf16(a.W, a.m, a.ell2, a.ldw, 64, nz);
    if (nz == 64) {
      switch (ncy) {
        case 32: launch_wide<32, 64>(ma, mx, mpw, p, sms, s); break;
        case 64: launch_wide<64, 64>(ma, mx, mpw, p, sms, s); break;
        default: launch_wide<128, 64>(ma, mx, mpw, p, sms, s); break;
      }
    } else {
      switch (ncy) {
        case 32: launch_wide<32, 128>(ma, mx, mpw, p, sms, s); break;
        default: launch_wide<64, 128>(ma, mx, mpw, p, sms, s); break;
      }
    }
  } else if (nh == 1) {
    switch (ncy) {
      case 32: launch_dual<32, 1>(ma, mx, mp, p, sms, s); break;
      case 64: launch_dual<64, 1>(ma, mx, mp, p, sms, s); break;
      default: launch_dual<128, 1>(ma, mx, mp, p, sms, s); break;
    }
  } else {
    switch (ncy) {
      case 32: launch_dual<32, 2>(ma, mx, mp, p, sms, s); break;
      case 64: launch_dual<64, 2>(ma, mx, mp, p, sms, s); break;
      default: launch_dual<128, 2>(ma, mx, mp, p, sms, s); break;
    }
  }
}

}  // namespace lr
