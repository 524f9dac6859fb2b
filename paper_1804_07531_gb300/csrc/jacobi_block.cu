// One-sided Jacobi SVD of a square core matrix, column blocks on a
// thread-block cluster.
//
// The core SVD (the final tsvd of R_r or R_c in Alg. 2 and Alg. 9, and of the
// small factors of Alg. 7) is an n x n problem with n up to a few hundred;
// one-sided Jacobi rotates column pairs of W = M V until every pair is
// orthogonal to working precision, then sigma_i = |w_i|, u_i = w_i / sigma_i.
// The rotations of one round are disjoint pairs; a sweep pairs every two
// columns once.
//
// Work split.  The columns are split into 2P blocks of b <= 32 columns; CTA
// pi of a cluster of P holds two blocks of W, whole (all rows), in shared
// memory.  A sweep is 2P - 1 block rounds following the circle method over
// the 2P blocks, so every two blocks meet once:
//   * in the first block round of a sweep the CTA pairs all 2b of its
//     columns among themselves (a circle over 2b positions: 2b - 1 local
//     rounds of b pairs): the pairs inside each block and the cross pairs of
//     that round's two blocks;
//   * in the other block rounds it pairs only across its two blocks: in
//     local round s, column i of the first block with column (i + s) mod b
//     of the second (b local rounds of b pairs).
// Every column pair is thus rotated once per sweep, as in a cyclic sweep.  A
// local round costs one barrier of the CTA's W warps: a group of 8 lanes owns
// one pair, each lane 1/8 of the rows as float4, forms the three inner
// products with packed f32x2 FMAs and a 3-level butterfly, and rotates both
// columns (in the cross rounds the first block's column stays in the group's
// registers for the whole block round).  Between block rounds each leaving
// block is one bulk copy shared::cta -> shared::cluster into its next
// holder's second buffer, completing transaction bytes on that CTA's
// mbarrier: 2P - 1 cluster exchanges per sweep.
//
// V.  The rotations of a block round are also applied to J, a 2b x 2b
// identity at the start of the round, so the two blocks' columns of V need
// V <- V J once per block round.  V lives in global memory (the input's
// buffer, n x n, read as M first), and the CTA's V warps apply each J during
// the next block round while the W warps rotate, so V is off the critical
// path and only W moves between CTAs.  Every V column's updates are ordered
// by the cluster barriers between block rounds.
//
// Convergence and faults are decided by the whole cluster from two counters
// kept in every CTA's shared memory: rotations (every CTA adds its count to
// all copies at the end of a sweep) and CTAs that gave up on an mbarrier
// wait (added to all copies at the next exchange).  Every CTA reads its own
// copy after the same cluster barrier, so all leave the loop at the same
// exchange and pass the same barriers afterwards.
//
// Rotation: zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| +
// sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2), s = c t (formed through cos 2theta
// without a division, see angle()), applied when gamma^2 > tol^2 alpha beta
// (tol = eps sqrt(n)).  t only has to be close (an
// inexact angle is still a rotation); c is the refined reciprocal square
// root, so c^2 + s^2 = 1 to about an ulp.  Outputs: sigma_i = |w_i| / |v_i|,
// u_i = w_i / |w_i|, v_i / |v_i|, sorted by sigma descending (ties by index).
#include <cooperative_groups.h>

#include "cluster.cuh"
#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace lr {
namespace {

constexpr int kG = 8;                              // lanes per column pair
constexpr int kPPW = 32 / kG;                      // pairs per warp
constexpr int kMaxB = 32;                          // columns per block: J is at most 64 x 64
// Warps applying V <- V J: 8 where the W side is at most 4 warps and its
// registers leave room (blocks of <= 16 columns, TM <= 12), else 4.
constexpr int kVWarpsMax = 8, kVWarpsMin = 4;
constexpr int kMaxThreads = 32 * ((kMaxB + kPPW - 1) / kPPW + kVWarpsMin);
static_assert(32 * ((16 + kPPW - 1) / kPPW + kVWarpsMax) <= kMaxThreads, "8 V warps fit the bound");
constexpr int kMaxTM = 16;                         // float4 per lane per column: n <= 512
// Threads of the TM = 16 form: its rows take most registers, so it runs only
// with blocks of <= 16 columns (4 + kVWarpsMin warps) and a matching bound.
constexpr int kThreadsTM16 = 32 * ((16 + kPPW - 1) / kPPW + kVWarpsMin);
constexpr int kMaxSweeps = 40;
constexpr uint64_t kTimeoutNs = 2000000000ull;     // bound of every mbarrier wait
constexpr size_t kSmemLimit = size_t(225) * 1024;  // dynamic shared memory per CTA

// Shared-memory geometry, used by the kernel and the host.
struct BGeo {
  int NB, b, npad, TM, ldj, wwarps, threads;
  int ws;        // floats of one block of W
  size_t bytes;
  __host__ __device__ BGeo(int n, int P) {
    NB = 2 * P;                                  // blocks
    b = (n + NB - 1) / NB;                       // columns per block (the last ones zero)
    const int t4 = (n + 4 * kG - 1) / (4 * kG);  // float4 per lane per column, rounded
    TM = t4 <= 4 ? 4 : t4 <= 8 ? 8 : t4 <= 12 ? 12 : 16;  // up to the compiled forms
    npad = 4 * kG * TM;                          // rows, zero-padded
    ldj = 2 * b <= 32 ? 32 : 64;                 // J: 2b x 2b in a ldj x ldj array
    wwarps = (b + kPPW - 1) / kPPW;
    threads = 32 * (wwarps + ((TM == 16 || ldj == 64) ? kVWarpsMin : kVWarpsMax));
    ws = b * npad;
    // [2 buffers][2 slots] blocks of W, J of two block rounds, sigma of
    // every column, |w| and 1/|v| of the local columns
    bytes = (size_t(4) * ws + size_t(2) * ldj * ldj + npad + 2 * 64) * sizeof(float);
  }
};

// The CTA and slot that hold block k in block round r.
__device__ __forceinline__ void holder(int k, int r, int NB, int& cta, int& slot) {
  cta = 0;
  slot = 0;
  for (int pi = 0; pi < NB / 2; ++pi) {
    int p, q;
    round_pair(pi, r, NB, p, q);
    if (p == k || q == k) {
      cta = pi;
      slot = (q == k);
      return;
    }
  }
}

__device__ __forceinline__ void bulk_s2c(uint32_t dst, uint32_t src, uint32_t bytes, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "r"(src), "r"(bytes), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void named_bar(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Packed FP32 pairs (one instruction for two lanes of arithmetic).
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 lo(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi(float4 v) { return make_float2(v.z, v.w); }

// 1 / sqrt(d): the hardware approximation and one Newton step.
__device__ __forceinline__ float rsqrt_nr(float d) {
  const float y = rsqrtf(d);
  return y * fmaf(-0.5f * d * y, y, 1.5f);
}

// The rotation of a pair with |x|^2 = al, |y|^2 = be, x . y = ga (the same
// values in the group's lanes, so the same decision).  With d = be - al and
// r = 1 / sqrt(d^2 + 4 ga^2): cos 2theta = q = |d| r, and with
// u = 1 / sqrt((1 + q) / 2) = 1 / cos theta,
//   c = ((1 + q) / 2) u,   s = sign(d) ga r u,
// which is the angle of t = sign(d) 2 ga / (|d| + sqrt(d^2 + 4 ga^2)).  The
// dependency chain holds two reciprocal square roots and no division; s
// comes from ga directly, so small angles lose no relative accuracy, and
// c^2 + s^2 = u^2 (1 + q) / 2 = 1 up to the (Newton-refined) u.  Where
// d^2 + 4 ga^2 leaves the normal range the same t is formed through zeta.
__device__ __forceinline__ bool angle(float al, float be, float ga, float tol2, float& c, float& s) {
  if (!(al > 0.f && be > 0.f && ga * ga > tol2 * al * be)) return false;
  const float d = be - al, g2 = ga + ga;
  const float h = fmaf(d, d, g2 * g2);
  if (h > 1.0e-30f && h < 3.0e38f) {
    const float r = rsqrtf(h);
    const float hq = fmaf(0.5f, fabsf(d) * r, 0.5f);
    const float u = rsqrt_nr(hq);
    c = hq * u;
    s = copysignf(1.f, d) * (ga * r) * u;
    return true;
  }
  const float zeta = __fdividef(d, g2), az = fabsf(zeta);
  const float t = az < 1e18f ? copysignf(__fdividef(1.f, az + sqrtf(fmaf(zeta, zeta, 1.f))), zeta)
                             : __fdividef(0.5f, zeta);
  c = rsqrt_nr(fmaf(t, t, 1.f));
  s = c * t;
  return true;
}

// [x y] <- [x y] [[c, s], [-s, c]] on float4s.
__device__ __forceinline__ void rot4(float4& x, float4& y, float2 c2, float2 s2, float2 ms2) {
  const float2 xl = fma2(c2, lo(x), mul2(ms2, lo(y))), xh = fma2(c2, hi(x), mul2(ms2, hi(y)));
  const float2 yl = fma2(s2, lo(x), mul2(c2, lo(y))), yh = fma2(s2, hi(x), mul2(c2, hi(y)));
  x = make_float4(xl.x, xl.y, xh.x, xh.y);
  y = make_float4(yl.x, yl.y, yh.x, yh.y);
}

// Partial |x|^2, |y|^2, x . y over a lane's float4s, then the group butterfly.
template <int TM>
__device__ __forceinline__ void dots(const float4 (&x)[TM], const float4 (&y)[TM], float& al, float& be, float& ga) {
  float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0, g0 = a0, g1 = a0;
#pragma unroll
  for (int t = 0; t < TM; ++t) {
      a0 = fma2(lo(x[t]), lo(x[t]), a0);
      a1 = fma2(hi(x[t]), hi(x[t]), a1);
      b0 = fma2(lo(y[t]), lo(y[t]), b0);
      b1 = fma2(hi(y[t]), hi(y[t]), b1);
      g0 = fma2(lo(x[t]), lo(y[t]), g0);
      g1 = fma2(hi(x[t]), hi(y[t]), g1);
    }
  al = (a0.x + a0.y) + (a1.x + a1.y);
  be = (b0.x + b0.y) + (b1.x + b1.y);
  ga = (g0.x + g0.y) + (g1.x + g1.y);
#pragma unroll
  for (int o = kG / 2; o > 0; o >>= 1) {
    al += __shfl_xor_sync(0xffffffffu, al, o);
    be += __shfl_xor_sync(0xffffffffu, be, o);
    ga += __shfl_xor_sync(0xffffffffu, ga, o);
  }
}

// Column p of J: its LDJ rows spread over the group's lanes as float4s.
template <int LDJ>
struct JCol {
  float4 v[LDJ / (4 * kG)];
  __device__ __forceinline__ void load(const float* J, int p, int gl) {
#pragma unroll
    for (int u = 0; u < LDJ / (4 * kG); ++u) v[u] = reinterpret_cast<const float4*>(J + p * LDJ)[gl + kG * u];
  }
  __device__ __forceinline__ void store(float* J, int p, int gl) const {
#pragma unroll
    for (int u = 0; u < LDJ / (4 * kG); ++u) reinterpret_cast<float4*>(J + p * LDJ)[gl + kG * u] = v[u];
  }
};
template <int LDJ>
__device__ __forceinline__ void rot_jc(JCol<LDJ>& x, JCol<LDJ>& y, float2 c2, float2 s2, float2 ms2) {
#pragma unroll
  for (int u = 0; u < LDJ / (4 * kG); ++u) rot4(x.v[u], y.v[u], c2, s2, ms2);
}

// V[:, blocks k0, k1] <- V[:, blocks k0, k1] J for rows t, t + nthr, ..,
// J (2b x 2b in LDJ x LDJ, column-major).  A thread holds its row's 2b
// inputs in registers, so its outputs overwrite them in place; output j is
// the row times column j of J (contiguous, read as broadcast float4s).
template <int LDJ>
__device__ __noinline__ void apply_vj(float* __restrict__ Vw, int ldv, int n, int b, int k0, int k1, const float* J,
                                      int t, int nthr) {
  const int nb2 = 2 * b;
  for (int r = t; r < n; r += nthr) {
    float v[LDJ];
#pragma unroll
    for (int k = 0; k < LDJ; ++k) {
      const int gk = k < b ? k0 * b + k : k1 * b + (k - b);
      v[k] = (k < nb2 && gk < n) ? Vw[r + int64_t(gk) * ldv] : 0.f;
    }
#pragma unroll 2
    for (int j = 0; j < nb2; ++j) {
      const float4* jc = reinterpret_cast<const float4*>(J + j * LDJ);
      float2 acc0 = make_float2(0.f, 0.f), acc1 = acc0;
#pragma unroll
      for (int u = 0; u < LDJ / 4; ++u) {
        const float4 j4 = jc[u];
        acc0 = fma2(make_float2(v[4 * u], v[4 * u + 1]), lo(j4), acc0);
        acc1 = fma2(make_float2(v[4 * u + 2], v[4 * u + 3]), hi(j4), acc1);
      }
      const int gj = j < b ? k0 * b + j : k1 * b + (j - b);
      if (gj < n) Vw[r + int64_t(gj) * ldv] = (acc0.x + acc0.y) + (acc1.x + acc1.y);
    }
  }
}

template <int TM, int LDJ>
__global__ void __launch_bounds__(TM == 16 ? kThreadsTM16 : kMaxThreads, 1)
    jacobi_block_kernel(float* __restrict__ Mw, int ldm, int n, float* __restrict__ Uout, int ldu,
                        float* __restrict__ Vout, int ldv, float* __restrict__ S, int* status) {
  cg::cluster_group cl = cg::this_cluster();
  const int P = int(cl.num_blocks());
  const int rank = int(cl.block_rank());
  const BGeo g(n, P);
  const int NB = g.NB, b = g.b, npad = g.npad, ws = g.ws;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x, nw = nt >> 5;
  const int wthreads = 32 * g.wwarps, vthreads = nt - wthreads;
  const bool is_w = tid < wthreads;
  const int gl = lane % kG;                // lane within the pair group
  const int pi = warp * kPPW + lane / kG;  // the group's pair (W warps)
  const bool live = is_w && pi < b;
  const uint32_t slot_bytes = uint32_t(ws) * 4u;

  extern __shared__ __align__(128) float sm[];
  float* Jb = sm + size_t(4) * ws;  // [2][LDJ][LDJ] J of a block round, column-major
  float* sig = Jb + 2 * LDJ * LDJ;  // sigma of every column (epilogue)
  float* wn = sig + npad;           // |w| of the local columns
  float* vi = wn + 64;              // 1/|v| of the local columns
  __shared__ __align__(8) uint64_t full;  // the blocks of the next round landed
  __shared__ unsigned rot_total;          // rotations so far, all CTAs
  __shared__ unsigned off_bits[2];        // largest |gamma| / sqrt(alpha beta) of a sweep (by parity), all CTAs
  __shared__ unsigned abort_total;        // CTAs that timed out
  __shared__ int timed_out;
  auto slot = [&](int buf, int s) { return sm + size_t(buf * 2 + s) * ws; };
  auto col4 = [&](int buf, int c) {  // local column c in [0, 2b) of buffer buf
    return reinterpret_cast<float4*>(c < b ? slot(buf, 0) + c * npad : slot(buf, 1) + (c - b) * npad);
  };

  // W = M for the blocks of block round 0; then V = I in the same columns of
  // the input's buffer (no other CTA touches them before the first exchange)
  {
    int k0, k1;
    round_pair(rank, 0, NB, k0, k1);
    for (int s = 0; s < 2; ++s) {
      const int k = s ? k1 : k0;
      float* base = slot(0, s);
      for (int idx = tid; idx < ws; idx += nt) {
        const int i = idx / npad, r = idx - i * npad, gi = k * b + i;
        base[idx] = (gi < n && r < n) ? Mw[r + int64_t(gi) * ldm] : 0.f;
      }
    }
    __syncthreads();
    for (int s = 0; s < 2; ++s) {
      const int k = s ? k1 : k0;
      for (int idx = tid; idx < b * n; idx += nt) {
        const int i = idx / n, r = idx - i * n, gi = k * b + i;
        if (gi < n) Mw[r + int64_t(gi) * ldm] = (r == gi) ? 1.f : 0.f;
      }
    }
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    rot_total = 0;
    off_bits[0] = 0;
    off_bits[1] = 0;
    abort_total = 0;
    timed_out = 0;
  }
  // every CTA's barrier and counters are initialised before a peer uses them
  if (P > 1) cluster_barrier();
  else __syncthreads();

  const float tol = 1.2e-7f * sqrtf(float(n));
  const float tol2 = tol * tol;
  // Early stop: the cyclic sweeps converge quadratically, the largest
  // relative off-diagonal of a sweep falling to about 10 times the square of
  // the previous one's (FP64 emulation of this schedule on the workload's
  // core: 8e-4, then 4e-6, then a sweep without rotations).  A sweep whose
  // largest one is below sqrt(tol / 1e4) leaves every pair below tol for any
  // constant up to 1e4, so the loop ends there instead of running one more
  // sweep that would rotate nothing.
  const float stop_off = sqrtf(tol * 1e-4f);
  const uint32_t rot_l = smem_u32(&rot_total), abort_l = smem_u32(&abort_total);
  const uint32_t off_l = smem_u32(&off_bits[0]);  // off_bits[1] follows at + 4
  int cur = 0, rpos = 0, jb = 0;  // W buffer, block round it is placed for, J buffer
  bool pend = false;              // J of the previous block round waits for V
  int pk0 = 0, pk1 = 0;           // its blocks
  uint32_t phase = 0;
  unsigned seen = 0;              // rot_total after the previous sweep
  bool local_abort = false, done = false;
  int sweep = 0;
  for (; sweep < kMaxSweeps && !done; ++sweep) {
    unsigned myrot = 0;  // this lane's rotations in the sweep (group lane 0)
    float myoff = 0.f;   // this group's largest |gamma| / sqrt(alpha beta) in the sweep
    for (int r = 0; r < NB - 1; ++r) {
      int c0, c1;
      round_pair(rank, r, NB, c0, c1);
      if (is_w) {
        // ---- the W warps: local rounds of this block round
        float* J = Jb + jb * LDJ * LDJ;
        for (int idx = tid; idx < LDJ * LDJ; idx += wthreads) J[idx] = (idx / LDJ == idx % LDJ) ? 1.f : 0.f;
        named_bar(1, wthreads);
        if (r == 0) {
          for (int rr = 0; rr < 2 * b - 1; ++rr) {
            int p = 0, q = 1;
            if (live) round_pair(pi, rr, 2 * b, p, q);
            // (a group without a pair reads columns 0 and 1 and discards them)
            float4 x[TM], y[TM];
            float4* xp = col4(cur, p);
            float4* yp = col4(cur, q);
#pragma unroll
            for (int t = 0; t < TM; ++t) {
              x[t] = xp[gl + kG * t];
              y[t] = yp[gl + kG * t];
            }
            JCol<LDJ> jx, jy;
            jx.load(J, p, gl);
            jy.load(J, q, gl);
            float al, be, ga, c, s;
            dots<TM>(x, y, al, be, ga);
            if (live && al > 0.f && be > 0.f) myoff = fmaxf(myoff, fabsf(ga) * rsqrtf(al * be));
            if (live && angle(al, be, ga, tol2, c, s)) {
              const float2 c2 = make_float2(c, c), s2 = make_float2(s, s), ms2 = make_float2(-s, -s);
#pragma unroll
              for (int t = 0; t < TM; ++t) {
                rot4(x[t], y[t], c2, s2, ms2);
                xp[gl + kG * t] = x[t];
                yp[gl + kG * t] = y[t];
              }
              rot_jc<LDJ>(jx, jy, c2, s2, ms2);
              jx.store(J, p, gl);
              jy.store(J, q, gl);
              myrot += (gl == 0);
            }
            named_bar(1, wthreads);
          }
        } else {
          // (a group without a pair reads columns 0 and b and discards them)
          float4 a[TM];
          float4* ap = col4(cur, live ? pi : 0);
#pragma unroll
          for (int t = 0; t < TM; ++t) a[t] = ap[gl + kG * t];
          JCol<LDJ> ja;  // column pi of J, also kept for the block round
          ja.load(J, live ? pi : 0, gl);
          for (int s0 = 0; s0 < b; ++s0) {
            int q = pi + s0;
            if (q >= b) q -= b;
            float4* yp = col4(cur, live ? b + q : b);
            float4 y[TM];
#pragma unroll
            for (int t = 0; t < TM; ++t) y[t] = yp[gl + kG * t];
            JCol<LDJ> jy;
            jy.load(J, live ? b + q : b, gl);
            float al, be, ga, c, s;
            dots<TM>(a, y, al, be, ga);
            if (live && al > 0.f && be > 0.f) myoff = fmaxf(myoff, fabsf(ga) * rsqrtf(al * be));
            if (live && angle(al, be, ga, tol2, c, s)) {
              const float2 c2 = make_float2(c, c), s2 = make_float2(s, s), ms2 = make_float2(-s, -s);
#pragma unroll
              for (int t = 0; t < TM; ++t) {
                rot4(a[t], y[t], c2, s2, ms2);
                yp[gl + kG * t] = y[t];
              }
              rot_jc<LDJ>(ja, jy, c2, s2, ms2);
              jy.store(J, b + q, gl);
              myrot += (gl == 0);
            }
            named_bar(1, wthreads);
          }
          if (live) {
#pragma unroll
            for (int t = 0; t < TM; ++t) ap[gl + kG * t] = a[t];
            ja.store(J, pi, gl);
          }
        }
      } else if (pend) {
        // ---- the V warps: the previous block round's J, meanwhile
        apply_vj<LDJ>(Mw, ldm, n, b, pk0, pk1, Jb + (jb ^ 1) * LDJ * LDJ, tid - wthreads, vthreads);
      }
      const bool sweep_end = r == NB - 2;
      pend = true;
      pk0 = c0;
      pk1 = c1;
      jb ^= 1;

      if (P == 1) {  // one CTA, one block round per sweep: no exchange
        if (sweep_end) {
          const unsigned wr = __reduce_add_sync(0xffffffffu, myrot);
          if (lane == 0 && wr) atomicAdd(&rot_total, wr);
          const unsigned wo = __reduce_max_sync(0xffffffffu, __float_as_uint(myoff));
          if (lane == 0) atomicMax(&off_bits[sweep & 1], wo);
        }
        __syncthreads();
        const unsigned tot = *static_cast<volatile unsigned*>(&rot_total);
        const float offmax = __uint_as_float(*static_cast<volatile unsigned*>(&off_bits[sweep & 1]));
        done = tot == seen || offmax < stop_off;
        seen = tot;
        __syncthreads();
        if (tid == 0) off_bits[(sweep + 1) & 1] = 0;
        continue;
      }

      // ---- exchange: the blocks of W move to their holders of the next round
      const int rn = sweep_end ? 0 : r + 1;
      int n0, n1;
      round_pair(rank, rn, NB, n0, n1);
      // thread writes of this block round -> visible to the bulk copies
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (sweep_end) {
        const unsigned wr = __reduce_add_sync(0xffffffffu, myrot);
        if (wr && lane < P) asm volatile("red.shared::cluster.add.u32 [%0], %1;" ::"r"(mapa(rot_l, lane)), "r"(wr) : "memory");
        const unsigned wo = __reduce_max_sync(0xffffffffu, __float_as_uint(myoff));
        if (wo && lane < P)
          asm volatile("red.shared::cluster.max.u32 [%0], %1;" ::"r"(mapa(off_l + 4u * uint32_t(sweep & 1), lane)), "r"(wo) : "memory");
      }
      if (local_abort && tid < P)
        asm volatile("red.shared::cluster.add.u32 [%0], %1;" ::"r"(mapa(abort_l, tid)), "r"(1u) : "memory");
      if (tid == 0) {
        // the previous sends have finished reading the slots peers refill now
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        if (!local_abort) {
          uint32_t bytes = 0;
          for (int s = 0; s < 2; ++s) {
            int hc, hs;
            holder(s ? n1 : n0, r, NB, hc, hs);
            if (hc != rank) bytes += slot_bytes;
          }
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&full)), "r"(bytes)
                       : "memory");
        }
      }
      // also orders the V warps' global writes before the next holders' reads
      cluster_barrier();
      // every thread reads this CTA's copies of the counters (the same values
      // in every CTA: no CTA adds again before all have arrived at the next
      // barrier, and this one arrives only after these reads)
      const unsigned ab = *static_cast<volatile unsigned*>(&abort_total);
      const unsigned tot = sweep_end ? *static_cast<volatile unsigned*>(&rot_total) : 0u;
      const float offmax =
          sweep_end ? __uint_as_float(*static_cast<volatile unsigned*>(&off_bits[sweep & 1])) : 0.f;
      if (ab) {
        done = true;  // some CTA gave up: all leave here, nothing moves
        break;
      }
      for (int s = 0; s < 2; ++s) {
        int hc, hs;
        holder(s ? c1 : c0, rn, NB, hc, hs);
        if (hc != rank) {
          if (tid == 0)
            bulk_s2c(mapa(smem_u32(slot(cur ^ 1, hs)), hc), smem_u32(slot(cur, s)), slot_bytes,
                     mapa(smem_u32(&full), hc));
        } else {
          const float4* src = reinterpret_cast<const float4*>(slot(cur, s));
          float4* dst = reinterpret_cast<float4*>(slot(cur ^ 1, hs));
          for (int i = tid; i < ws / 4; i += nt) dst[i] = src[i];
        }
      }
      if (tid == 0) asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      if (!local_abort && !mbar_wait_bounded(smem_u32(&full), phase, kTimeoutNs)) {
        timed_out = 1;
        set_status(status, LR_ERR_TIMEOUT);
      }
      __syncthreads();
      local_abort = local_abort || timed_out;
      phase ^= 1u;
      cur ^= 1;
      rpos = rn;
      if (sweep_end) {
        // no rotation anywhere in this sweep, or (early stop) none left to
        // reach tol in the next one
        done = tot == seen || offmax < stop_off;
        seen = tot;
        if (tid == 0) off_bits[(sweep + 1) & 1] = 0;  // no CTA adds to it before the next sweep's last exchange
      }
    }
  }
  if (sweep == kMaxSweeps && !done && rank == 0 && tid == 0) set_status(status, LR_ERR_NONFINITE);
  if (tid == 0 && P > 1) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");

  // ---- the last J, by every thread; then V is complete in the cluster
  __syncthreads();
  if (pend) apply_vj<LDJ>(Mw, ldm, n, b, pk0, pk1, Jb + (jb ^ 1) * LDJ * LDJ, tid, nt);
  if (P > 1) cluster_barrier();
  else __syncthreads();

  // ---- sigma of the local columns, into every CTA's sig[]
  int e0, e1;
  round_pair(rank, rpos, NB, e0, e1);
  for (int c = warp; c < 2 * b; c += nw) {
    const int s = c >= b, i = c - s * b, gi = (s ? e1 : e0) * b + i;
    const float* w = slot(cur, s) + i * npad;
    float sw = 0.f, sv = 0.f;
    for (int r = lane; r < npad; r += 32) sw = fmaf(w[r], w[r], sw);
    if (gi < n)
      for (int r = lane; r < n; r += 32) {
        const float v = Mw[r + int64_t(gi) * ldm];
        sv = fmaf(v, v, sv);
      }
    sw = warp_sum(sw);
    sv = warp_sum(sv);
    const float iv = sv > 0.f ? 1.f / sqrtf(sv) : 0.f;
    if (lane == 0) {
      wn[c] = sqrtf(sw);
      vi[c] = iv;
    }
    if (gi < n && lane < P) cl.map_shared_rank(sig, lane)[gi] = sqrtf(sw) * iv;
  }
  if (P > 1) cluster_barrier();
  else __syncthreads();
  // ---- rank of each local column among all n, and the outputs
  for (int c = warp; c < 2 * b; c += nw) {
    const int s = c >= b, i = c - s * b, gi = (s ? e1 : e0) * b + i;
    if (gi >= n) continue;
    const float sg = sig[gi];
    int cnt = 0;
    for (int d = lane; d < n; d += 32) {
      const float o = sig[d];
      cnt += (o > sg) || (o == sg && d < gi);
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    const float* w = slot(cur, s) + i * npad;
    const float sc = wn[c], iv = vi[c];
    for (int r = lane; r < n; r += 32) {
      Uout[r + int64_t(cnt) * ldu] = sc > 0.f ? w[r] / sc : 0.f;
      Vout[r + int64_t(cnt) * ldv] = Mw[r + int64_t(gi) * ldm] * iv;
    }
    if (lane == 0) S[cnt] = sg;
  }
}

using KernelFn = void (*)(float*, int, int, float*, int, float*, int, float*, int*);

KernelFn kernel_for(const BGeo& g) {
  if (g.ldj == 32)
    return g.TM == 4 ? jacobi_block_kernel<4, 32> : g.TM == 8 ? jacobi_block_kernel<8, 32>
                     : g.TM == 12 ? jacobi_block_kernel<12, 32> : jacobi_block_kernel<16, 32>;
  return g.TM == 4 ? jacobi_block_kernel<4, 64> : g.TM == 8 ? jacobi_block_kernel<8, 64> : jacobi_block_kernel<12, 64>;
}
bool fits(const BGeo& g, int n) {
  if (n > 4 * kG * kMaxTM || g.b > kMaxB || g.bytes > kSmemLimit) return false;
  return g.TM == 16 ? (g.ldj == 32 && g.threads <= kThreadsTM16) : g.threads <= kMaxThreads;
}

cudaLaunchConfig_t config(int n, int P, cudaStream_t s, cudaLaunchAttribute* at) {
  const BGeo g(n, P);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P, 1, 1);
  cfg.blockDim = dim3(g.threads, 1, 1);
  cfg.dynamicSmemBytes = g.bytes;
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = P;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

void set_attrs(KernelFn f) {
  LR_CHECK_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmemLimit)));
  LR_CHECK_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
}

}  // namespace

// Cluster size for the column-block kernel on an n x n core: the smallest P
// whose blocks have at most 16 columns (J of 32 x 32; wider blocks halve the
// exchanges but make V <- V J the longer path, measured slower), else at
// most 32, that fits and whose cluster the device can place; 0 if none.
int jacobi_block_size(int n) {
  static std::atomic<int> cache[64][1025];  // per device and n; 0: not yet known, -1: none
  if (n < 2 || n > 1024) return 0;
  int dev = 0;
  LR_CHECK_CUDA(cudaGetDevice(&dev));
  const int known = cache[dev & 63][n].load();
  if (known != 0) return known > 0 ? known : 0;
  int c = -1;
  for (int i = 0; i < 10; ++i) {
    const int P = 1 << (i % 5);
    const BGeo g(n, P);
    if (!fits(g, n) || (i < 5 && g.ldj != 32)) continue;
    KernelFn f = kernel_for(g);
    set_attrs(f);
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = config(n, P, nullptr, at);
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, f, &cfg) != cudaSuccess) {
      (void)cudaGetLastError();
      clusters = 0;
    }
    if (clusters > 0) {
      c = P;
      break;
    }
  }
  cache[dev & 63][n].store(c);
  return c > 0 ? c : 0;
}

void jacobi_svd_block(float* M, int ldm, int n, float* U, int ldu, float* V, int ldv, float* S, int* status,
                      cudaStream_t s, int P) {
  if (P <= 0) P = jacobi_block_size(n);
  LR_REQUIRE(P == 1 || P == 2 || P == 4 || P == 8 || P == 16, LR_ERR_UNSUPPORTED,
             "core SVD too large for the column-block cluster kernel");
  const BGeo g(n, P);
  LR_REQUIRE(fits(g, n), LR_ERR_UNSUPPORTED, "core SVD blocks do not fit the cluster");
  KernelFn f = kernel_for(g);
  set_attrs(f);
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = config(n, P, s, at);
  LR_CHECK_CUDA(cudaLaunchKernelEx(&cfg, f, M, ldm, n, U, ldu, V, ldv, S, status));
  LR_LAUNCH_CHECK();
}

}  // namespace lr
