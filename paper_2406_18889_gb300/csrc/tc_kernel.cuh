// Tensor-core GEMM kernel (tcgen05 + TMA + TMEM) for the reduced-precision
// complex path; included by one translation unit per tile width
// (k_gemm_tc_bn*.cu), each of which instantiates launch_tc_tiles<BN>.
//
// A pairwise contraction (arXiv 2406.18889, Sec. III, per-step contraction) in
// complex numbers is lowered to ONE real GEMM ("stacked 4M"): with complex
// elements stored interleaved (re, im) in fp16/bf16,
//   A'[m][2k+r]          = (Re A, Im A)[m][k]            (A used as stored)
//   B'[2n+c][2k+r]       = [[Re B, -Im B], [Im B, Re B]]  (expanded from B)
//   C'[m][2n+c] = sum_k' A'[m][k'] B'[2n+c][k']  = (Re C, Im C)[m][n]
// so the real GEMM's output is already interleaved complex.  8 real flops per
// complex multiply-add: the useful flop count of the paper's Table I
// convention, with no 3M cancellation.
//
// Kernel: persistent CTAs over 128 x BN output tiles (real columns), 2 + 16 warps:
//   warp 0      TMA producer: 3-D tiled loads of A' (box 64 x 128) and B'
//               (box 64 x BN), 128-byte swizzle, into a ring of stages;
//   warp 1      allocates 2 x BN TMEM columns (double-buffered accumulator);
//               one thread issues tcgen05.mma (kind::f16, M = 128, N = BN,
//               K = 16, FP32 accumulate in TMEM); tcgen05.commit releases ring
//               stages and hands finished accumulators to the epilogue;
//   warps 2..17 epilogue: tcgen05.ld of the accumulator (warp w reads TMEM
//               lanes 32*(w%4)..+31; four warps per lane quarter share its
//               32-column chunks), scale by 2^shift, convert, store -- directly along
//               m, or (STAGE) transposed through shared memory so that lanes
//               run along n when n is the output's contiguous index.
// Every mbarrier wait is bounded by the global timer (2 s); on timeout the
// kernel raises the device error flag and every role stops; the producer and
// the MMA thread drain their own in-flight work (bounded) before TMEM is freed.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <cstring>

#include "tn_internal.h"

namespace tn {

constexpr int kTcBK = kTcKTile;  // real k per stage: one 128-byte swizzle row of 16-bit values

namespace {

constexpr int BM = 128;
constexpr int BK = kTcBK;
constexpr uint64_t kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// true when the phase with `parity` has completed; false on abort or after
// limit_ns nanoseconds (then *err is raised)
__device__ bool wait_bounded_ns(uint64_t* bar, uint32_t parity, int* err, uint64_t limit_ns) {
  const uint64_t t0 = gtimer();
  for (uint32_t i = 0; !mbar_try_wait(bar, parity); ++i) {
    // another role's timeout: the flag is read every 64 polls (a global load
    // per poll would keep waiting warps on the memory pipe)
    if ((i & 63) == 63 && *(volatile int*)err) return false;
    if (gtimer() - t0 > limit_ns) {
      atomicExch(err, 1);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity, int* err) {
  return wait_bounded_ns(bar, parity, err, kWaitNs);
}
__device__ __forceinline__ void tma_load_3d(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y,
                                            int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}
// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// groups 1024 bytes apart (SBO), descriptor version 1 (tcgen05)
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // version
  d |= (uint64_t)2 << 61;             // swizzle: 128B
  return d;
}
// instruction descriptor, kind::f16: D = F32, A/B = F16 (0) or BF16 (1), both K-major
__host__ __device__ constexpr uint32_t make_idesc(int n, bool bf16) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}

// epilogue staging: per warp 32 rows x 16 complex (padded) + 32 row offsets
constexpr int kStagePitch = 17;
constexpr int kEpiWarps = 16;  // four warps per TMEM lane quarter, each taking every fourth column chunk
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr size_t kStageBytes = kEpiWarps * 32 * kStagePitch * 8 + kEpiWarps * 32 * 8;

// ring depth: as many stages as fit in 227 KB of shared memory next to the
// barriers, the column-offset table and (STAGE) the epilogue staging, at most
// 8 (a deeper ring of narrow tiles measured slower: 11 stages at tile width
// 32 took the 4096 x 4096 x 16 x 16 step from 0.524 to 0.562 ms)
template <int BN, bool STAGE = false, int MH = 1>
__host__ __device__ constexpr int stages_for() {
  constexpr long budget = 232448 - 1024 - 512 - (long)BN / 2 * 12 - (STAGE ? (long)kStageBytes : 0L) - 512;
  constexpr long per = (long)(MH * BM + BN) * BK * 2;
  return budget / per > 8 ? 8 : (int)(budget / per);
}
template <int BN, bool STAGE, int MH = 1>
__host__ __device__ constexpr size_t smem_bytes() {
  return 1024 + (size_t)stages_for<BN, STAGE, MH>() * (MH * BM + BN) * BK * 2 + 512 + (size_t)BN / 2 * 12 +
         (STAGE ? kStageBytes : 0);
}


// Coordinates of the tiles t0, t0 + step, t0 + 2 step, ... (t = (bt * n_mu + m)
// * n_n + n).  Walking: one division when the walk starts, then a mixed-radix
// add per tile instead of three 64-bit divisions.  Not walking (register-lean):
// the divisions, per tile.
template <bool kWalk>
struct TileWalk {
  int n, m, b;     // current tile
  int dn, dm, db;  // the step in the same radix
  int n_n, n_mu;
  __device__ __forceinline__ TileWalk(int64_t t0, int64_t step, int64_t nn, int64_t nmu)
      : n_n((int)nn), n_mu((int)nmu) {
    n = (int)(t0 % nn);
    m = (int)((t0 / nn) % nmu);
    b = (int)(t0 / (nn * nmu));
    dn = (int)(step % nn);
    dm = (int)((step / nn) % nmu);
    db = (int)(step / (nn * nmu));
  }
  __device__ __forceinline__ void next() {
    n += dn;
    const int cn = n >= n_n;
    n -= cn ? n_n : 0;
    m += dm + cn;
    const int cm = m >= n_mu;
    m -= cm ? n_mu : 0;
    b += db + cm;
  }
  __device__ __forceinline__ void at(int64_t, int& n_tile, int& m_unit, int& bt) const {
    n_tile = n;
    m_unit = m;
    bt = b;
  }
};
template <>
struct TileWalk<false> {
  int64_t n_n, n_mu;
  __device__ __forceinline__ TileWalk(int64_t, int64_t, int64_t nn, int64_t nmu) : n_n(nn), n_mu(nmu) {}
  __device__ __forceinline__ void next() {}
  __device__ __forceinline__ void at(int64_t t, int& n_tile, int& m_unit, int& bt) const {
    n_tile = (int)(t % n_n);
    m_unit = (int)((t / n_n) % n_mu);
    bt = (int)(t / (n_n * n_mu));
  }
};

// complex value -> one 32-bit word of two 16-bit reals
template <bool BF16>
__device__ __forceinline__ uint32_t pack16(float re, float im) {
  uint32_t w;
  if constexpr (BF16) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
    memcpy(&w, &h, 4);
  } else {
    const __half2 h = __floats2half2_rn(re, im);
    memcpy(&w, &h, 4);
  }
  return w;
}
// rounding residual of (re, im) given its 16-bit word
template <bool BF16>
__device__ __forceinline__ uint32_t resid16(float re, float im, uint32_t w) {
  float2 h;
  if constexpr (BF16) {
    __nv_bfloat162 x;
    memcpy(&x, &w, 4);
    h = __bfloat1622float2(x);
  } else {
    __half2 x;
    memcpy(&x, &w, 4);
    h = __half22float2(x);
  }
  return pack16<BF16>(re - h.x, im - h.y);
}
// the same at 32-bit element offset o from a tile's base pointers; the
// residual goes to C2t when it is non-null (the output is stored hi + lo)
template <bool BF16, bool F32OUT>
__device__ __forceinline__ void store_el32(char* Ct, char* C2t, uint32_t o, float re, float im) {
  if constexpr (F32OUT) {
    *reinterpret_cast<float2*>(Ct + (size_t)o * 8) = make_float2(re, im);
  } else {
    const uint32_t h = pack16<BF16>(re, im);
    *reinterpret_cast<uint32_t*>(Ct + (size_t)o * 4) = h;
    if (C2t) *reinterpret_cast<uint32_t*>(C2t + (size_t)o * 4) = resid16<BF16>(re, im, h);
  }
}
// one complex output element at element offset o: fp32 pair, or 16-bit pair
// (plus its residual in the second array when it is non-null)
template <bool BF16, bool F32OUT>
__device__ __forceinline__ void store_el(char* Cb, char* C2b, int64_t o, float re, float im) {
  if constexpr (F32OUT) {
    *reinterpret_cast<float2*>(Cb + o * 8) = make_float2(re, im);
  } else {
    const uint32_t h = pack16<BF16>(re, im);
    *reinterpret_cast<uint32_t*>(Cb + o * 4) = h;
    if (C2b) *reinterpret_cast<uint32_t*>(C2b + o * 4) = resid16<BF16>(re, im, h);
  }
}

// 16 bytes of consecutive complex outputs from v (re, im of each, unscaled):
// 4 values as 16-bit pairs in hv (their residuals in lv when res), or 2
// values as fp32 pairs
template <bool BF16, bool F32OUT>
__device__ __forceinline__ void pack_vec16(const uint32_t* v, float scale, bool res, uint4& hv, uint4& lv) {
  if constexpr (F32OUT) {
    hv = make_uint4(__float_as_uint(__uint_as_float(v[0]) * scale), __float_as_uint(__uint_as_float(v[1]) * scale),
                    __float_as_uint(__uint_as_float(v[2]) * scale), __float_as_uint(__uint_as_float(v[3]) * scale));
    lv = hv;
  } else {
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float re = __uint_as_float(v[2 * q]) * scale, im = __uint_as_float(v[2 * q + 1]) * scale;
      h[q] = pack16<BF16>(re, im);
      l[q] = res ? resid16<BF16>(re, im, h[q]) : 0u;
    }
    hv = make_uint4(h[0], h[1], h[2], h[3]);
    lv = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

// the same stored at 32-bit element offset o (16-byte aligned) of Ct, and the
// residuals at o of C2t when it is non-null
template <bool BF16, bool F32OUT>
__device__ __forceinline__ void store_vec16(char* Ct, char* C2t, uint32_t o, const uint32_t* v, float scale) {
  uint4 hv, lv;
  pack_vec16<BF16, F32OUT>(v, scale, !F32OUT && C2t != nullptr, hv, lv);
  *reinterpret_cast<uint4*>(Ct + (size_t)o * (F32OUT ? 8 : 4)) = hv;
  if (!F32OUT && C2t) *reinterpret_cast<uint4*>(C2t + (size_t)o * 4) = lv;
}

// Shared-memory slot (in 16-byte units) of piece q of row r of a warp's
// staged chunk (32 rows x PR pieces, PR = 4 or 8): line (r / 8) * PR + q, bank
// group (r ^ reverse(q)) mod 8.  Rows write their pieces one q at a time
// (8 consecutive rows per phase) and lanes read back L consecutive pieces of
// 8 / L consecutive rows per phase (L = 1 .. PR, powers of two): reversing
// q's bits puts its low bits on the group's high bits, so either phase sees
// 8 distinct bank groups.
template <int PR>
__device__ __forceinline__ int stage_slot(int r, int q) {
  const int rq = PR == 4 ? (((q & 1) << 2) | (q & 2)) : (((q & 1) << 2) | (q & 2) | ((q >> 2) & 1));
  return ((((r >> 3) * PR + q) << 3) | ((r ^ rq) & 7));
}

// 32 consecutive accumulator columns of this warp's TMEM lane quarter
__device__ __forceinline__ void tmem_ld32_h(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 16 consecutive accumulator columns of this warp's TMEM lane quarter
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}


__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Persistent: CTA c walks output tiles c, c + gridDim.x, ... (n tile fastest,
// then m tile, then batch).  The TMEM accumulator is double-buffered (2 x BN
// columns): the MMA thread fills buffer (i & 1) for the CTA's i-th tile while
// the epilogue drains the other; tfull/tempty hand the buffers back and forth.
// Narrow tiles (BN <= 64, one 128-row half, K in one accumulator): a tile has
// at most two 32-column chunks, so the 16 epilogue warps form 4 groups of 4
// (one warp per TMEM lane quarter), group g draining the CTA's tiles g, g + 4,
// ... with 8 accumulator buffers (2 per group): four tiles' epilogues run at
// once instead of one tile's on 4 warps.
// MH: m halves per tile.  MH = 2 gives a CTA 256 rows (two 128-row MMAs per k
// step sharing one B tile, so B is loaded once per 256 rows) and one TMEM
// accumulator of 2 x BN columns instead of two alternating ones.
template <int BN, bool BF16, bool HILO, bool STAGE, bool F32OUT, bool SPLIT, int MH = 1>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmA2,
                   const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmB2,
                   TcGemmParams p) {
  static_assert(MH == 1 || (MH == 2 && !STAGE && !SPLIT), "two m halves: direct stores");
  constexpr int S = stages_for<BN, STAGE, MH>();
  constexpr int TBM = MH * BM;             // rows per tile
  constexpr int kTG = (MH == 1 && !SPLIT && BN <= 64) ? 4 : 1;  // epilogue tile groups
  constexpr int NBUF = MH == 1 ? 2 * kTG : 1;                   // TMEM accumulator buffers
  constexpr uint32_t kTmemCols = (uint32_t)(MH == 1 ? NBUF * BN : 2 * BN);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = sA + S * TBM * BK * 2;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + S * BN * BK * 2);
  uint64_t* empty = full + S;
  // accumulator hand-off barriers: one pair per buffer, and (MH = 2) one per
  // 128-row half of the single buffer
  constexpr int kTBar = NBUF > 2 ? NBUF : 2;
  uint64_t* tfull = empty + S;       // [kTBar] MMA -> epilogue
  uint64_t* tempty = tfull + kTBar;  // [kTBar] epilogue -> MMA
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + kTBar);
  static_assert((2 * S + 2 * kTBar) * 8 + 4 <= 512, "barrier region");
  int64_t* n_rel = reinterpret_cast<int64_t*>(reinterpret_cast<uint8_t*>(full) + 512);  // [BN / 2]
  uint32_t* n32 = reinterpret_cast<uint32_t*>(n_rel + BN / 2);                           // [BN / 2]
  float2* stage_buf = reinterpret_cast<float2*>(n32 + BN / 2);                           // [warps][32][pitch]
  int64_t* row_base = reinterpret_cast<int64_t*>(stage_buf + kEpiWarps * 32 * kStagePitch);  // [warps][32]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k_tiles1 = (int)((2 * p.K + BK - 1) / BK);
  const int k_tiles = HILO ? 3 * k_tiles1 : k_tiles1;
  const int64_t n_n = (2 * p.N + BN - 1) / BN, n_m = (p.M + TBM - 1) / TBM;
  const int64_t n_mu = n_m;
  const int64_t tiles = p.nbt * n_mu * n_n;
  const int64_t unit0 = blockIdx.x;
  const int64_t ustride = gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < kTBar; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kEpiWarps / kTG);  // one arrival per epilogue warp draining the buffer
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int64_t g = 0;  // ring position over all of this CTA's k tiles
      bool stop = false;
      TileWalk<true> w(unit0, ustride, n_n, n_mu);
      for (int64_t t = unit0; t < tiles && !stop; t += ustride, w.next()) {
        const int n_tile = w.n, bt = w.b;
        const int m_tile = w.m;
        for (int kt = 0; kt < k_tiles; ++kt, ++g) {
          const int s = (int)(g % S);
          const uint32_t use = (uint32_t)(g / S);
          if (g >= S && !wait_bounded(&empty[s], (use & 1) ^ 1, p.err)) {
            stop = true;
            break;
          }
          const int pass = HILO ? kt / k_tiles1 : 0;
          const int kx = (kt - pass * k_tiles1) * BK;
          mbar_expect_tx(&full[s], (uint32_t)((TBM + BN) * BK * 2));
#pragma unroll
          for (int h = 0; h < MH; ++h)
            tma_load_3d(pass == 2 ? &tmA2 : &tmA, &full[s], sA + (s * TBM + h * BM) * BK * 2, kx,
                        m_tile * TBM + h * BM, bt);
          tma_load_3d(pass == 1 ? &tmB2 : &tmB, &full[s], sB + s * BN * BK * 2, kx, n_tile * BN, bt);
        }
      }
      // drain: every issued load must have landed before the CTA can exit
      for (int64_t q = (g > S ? g - S : 0); q < g; ++q) {
        const uint64_t t0 = gtimer();
        while (!mbar_try_wait(&full[q % S], (uint32_t)((q / S) & 1)) && gtimer() - t0 < kWaitNs) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = make_idesc(BN, BF16);
      // accumulation units: one per tile, or (SPLIT) one per chunk of k tiles;
      // the two TMEM buffers alternate between consecutive units
      // SPLIT: K accumulated in chunks of p.acc_split k tiles; each chunk's
      // partial sums are added in FP32 registers by the epilogue (round to
      // nearest), so the tensor cores never accumulate more than
      // p.acc_split * BK real products
      const int kch = SPLIT ? p.acc_split : k_tiles;
      int64_t g = 0;
      int64_t gu = 0;
      bool stop = false;
      for (int64_t t = unit0; t < tiles && !stop; t += ustride)
      for (int c0 = 0; c0 < k_tiles && !stop; c0 += kch, ++gu) {
        const int c1 = c0 + kch < k_tiles ? c0 + kch : k_tiles;
        const int b = (int)(gu % NBUF);
        const uint32_t u = (uint32_t)(gu / NBUF);
        if constexpr (MH == 2) {
          // 256-row tiles: the two TMEM halves (columns h * BN, rows h * 128 of
          // the tile) come back separately (tempty[h]).  The tile's half-0 MMAs
          // start once half 0 is drained; its half-1 MMAs wait, over at most
          // the S staged k tiles, until half 1 is drained too, and each stage is
          // released after both halves have used it.
          auto mma_half = [&](int s, int h, bool acc_in) {
            const uint32_t a0 = smem_u32(sA + s * TBM * BK * 2) + h * BM * BK * 2;
            const uint32_t b0 = smem_u32(sB + s * BN * BK * 2);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint32_t acc = (acc_in || kk > 0) ? 1u : 0u;
              asm volatile(
                  "{\n\t.reg .pred p;\n\t"
                  "setp.ne.b32 p, %4, 0;\n\t"
                  "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem + (uint32_t)(h * BN)),
                  "l"(sw128_desc(a0 + kk * 32)), "l"(sw128_desc(b0 + kk * 32)), "r"(idesc), "r"(acc)
                  : "memory");
            }
          };
          auto release = [&](int s) {
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
          };
          if (gu >= 1 && !wait_bounded(&tempty[0], (u & 1) ^ 1, p.err)) {
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          bool h1 = gu == 0;  // half 1 free
          const int64_t g0 = g;
          for (int kt = c0; kt < c1; ++kt, ++g) {
            const int s = (int)(g % S);
            if (!wait_bounded(&full[s], (uint32_t)((g / S) & 1), p.err)) {
              stop = true;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            mma_half(s, 0, kt > c0);
            if (h1) {
              mma_half(s, 1, kt > c0);
              release(s);
              continue;
            }
            if (kt + 1 < c1 && g - g0 + 1 < S) continue;  // defer half 1 while stages remain
            if (!wait_bounded(&tempty[1], (u & 1) ^ 1, p.err)) {
              stop = true;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            h1 = true;
            for (int64_t j = g0; j <= g; ++j) {
              mma_half((int)(j % S), 1, j > g0);
              release((int)(j % S));
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&tfull[0]))
                       : "memory");
          continue;
        }
        if (gu >= NBUF && !wait_bounded(&tempty[b], (u & 1) ^ 1, p.err)) {
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc_addr = tmem + (uint32_t)(b * BN);
        for (int kt = c0; kt < c1; ++kt, ++g) {
          const int s = (int)(g % S);
          if (!wait_bounded(&full[s], (uint32_t)((g / S) & 1), p.err)) {
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_u32(sA + s * TBM * BK * 2);
          const uint32_t b0 = smem_u32(sB + s * BN * BK * 2);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t bd = sw128_desc(b0 + kk * 32);
            const uint32_t acc = (kt > c0 || kk > 0) ? 1u : 0u;
#pragma unroll
            for (int h = 0; h < MH; ++h) {
              const uint64_t ad = sw128_desc(a0 + h * BM * BK * 2 + kk * 32);
              asm volatile(
                  "{\n\t.reg .pred p;\n\t"
                  "setp.ne.b32 p, %4, 0;\n\t"
                  "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc_addr + h * BN),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                  : "memory");
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&empty[s]))
                       : "memory");
        }
        // tfull[b] completes when this unit's MMAs (and all earlier ones) finish
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&tfull[b]))
                     : "memory");
      }
      // before TMEM is freed: wait (bounded) for the last committed unit's MMAs
      if (gu > 0) {
        const int64_t last = gu - 1;
        const int lb = (int)(last % NBUF);
        const uint32_t lu = (uint32_t)(last / NBUF);
        const uint64_t t0 = gtimer();
        while (!mbar_try_wait(&tfull[lb], lu & 1) && gtimer() - t0 < kWaitNs) {
        }
      }
    }
  } else {
    // epilogue warps
    const int et = threadIdx.x - 64;  // 0..32*kEpiWarps-1
    const int quarter = warp & 3;      // TMEM lanes 32*quarter.. (warp w may read lanes 32*(w%4)..)
    const int ew = warp - 2;           // epilogue warp index
    constexpr int kGroups = kEpiWarps / 4;  // warps per lane quarter
    constexpr int kChunks = BN / 32;        // 32-column accumulator loads per tile
    const int cgrp = ew >> 2;               // this warp takes chunks cgrp, cgrp + kGroups, ...
    // Tile-relative output offsets, once per CTA: tile origins are multiples of
    // the (power-of-two) tile extents, and a run offset is linear over disjoint
    // index bits, so offset(origin + i) = offset(origin) + offset(i).
    for (int j = et; j < BN / 2; j += 32 * kEpiWarps) {
      n_rel[j] = run_offset(p.c_n, j);
      n32[j] = (uint32_t)n_rel[j];  // used when p.off32: a tile's offsets fit in 32 bits
    }
    const int64_t m_rel = run_offset(p.c_m, quarter * 32 + lane);
    // rows h * 128 + quarter * 32 + lane of a 256-row tile
    const int64_t m_rel2[2] = {m_rel, MH == 2 ? run_offset(p.c_m, BM + quarter * 32 + lane) : 0};
    // Tile base offsets.  Tile width 256: the output offset of bit `lane` of
    // each tile-origin index, so that a tile's base offset is the sum over its
    // origin's set bits (offsets are linear over disjoint index bits), reduced
    // across the warp.  Otherwise (measured faster at width 128, and SPLIT is
    // at its register limit): the runs walked per tile.
    constexpr bool kBaseByBits = BN == 256 && !SPLIT;
    const int64_t w_bt = kBaseByBits && lane < 31 ? run_offset(p.c_bt, int64_t(1) << lane) : 0;
    const int64_t w_m = kBaseByBits && lane < 31 ? run_offset(p.c_m, int64_t(1) << lane) : 0;
    const int64_t w_n = kBaseByBits && lane < 31 ? run_offset(p.c_n, int64_t(1) << lane) : 0;
    const uint32_t m32 = (uint32_t)m_rel;
    constexpr int ES = F32OUT ? 8 : 4;  // bytes per output element
    // staged 16-byte pieces (STAGE with p.vec_staged): a chunk row holds kPR
    // pieces of kVN outputs; in store i, lane L takes piece q_i(L) of row
    // r_i(L), 2^lgL lanes per row (mr[i]: that row's in-tile offset)
    constexpr int kVN = F32OUT ? 2 : 4, kPR = 16 / kVN, kLgPR = kPR == 4 ? 2 : 3;
    static_assert(32 * kPR * 16 * (F32OUT ? 1 : 2) <= 32 * kStagePitch * 8, "staged pieces fit a warp's stage");
    const bool vst = STAGE && p.vec && p.vec_staged && p.off32;
    const int lgL = vst ? p.vec_lpr_lg : 0;
    uint32_t mr[kPR];
#pragma unroll
    for (int i = 0; i < kPR; ++i)
      mr[i] = STAGE ? __shfl_sync(0xffffffffu, m32, ((i >> (kLgPR - lgL)) << (5 - lgL)) + (lane >> lgL)) : 0u;
    asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory");
    char* const Cb = reinterpret_cast<char*>(p.C);
    char* const C2b = reinterpret_cast<char*>(p.C2);
    // the 16-bit output is stored hi + lo (its consumer splits its product),
    // whether or not this step's own product is split
    const bool res = !F32OUT && C2b != nullptr;
    // staging (STAGE): float2 [32][pitch] (fp32 out), or words [32][pitch] hi then lo
    uint32_t* stg = reinterpret_cast<uint32_t*>(stage_buf + ew * 32 * kStagePitch);
    int64_t* rb = row_base + ew * 32;
    // tile groups (kTG > 1): this warp's group drains the CTA's tiles eg, eg + kTG, ...
    const int eg = kTG > 1 ? (ew >> 2) : 0;
    constexpr int kCStep = kTG > 1 ? 1 : kGroups;  // chunks of a tile taken by this warp: c0, c0 + kCStep, ...
    const int c0 = kTG > 1 ? 0 : cgrp;
    int64_t local = eg;
    int64_t gu = 0;  // SPLIT: accumulation units consumed
    TileWalk<!SPLIT> w(unit0 + eg * ustride, kTG * ustride, n_n, n_mu);
    for (int64_t t = unit0 + eg * ustride; t < tiles; t += kTG * ustride, local += kTG, w.next()) {
      int n_tile, m_unit, bt;
      w.at(t, n_tile, m_unit, bt);
      const int m_tile = m_unit;
      const int b = (int)(local % NBUF);
      const uint32_t u = (uint32_t)(local / NBUF);
      const int64_t nbase = (int64_t)n_tile * BN / 2, mbase = (int64_t)m_tile * TBM;
      int64_t tbase;
      if constexpr (!kBaseByBits) {
        tbase = run_offset(p.c_bt, bt) + run_offset(p.c_m, mbase) + run_offset(p.c_n, nbase);
      } else {
        tbase = (((uint32_t)bt >> lane) & 1u ? w_bt : 0) + (((uint32_t)mbase >> lane) & 1u ? w_m : 0) +
                (((uint32_t)nbase >> lane) & 1u ? w_n : 0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tbase += __shfl_xor_sync(0xffffffffu, tbase, o);
      }
      const int64_t row = tbase + m_rel;
      char* const Ct = Cb + tbase * ES;
      char* const C2t = res ? C2b + tbase * 4 : nullptr;
      // this lane's row of the tile (32-bit offsets: p.off32 keeps every
      // in-tile offset below 2^31, so row + column never wraps)
      char* const Ctm = Ct + (size_t)m32 * ES;
      char* const C2tm = res ? C2t + (size_t)m32 * 4 : nullptr;
      const bool row_ok = mbase + quarter * 32 + lane < p.M;
      // the tile lies wholly inside M x N
      const bool whole = mbase + TBM <= p.M && nbase + BN / 2 <= p.N;
      if constexpr (MH == 2) {
        // one accumulator (unit = tile); rows h * 128 + quarter * 32 + lane of the tile
        const uint32_t uu = (uint32_t)local;
        const bool ok = __all_sync(0xffffffffu, wait_bounded(&tfull[0], uu & 1, p.err));
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int64_t mr = m_rel2[h];
          const int64_t rowh = tbase + mr;
          const uint32_t m32h = (uint32_t)mr;
          char* const Cth = Ct + (size_t)m32h * ES;
          char* const C2th = res ? C2t + (size_t)m32h * 4 : nullptr;
          const bool rowh_ok = mbase + h * BM + quarter * 32 + lane < p.M;
#pragma unroll 1
          for (int c = cgrp; c < kChunks && ok; c += kGroups) {
            uint32_t v[32];
            tmem_ld32_h(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(h * BN + c * 32), v);
            const int j0 = c * 16;
            if (whole && p.off32 && p.vec) {
              constexpr int VN = F32OUT ? 2 : 4;
#pragma unroll
              for (int j = 0; j < 16; j += VN) store_vec16<BF16, F32OUT>(Cth, C2th, n32[j0 + j], v + 2 * j, p.scale);
            } else if (whole && p.off32) {
#pragma unroll
              for (int j = 0; j < 16; j += 4) {
                const uint4 nn = *reinterpret_cast<const uint4*>(n32 + j0 + j);
                const uint32_t o4[4] = {nn.x, nn.y, nn.z, nn.w};
#pragma unroll
                for (int q = 0; q < 4; ++q)
                  store_el32<BF16, F32OUT>(Cth, C2th, o4[q], __uint_as_float(v[2 * (j + q)]) * p.scale,
                                                 __uint_as_float(v[2 * (j + q) + 1]) * p.scale);
              }
            } else if (rowh_ok) {
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                if (nbase + j0 + j >= p.N) break;
                store_el<BF16, F32OUT>(Cb, C2b, rowh + n_rel[j0 + j], __uint_as_float(v[2 * j]) * p.scale,
                                             __uint_as_float(v[2 * j + 1]) * p.scale);
              }
            }
          }
          // hand this half's TMEM columns back: the next tile's MMAs into them
          // may start while the other half is still being read
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[h]);
        }
        continue;
      }
      if constexpr (SPLIT) {
        // sum the tile's K chunks in FP32 registers, then store once
        constexpr int kMaxCh = (kChunks + kGroups - 1) / kGroups;
        float acc[kMaxCh][32];
#pragma unroll
        for (int ci = 0; ci < kMaxCh; ++ci)
#pragma unroll
          for (int j = 0; j < 32; ++j) acc[ci][j] = 0.f;
        bool ok_all = true;
        for (int c0 = 0; c0 < k_tiles; c0 += p.acc_split, ++gu) {
          const int b = (int)(gu & 1);
          const uint32_t u = (uint32_t)(gu >> 1);
          const bool ok = __all_sync(0xffffffffu, wait_bounded(&tfull[b], u & 1, p.err));
          ok_all = ok_all && ok;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          if (ok) {
#pragma unroll
            for (int ci = 0; ci < kMaxCh; ++ci) {
              const int c = cgrp + ci * kGroups;
              if (c < kChunks) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  uint32_t v[16];
                  tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * BN + c * 32 + h * 16), v);
#pragma unroll
                  for (int j = 0; j < 16; ++j) acc[ci][h * 16 + j] += __uint_as_float(v[j]);
                }
              }
            }
          }
          // hand the accumulator buffer back to the MMA thread
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[b]);
        }
        if (ok_all) {
#pragma unroll
          for (int ci = 0; ci < kMaxCh; ++ci) {
            const int c = cgrp + ci * kGroups;
            if (c >= kChunks) continue;
            const int j0 = c * 16;
            if (whole && p.off32) {
#pragma unroll
              for (int j = 0; j < 16; j += 4) {
                const uint4 nn = *reinterpret_cast<const uint4*>(n32 + j0 + j);
                const uint32_t o4[4] = {nn.x, nn.y, nn.z, nn.w};
#pragma unroll
                for (int q = 0; q < 4; ++q)
                  store_el32<BF16, F32OUT>(Ct, C2t, m32 + o4[q], acc[ci][2 * (j + q)] * p.scale,
                                                 acc[ci][2 * (j + q) + 1] * p.scale);
              }
            } else if (whole) {
#pragma unroll
              for (int j = 0; j < 16; ++j)
                store_el<BF16, F32OUT>(Cb, C2b, row + n_rel[j0 + j], acc[ci][2 * j] * p.scale,
                                             acc[ci][2 * j + 1] * p.scale);
            } else if (row_ok) {
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                if (nbase + j0 + j >= p.N) break;
                store_el<BF16, F32OUT>(Cb, C2b, row + n_rel[j0 + j], acc[ci][2 * j] * p.scale,
                                             acc[ci][2 * j + 1] * p.scale);
              }
            }
          }
        }
        continue;
      }
      // every epilogue thread runs every iteration; after a timed-out wait
      // (warp-uniform) the tile's reads and stores are skipped
      const bool ok = __all_sync(0xffffffffu, wait_bounded(&tfull[b], u & 1, p.err));
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (STAGE) {
        rb[lane] = row;
        __syncwarp();
      }
#pragma unroll 1
      for (int c = c0; c < kChunks && ok; c += kCStep) {
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * BN + c * 32);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
            "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
            "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
              "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
              "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
              "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int j0 = c * 16;  // first complex column of the chunk
        if (STAGE && vst && whole) {
          // 16-byte pieces staged through shared memory: each lane writes its
          // row's pieces, then 2^lgL lanes store consecutive pieces of one
          // row together, so that a store covers whole sectors
          uint4* sv = reinterpret_cast<uint4*>(stg);
#pragma unroll
          for (int q = 0; q < kPR; ++q) {
            uint4 hv, lv;
            pack_vec16<BF16, F32OUT>(v + 2 * kVN * q, p.scale, res, hv, lv);
            const int sl = stage_slot<kPR>(lane, q);
            sv[sl] = hv;
            if (res) sv[32 * kPR + sl] = lv;
          }
          __syncwarp();
#pragma unroll
          for (int i = 0; i < kPR; ++i) {
            const int q = ((i & ((kPR >> lgL) - 1)) << lgL) + (lane & ((1 << lgL) - 1));
            const int r = ((i >> (kLgPR - lgL)) << (5 - lgL)) + (lane >> lgL);
            const int sl = stage_slot<kPR>(r, q);
            const uint32_t o = mr[i] + n32[j0 + q * kVN];
            *reinterpret_cast<uint4*>(Ct + (size_t)o * ES) = sv[sl];
            if (res) *reinterpret_cast<uint4*>(C2t + (size_t)o * 4) = sv[32 * kPR + sl];
          }
          __syncwarp();
        } else if (STAGE) {
          // transpose through shared memory, already converted: lanes then run along n
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float re = __uint_as_float(v[2 * j]) * p.scale, im = __uint_as_float(v[2 * j + 1]) * p.scale;
            if constexpr (F32OUT) {
              reinterpret_cast<float2*>(stg)[lane * kStagePitch + j] = make_float2(re, im);
            } else {
              const uint32_t h = pack16<BF16>(re, im);
              stg[lane * kStagePitch + j] = h;
              if (res) stg[32 * kStagePitch + lane * kStagePitch + j] = resid16<BF16>(re, im, h);
            }
          }
          __syncwarp();
          const int jj = lane & 15;
          const int64_t col = n_rel[j0 + jj];
          const bool col_ok = nbase + j0 + jj < p.N;
#pragma unroll 4
          for (int it = 0; it < 16; ++it) {
            const int r = 2 * it + (lane >> 4);
            if (whole || (col_ok && mbase + quarter * 32 + r < p.M)) {
              const int64_t o = rb[r] + col;
              if constexpr (F32OUT) {
                *reinterpret_cast<float2*>(Cb + o * 8) = reinterpret_cast<const float2*>(stg)[r * kStagePitch + jj];
              } else {
                *reinterpret_cast<uint32_t*>(Cb + o * 4) = stg[r * kStagePitch + jj];
                if (res) *reinterpret_cast<uint32_t*>(C2b + o * 4) = stg[32 * kStagePitch + r * kStagePitch + jj];
              }
            }
          }
          __syncwarp();
        } else if (whole && p.off32 && p.vec) {
          // runs of VN outputs consecutive along n: one 16-byte store each
          constexpr int VN = F32OUT ? 2 : 4;
#pragma unroll
          for (int j = 0; j < 16; j += VN) store_vec16<BF16, F32OUT>(Ctm, C2tm, n32[j0 + j], v + 2 * j, p.scale);
        } else if (whole && p.off32) {
#pragma unroll
          for (int j = 0; j < 16; j += 4) {
            const uint4 nn = *reinterpret_cast<const uint4*>(n32 + j0 + j);
            const uint32_t o4[4] = {nn.x, nn.y, nn.z, nn.w};
#pragma unroll
            for (int q = 0; q < 4; ++q)
              store_el32<BF16, F32OUT>(Ctm, C2tm, o4[q], __uint_as_float(v[2 * (j + q)]) * p.scale,
                                             __uint_as_float(v[2 * (j + q) + 1]) * p.scale);
          }
        } else if (whole) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            store_el<BF16, F32OUT>(Cb, C2b, row + n_rel[j0 + j], __uint_as_float(v[2 * j]) * p.scale,
                                         __uint_as_float(v[2 * j + 1]) * p.scale);
        } else if (row_ok) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            if (nbase + j0 + j >= p.N) break;
            store_el<BF16, F32OUT>(Cb, C2b, row + n_rel[j0 + j], __uint_as_float(v[2 * j]) * p.scale,
                                         __uint_as_float(v[2 * j + 1]) * p.scale);
          }
        }
      }
      // hand the accumulator buffer back to the MMA thread
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
  }
}

template <int BN, bool BF16, bool HILO, bool STAGE, bool F32OUT, bool SPLIT = false, int MH = 1>
void launch_tc6(const CUtensorMap& ma, const CUtensorMap& ma2, const CUtensorMap& mb, const CUtensorMap& mb2,
                const TcGemmParams& p, cudaStream_t s) {
  const size_t sm = smem_bytes<BN, STAGE, MH>();
  auto kern = tc_gemm_kernel<BN, BF16, HILO, STAGE, F32OUT, SPLIT, MH>;
  // the shared-memory opt-in is a per-device property of the function
  static std::atomic<uint64_t> attr_set{0};
  int dev = 0;
  TN_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = uint64_t(1) << (dev & 63);
  if (!(attr_set.load() & bit)) {
    TN_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr_set.fetch_or(bit);
  }
  const int64_t n_m = (p.M + MH * BM - 1) / (MH * BM), n_n = (2 * p.N + BN - 1) / BN;
  const unsigned grid = (unsigned)std::min<int64_t>(n_m * n_n * p.nbt, 152);
  kern<<<grid, kThreads, sm, s>>>(ma, ma2, mb, mb2, p);
}
template <int BN, bool BF16, bool HILO, bool STAGE>
void launch_tc4(const CUtensorMap& ma, const CUtensorMap& ma2, const CUtensorMap& mb, const CUtensorMap& mb2,
                const TcGemmParams& p, cudaStream_t s) {
  if (p.out_kind == 2)
    launch_tc6<BN, BF16, HILO, STAGE, true>(ma, ma2, mb, mb2, p, s);
  else
    launch_tc6<BN, BF16, HILO, STAGE, false>(ma, ma2, mb, mb2, p, s);
}
template <int BN, bool BF16, bool HILO>
void launch_tc3(const CUtensorMap& ma, const CUtensorMap& ma2, const CUtensorMap& mb, const CUtensorMap& mb2,
                const TcGemmParams& p, cudaStream_t s) {
  // 256-row tiles (two m halves sharing each B tile): direct stores
  if constexpr (BN == 256) {
    if (p.m_halves == 2) {
      if (p.out_kind == 2)
        launch_tc6<BN, BF16, HILO, false, true, false, 2>(ma, ma2, mb, mb2, p, s);
      else
        launch_tc6<BN, BF16, HILO, false, false, false, 2>(ma, ma2, mb, mb2, p, s);
      return;
    }
  }
  // K accumulated in chunks: direct stores along m (no staging)
  if (p.acc_split) {
    if (p.out_kind == 2)
      launch_tc6<BN, BF16, HILO, false, true, true>(ma, ma2, mb, mb2, p, s);
    else
      launch_tc6<BN, BF16, HILO, false, false, true>(ma, ma2, mb, mb2, p, s);
    return;
  }
  if (p.stage_n)
    launch_tc4<BN, BF16, HILO, true>(ma, ma2, mb, mb2, p, s);
  else
    launch_tc4<BN, BF16, HILO, false>(ma, ma2, mb, mb2, p, s);
}

}  // namespace

// Launch the persistent tensor-core kernel of tile width BN for p (maps built
// by the host side); the variant follows the precision, the split, the
// epilogue form and the output kind.
template <int BN>
void launch_tc_tiles(const CUtensorMap& ma, const CUtensorMap& ma2, const CUtensorMap& mb, const CUtensorMap& mb2,
                     const TcGemmParams& p, bool bf16, bool hilo, cudaStream_t s) {
  if (bf16) {
    if (hilo)
      launch_tc3<BN, true, true>(ma, ma2, mb, mb2, p, s);
    else
      launch_tc3<BN, true, false>(ma, ma2, mb, mb2, p, s);
  } else {
    if (hilo)
      launch_tc3<BN, false, true>(ma, ma2, mb, mb2, p, s);
    else
      launch_tc3<BN, false, false>(ma, ma2, mb, mb2, p, s);
  }
}

}  // namespace tn
