// Tensor-core GEMM (tcgen05 + TMA + TMEM) for the reduced-precision complex
// path.
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
// Kernel: one CTA per 128 x BN output tile (real columns), 6 warps:
//   warp 0      TMA producer: 3-D tiled loads of A' (box 64 x 128) and B'
//               (box 64 x BN), 128-byte swizzle, into a 4-stage ring;
//   warp 1      allocates BN TMEM columns, one thread issues tcgen05.mma
//               (kind::f16, M = 128, N = BN, K = 16, FP32 accumulate in TMEM)
//               and tcgen05.commit releases ring stages / signals the end;
//   warps 2..5  epilogue: tcgen05.ld rows of the accumulator (warp w reads
//               TMEM lanes 32*(w%4)..+31), scale by 2^shift, convert, store.
// Every mbarrier wait is bounded by the global timer (2 s); on timeout the
// kernel raises the device error flag and every role stops; the producer and
// the MMA thread drain their own in-flight work (bounded) before TMEM is freed.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstring>
#include <string>

#include "tn_internal.h"

namespace tn {
namespace {

constexpr int BM = 128;
constexpr int BK = 64;  // real k per stage: one 128-byte swizzle row of 16-bit values
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
// true when the phase with `parity` has completed; false on abort or timeout
__device__ bool wait_bounded(uint64_t* bar, uint32_t parity, int* err) {
  const uint64_t t0 = gtimer();
  while (!mbar_try_wait(bar, parity)) {
    if (*(volatile int*)err) return false;
    if (gtimer() - t0 > kWaitNs) {
      atomicExch(err, 1);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void tma_load_3d(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y,
                                            int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}
// the same load delivered to every CTA of the cluster in `mask` (same smem
// offset, each CTA's own mbarrier at the same offset)
__device__ __forceinline__ void tma_load_3d_mc(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y, int z,
                                               uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster"
      " [%0], [%1, {%3, %4, %5}], [%2], %6;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z), "h"(mask)
      : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
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
constexpr int kEpiWarps = 8;  // two warps per TMEM lane quarter, each taking half the columns
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr size_t kStageBytes = kEpiWarps * 32 * kStagePitch * 8 + kEpiWarps * 32 * 8;

// ring depth: as many stages as fit in 227 KB of shared memory next to the
// barriers, the column-offset table and (STAGE) the epilogue staging, at most 8
template <int BN, bool STAGE = false>
__host__ __device__ constexpr int stages_for() {
  constexpr long budget = 232448 - 1024 - 256 - (long)BN / 2 * 8 - (STAGE ? (long)kStageBytes : 0L) - 512;
  constexpr long per = (long)(BM + BN) * BK * 2;
  return budget / per > 8 ? 8 : (int)(budget / per);
}
template <int BN, bool STAGE>
__host__ __device__ constexpr size_t smem_bytes() {
  return 1024 + (size_t)stages_for<BN, STAGE>() * (BM + BN) * BK * 2 + 256 + (size_t)BN / 2 * 8 +
         (STAGE ? kStageBytes : 0);
}

// one complex output element, converted to the output kind (hi + lo when split)
__device__ __forceinline__ void store_c(const TcGemmParams& p, int64_t o, float re, float im) {
  if (p.out_kind == 2) {
    reinterpret_cast<float2*>(p.C)[o] = make_float2(re, im);
  } else if (p.out_kind == 1) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
    reinterpret_cast<__nv_bfloat162*>(p.C)[o] = h;
    if (p.out_hilo) {
      const float2 hf = __bfloat1622float2(h);
      reinterpret_cast<__nv_bfloat162*>(p.C2)[o] = __floats2bfloat162_rn(re - hf.x, im - hf.y);
    }
  } else {
    const __half2 h = __floats2half2_rn(re, im);
    reinterpret_cast<__half2*>(p.C)[o] = h;
    if (p.out_hilo) {
      const float2 hf = __half22float2(h);
      reinterpret_cast<__half2*>(p.C2)[o] = __floats2half2_rn(re - hf.x, im - hf.y);
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Persistent: CTA c walks output tiles c, c + gridDim.x, ... (n tile fastest,
// then m tile, then batch).  The TMEM accumulator is double-buffered (2 x BN
// columns): the MMA thread fills buffer (i & 1) for the CTA's i-th tile while
// the epilogue drains the other; tfull/tempty hand the buffers back and forth.
// C2: a cluster of two CTAs takes two adjacent m tiles of one n tile; each CTA
// loads its own A tile and one half of the shared B tile, multicast to both,
// so every SM reads a third less from L2 per k step.  A stage is refilled only
// after both CTAs' MMAs released it (their commits arrive on both CTAs'
// `empty` barriers).
template <int BN, bool BF16, bool HILO, bool STAGE, bool C2>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmA2,
                   const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmB2,
                   TcGemmParams p) {
  constexpr int S = stages_for<BN, STAGE>();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = sA + S * BM * BK * 2;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + S * BN * BK * 2);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;   // [2] MMA -> epilogue
  uint64_t* tempty = tfull + 2;  // [2] epilogue -> MMA
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  int64_t* n_off = reinterpret_cast<int64_t*>(reinterpret_cast<uint8_t*>(full) + 256);  // [BN / 2]
  float2* stage_buf = reinterpret_cast<float2*>(n_off + BN / 2);                         // [warps][32][pitch]
  int64_t* row_base = reinterpret_cast<int64_t*>(stage_buf + kEpiWarps * 32 * kStagePitch);  // [warps][32]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k_tiles1 = (int)((2 * p.K + BK - 1) / BK);
  const int k_tiles = HILO ? 3 * k_tiles1 : k_tiles1;
  const int64_t n_n = (2 * p.N + BN - 1) / BN, n_m = (p.M + BM - 1) / BM;
  // work units: single tiles, or (C2) pairs of m tiles sharing an n tile
  const int64_t n_mu = C2 ? (n_m + 1) / 2 : n_m;
  const int64_t tiles = p.nbt * n_mu * n_n;
  const int rank = C2 ? (int)cluster_rank() : 0;
  const int64_t unit0 = C2 ? blockIdx.x / 2 : blockIdx.x;
  const int64_t ustride = C2 ? gridDim.x / 2 : gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], C2 ? 2 : 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kEpiWarps);  // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)(2 * BN))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (C2) cluster_sync_all();  // the peer's barriers are initialised before any multicast
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int64_t g = 0;  // ring position over all of this CTA's k tiles
      bool stop = false;
      for (int64_t t = unit0; t < tiles && !stop; t += ustride) {
        const int n_tile = (int)(t % n_n), bt = (int)(t / (n_n * n_mu));
        const int m_tile = (int)((t / n_n) % n_mu) * (C2 ? 2 : 1) + rank;
        for (int kt = 0; kt < k_tiles; ++kt, ++g) {
          const int s = (int)(g % S);
          const uint32_t use = (uint32_t)(g / S);
          if (g >= S && !wait_bounded(&empty[s], (use & 1) ^ 1, p.err)) {
            stop = true;
            break;
          }
          const int pass = HILO ? kt / k_tiles1 : 0;
          const int kx = (kt - pass * k_tiles1) * BK;
          mbar_expect_tx(&full[s], (uint32_t)((BM + BN) * BK * 2));
          tma_load_3d(pass == 2 ? &tmA2 : &tmA, &full[s], sA + s * BM * BK * 2, kx, m_tile * BM, bt);
          if (C2)
            tma_load_3d_mc(pass == 1 ? &tmB2 : &tmB, &full[s], sB + s * BN * BK * 2 + rank * (BN / 2) * BK * 2, kx,
                           n_tile * BN + rank * (BN / 2), bt, (uint16_t)0x3);
          else
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
      int64_t g = 0;
      int64_t local = 0;
      bool stop = false;
      for (int64_t t = unit0; t < tiles && !stop; t += ustride, ++local) {
        const int b = (int)(local & 1);
        const uint32_t u = (uint32_t)(local >> 1);
        if (local >= 2 && !wait_bounded(&tempty[b], (u & 1) ^ 1, p.err)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc_addr = tmem + (uint32_t)(b * BN);
        for (int kt = 0; kt < k_tiles; ++kt, ++g) {
          const int s = (int)(g % S);
          if (!wait_bounded(&full[s], (uint32_t)((g / S) & 1), p.err)) {
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_u32(sA + s * BM * BK * 2);
          const uint32_t b0 = smem_u32(sB + s * BN * BK * 2);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t ad = sw128_desc(a0 + kk * 32);
            const uint64_t bd = sw128_desc(b0 + kk * 32);
            const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc_addr),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
          }
          if (C2)
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                    smem_u32(&empty[s])),
                "h"((uint16_t)0x3)
                : "memory");
          else
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
        }
        // tfull[b] completes when this tile's MMAs (and all earlier ones) finish
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&tfull[b]))
                     : "memory");
      }
      // before TMEM is freed: wait (bounded) for the last committed tile's MMAs
      if (local > 0) {
        const int64_t last = local - 1;
        const uint64_t t0 = gtimer();
        while (!mbar_try_wait(&tfull[last & 1], (uint32_t)((last >> 1) & 1)) && gtimer() - t0 < kWaitNs) {
        }
      }
    }
  } else {
    // epilogue warps 2..5
    const int et = threadIdx.x - 64;  // 0..32*kEpiWarps-1
    const int quarter = warp & 3;      // TMEM lanes 32*quarter.. (warp w may read lanes 32*(w%4)..)
    const int ew = warp - 2;           // epilogue warp index
    const int col_half = ew / 4;       // columns [col_half*BN/2, (col_half+1)*BN/2)
    int64_t local = 0;
    for (int64_t t = unit0; t < tiles; t += ustride, ++local) {
      const int n_tile = (int)(t % n_n), bt = (int)(t / (n_n * n_mu));
      const int m_tile = (int)((t / n_n) % n_mu) * (C2 ? 2 : 1) + rank;
      const int b = (int)(local & 1);
      const uint32_t u = (uint32_t)(local >> 1);
      const int64_t nbase = (int64_t)n_tile * BN / 2;
      asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory");  // previous table no longer read
      for (int j = et; j < BN / 2; j += 32 * kEpiWarps) n_off[j] = nbase + j < p.N ? run_offset(p.c_n, nbase + j) : 0;
      asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory");
      // every epilogue thread runs every iteration (the named barriers above need all
      // of them); after a timed-out wait (warp-uniform) the tile's reads and stores are skipped
      const bool ok = __all_sync(0xffffffffu, wait_bounded(&tfull[b], u & 1, p.err));
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int64_t m = (int64_t)m_tile * BM + quarter * 32 + lane;
      const int64_t base = m < p.M ? run_offset(p.c_bt, bt) + run_offset(p.c_m, m) : 0;
      float2* stg = stage_buf + ew * 32 * kStagePitch;
      int64_t* rb = row_base + ew * 32;
      if (STAGE) {
        rb[lane] = base;
        __syncwarp();
      }
      // column range of this warp (32-column loads): halves for BN >= 64, else all in half 0
      constexpr int kHalf = BN >= 64 ? BN / 2 : BN;
      const int c_beg = BN >= 64 ? col_half * kHalf : (col_half ? BN : 0);
      const int c_end = BN >= 64 ? c_beg + kHalf : BN;
#pragma unroll 1
      for (int c0 = c_beg; c0 < c_end && ok; c0 += 32) {
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * BN + c0);
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
        const int j0 = c0 / 2;
        if (STAGE) {
          // transpose through shared memory: lanes then run along n (16 per row)
#pragma unroll
          for (int j = 0; j < 16; ++j)
            stg[lane * kStagePitch + j] =
                make_float2(__uint_as_float(v[2 * j]) * p.scale, __uint_as_float(v[2 * j + 1]) * p.scale);
          __syncwarp();
#pragma unroll 4
          for (int it = 0; it < 16; ++it) {
            const int e = it * 32 + lane;
            const int r = e >> 4, jj = e & 15;
            const int64_t mr = (int64_t)m_tile * BM + quarter * 32 + r;
            if (mr < p.M && nbase + j0 + jj < p.N) {
              const float2 val = stg[r * kStagePitch + jj];
              store_c(p, rb[r] + n_off[j0 + jj], val.x, val.y);
            }
          }
          __syncwarp();
        } else if (m < p.M) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            if (nbase + j0 + j >= p.N) break;
            store_c(p, base + n_off[j0 + j], __uint_as_float(v[2 * j]) * p.scale,
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
  if (C2) cluster_sync_all();  // no CTA leaves while its peer may still multicast into it
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * BN))
                 : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* ptr = nullptr;
    TN_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q));
    TN_CHECK(q == cudaDriverEntryPointSuccess && ptr, TN_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  return fn;
}

// 3-D map over a 16-bit real matrix: dims {inner, rows, batch}, strides in bytes
void make_map(CUtensorMap* map, const void* base, bool bf16, uint64_t inner, uint64_t rows, uint64_t batch,
              uint64_t row_bytes, uint64_t batch_bytes, uint32_t box_rows) {
  TN_CHECK((reinterpret_cast<uintptr_t>(base) & 15) == 0, TN_ERR_UNSUPPORTED, "TMA base not 16-byte aligned");
  TN_CHECK(row_bytes % 16 == 0 && batch_bytes % 16 == 0, TN_ERR_UNSUPPORTED, "TMA stride not 16-byte aligned");
  cuuint64_t dims[3] = {inner, rows, batch};
  cuuint64_t strides[2] = {row_bytes, batch_bytes};
  cuuint32_t box[3] = {(cuuint32_t)BK, box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = encode_fn()(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3,
                           const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  TN_CHECK(r == CUDA_SUCCESS, TN_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
}

template <int BN, bool BF16, bool HILO, bool STAGE, bool C2>
void launch_bn5(const CUtensorMap& ma, const CUtensorMap& ma2, const CUtensorMap& mb, const CUtensorMap& mb2,
                const TcGemmParams& p, cudaStream_t s) {
  const size_t sm = smem_bytes<BN, STAGE>();
  auto kern = tc_gemm_kernel<BN, BF16, HILO, STAGE, C2>;
  static bool attr = false;
  if (!attr) {
    TN_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr = true;
  }
  const int64_t n_m = (p.M + BM - 1) / BM, n_n = (2 * p.N + BN - 1) / BN;
  if (!C2) {
    const unsigned grid = (unsigned)std::min<int64_t>(n_m * n_n * p.nbt, 152);
    kern<<<grid, kThreads, sm, s>>>(ma, ma2, mb, mb2, p);
    return;
  }
  const int64_t pairs = ((n_m + 1) / 2) * n_n * p.nbt;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(2 * std::min<int64_t>(pairs, 76)));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  TN_CUDA(cudaLaunchKernelEx(&cfg, kern, ma, ma2, mb, mb2, p));
}
template <int BN, bool BF16, bool HILO, bool STAGE>
void launch_bn4(const CUtensorMap& ma, const CUtensorMap& ma2, const CUtensorMap& mb, const CUtensorMap& mb2,
                const TcGemmParams& p, cudaStream_t s) {
  if (p.cluster2)
    launch_bn5<BN, BF16, HILO, STAGE, true>(ma, ma2, mb, mb2, p, s);
  else
    launch_bn5<BN, BF16, HILO, STAGE, false>(ma, ma2, mb, mb2, p, s);
}
template <int BN, bool BF16, bool HILO>
void launch_bn(const CUtensorMap& ma, const CUtensorMap& ma2, const CUtensorMap& mb, const CUtensorMap& mb2,
               const TcGemmParams& p, cudaStream_t s) {
  if (p.stage_n)
    launch_bn4<BN, BF16, HILO, true>(ma, ma2, mb, mb2, p, s);
  else
    launch_bn4<BN, BF16, HILO, false>(ma, ma2, mb, mb2, p, s);
}

}  // namespace

bool tc_gemm_supported(int64_t nbt, int64_t M, int64_t N, int64_t K, int64_t sa_bt, int64_t sa_m, int64_t sa_k) {
  return sa_k == 1 && K >= 4 && M >= 1 && N >= 1 && nbt >= 1 && nbt <= 65535 && sa_m % 4 == 0 &&
         (nbt == 1 || sa_bt % 4 == 0) && (M + BM - 1) / BM <= 65535;
}

int tc_gemm_bn(int64_t N) {
  const int64_t n2 = 2 * N;
  return n2 >= 256 ? 256 : n2 >= 128 ? 128 : n2 >= 64 ? 64 : 32;
}

// A: complex 16-bit [bt][M][K] with k contiguous (strides sa_bt, sa_m in complex
// elements); Bx: expanded real [bt][2N][pitch] (pitch = round_up(2K, 64)).
void launch_gemm_tc(const void* A, const void* A_lo, int64_t sa_bt, int64_t sa_m, const void* Bx,
                    const void* Bx_lo, const TcGemmParams& p_in, bool bf16, cudaStream_t s) {
  TcGemmParams p = p_in;
  if (p.nbt <= 0 || p.M <= 0 || p.N <= 0) return;
  TN_CHECK(tc_gemm_supported(p.nbt, p.M, p.N, p.K, sa_bt, sa_m, 1), TN_ERR_UNSUPPORTED,
           "shape not supported by the tensor-core GEMM");
  const bool hilo = A_lo != nullptr && Bx_lo != nullptr;
  const int bn = p.bn;
  {
    // stage the epilogue when n is the output's more contiguous index
    const int64_t big = int64_t(1) << 62;
    const int64_t sn = p.c_n.n > 0 ? p.c_n.st[0] : big, sm = p.c_m.n > 0 ? p.c_m.st[0] : big;
    // only for write-heavy tiles (up to four k tiles); deeper tiles hide the per-row stores
    p.stage_n = (sn < sm && 2 * p.K <= 4 * BK) ? 1 : 0;
  }
  const uint64_t pitch = (uint64_t)((2 * p.K + BK - 1) / BK * BK);
  CUtensorMap ma, ma2, mb, mb2;
  const uint64_t a_row = (uint64_t)sa_m * 4, a_bt = p.nbt > 1 ? (uint64_t)sa_bt * 4 : a_row * (uint64_t)p.M;
  make_map(&ma, A, bf16, (uint64_t)(2 * p.K), (uint64_t)p.M, (uint64_t)p.nbt, a_row, (a_bt + 15) / 16 * 16, BM);
  const uint32_t b_box = (uint32_t)(p.cluster2 ? bn / 2 : bn);
  make_map(&mb, Bx, bf16, pitch, (uint64_t)(2 * p.N), (uint64_t)p.nbt, pitch * 2, pitch * 2 * 2 * p.N, b_box);
  if (hilo) {
    make_map(&ma2, A_lo, bf16, (uint64_t)(2 * p.K), (uint64_t)p.M, (uint64_t)p.nbt, a_row, (a_bt + 15) / 16 * 16,
             BM);
    make_map(&mb2, Bx_lo, bf16, pitch, (uint64_t)(2 * p.N), (uint64_t)p.nbt, pitch * 2, pitch * 2 * 2 * p.N,
             b_box);
  } else {
    ma2 = ma;
    mb2 = mb;
  }
#define TN_TC_CASE(BNV)                                                       \
  case BNV:                                                                   \
    if (bf16) {                                                               \
      if (hilo)                                                               \
        launch_bn<BNV, true, true>(ma, ma2, mb, mb2, p, s);                   \
      else                                                                    \
        launch_bn<BNV, true, false>(ma, ma2, mb, mb2, p, s);                  \
    } else {                                                                  \
      if (hilo)                                                               \
        launch_bn<BNV, false, true>(ma, ma2, mb, mb2, p, s);                  \
      else                                                                    \
        launch_bn<BNV, false, false>(ma, ma2, mb, mb2, p, s);                 \
    }                                                                         \
    break;
  switch (bn) {
    TN_TC_CASE(32)
    TN_TC_CASE(64)
    TN_TC_CASE(128)
    TN_TC_CASE(256)
    default:
      fail(TN_ERR_UNSUPPORTED, "bad tensor-core tile");
  }
#undef TN_TC_CASE
}

// ------------------------------------------------------------ B expansion
namespace {
template <class T>
__device__ __forceinline__ T neg16(T x);
template <>
__device__ __forceinline__ __half neg16(__half x) {
  return __hneg(x);
}
template <>
__device__ __forceinline__ __nv_bfloat16 neg16(__nv_bfloat16 x) {
  return __hneg(x);
}

// Bx[bt][2n+0][2k..2k+1] = (Re B, -Im B)[k][n], Bx[bt][2n+1][2k..2k+1] = (Im B, Re B)[k][n];
// columns past 2K up to the pitch are zero.  With Bx_lo, every entry's
// rounding residual (exact value - 16-bit value) goes to Bx_lo.
template <class I>
__device__ __forceinline__ I run_off_i(const Runs& R, I i) {
  I o = 0;
  for (int r = 0; r < R.n; ++r) {
    o += (i & ((I(1) << R.lg[r]) - 1)) * (I)R.st[r];
    i >>= R.lg[r];
  }
  return o;
}

// I: index type (32-bit when B and Bx have fewer than 2^31 elements)
template <class T2, class T, class TIN, class I>
__global__ void expand_b_kernel(const TIN* __restrict__ B, Runs b_bt, Runs b_k, Runs b_n, int64_t nbt, int64_t N,
                                int64_t K, int64_t half_pitch, T2* __restrict__ Bx, T2* __restrict__ Bx_lo,
                                float bscale) {
  const I total = (I)(nbt * N * half_pitch);
  const I hp = (I)half_pitch, NN = (I)N, KK = (I)K;
  for (I x = blockIdx.x * (I)blockDim.x + threadIdx.x; x < total; x += (I)gridDim.x * blockDim.x) {
    const I k = x % hp;
    const I t = x / hp;
    const I n = t % NN, bt = t / NN;
    float re = 0.f, im = 0.f;
    if (k < KK) {
      const TIN v = B[run_off_i<I>(b_bt, bt) + run_off_i<I>(b_k, k) + run_off_i<I>(b_n, n)];
      re = (float)v.x * bscale;  // power of two: exact unless out of range
      im = (float)v.y * bscale;
    }
    const T hre = T(re), him = T(im);
    T2 r0, r1;
    r0.x = hre;
    r0.y = neg16<T>(him);
    r1.x = him;
    r1.y = hre;
    const int64_t row0 = ((int64_t)bt * 2 * N + 2 * (int64_t)n) * half_pitch;
    Bx[row0 + k] = r0;
    Bx[row0 + half_pitch + k] = r1;
    if (Bx_lo) {
      const T lre = T(re - (float)hre), lim = T(im - (float)him);
      T2 l0, l1;
      l0.x = lre;
      l0.y = neg16<T>(lim);
      l1.x = lim;
      l1.y = lre;
      Bx_lo[row0 + k] = l0;
      Bx_lo[row0 + half_pitch + k] = l1;
    }
  }
}

template <class I>
void expand_typed(const void* B, const Runs& b_bt, const Runs& b_k, const Runs& b_n, int64_t nbt, int64_t N,
                  int64_t K, int64_t half_pitch, bool bf16, void* Bx, cudaStream_t s, bool in_c64, void* Bx_lo,
                  float bscale, unsigned blocks) {
  if (bf16) {
    if (in_c64)
      expand_b_kernel<__nv_bfloat162, __nv_bfloat16, float2, I><<<blocks, 256, 0, s>>>(
          (const float2*)B, b_bt, b_k, b_n, nbt, N, K, half_pitch, (__nv_bfloat162*)Bx, (__nv_bfloat162*)Bx_lo,
          bscale);
    else
      expand_b_kernel<__nv_bfloat162, __nv_bfloat16, __nv_bfloat162, I><<<blocks, 256, 0, s>>>(
          (const __nv_bfloat162*)B, b_bt, b_k, b_n, nbt, N, K, half_pitch, (__nv_bfloat162*)Bx,
          (__nv_bfloat162*)Bx_lo, bscale);
  } else {
    if (in_c64)
      expand_b_kernel<__half2, __half, float2, I><<<blocks, 256, 0, s>>>(
          (const float2*)B, b_bt, b_k, b_n, nbt, N, K, half_pitch, (__half2*)Bx, (__half2*)Bx_lo, bscale);
    else
      expand_b_kernel<__half2, __half, __half2, I><<<blocks, 256, 0, s>>>(
          (const __half2*)B, b_bt, b_k, b_n, nbt, N, K, half_pitch, (__half2*)Bx, (__half2*)Bx_lo, bscale);
  }
}
}  // namespace

void launch_expand_b(const void* B, const Runs& b_bt, const Runs& b_k, const Runs& b_n, int64_t nbt, int64_t N,
                     int64_t K, bool bf16, void* Bx, cudaStream_t s, bool in_c64, void* Bx_lo, float bscale) {
  const int64_t half_pitch = (2 * K + BK - 1) / BK * BK / 2;
  const int64_t total = nbt * N * half_pitch;
  if (total <= 0) return;
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
  // 32-bit indices when every index and offset of B and the expanded copy fits
  if (2 * total < (int64_t(1) << 31) && nbt * N * K < (int64_t(1) << 30))
    expand_typed<int32_t>(B, b_bt, b_k, b_n, nbt, N, K, half_pitch, bf16, Bx, s, in_c64, Bx_lo, bscale, blocks);
  else
    expand_typed<int64_t>(B, b_bt, b_k, b_n, nbt, N, K, half_pitch, bf16, Bx, s, in_c64, Bx_lo, bscale, blocks);
}

int64_t expanded_half_pitch(int64_t K) { return (2 * K + BK - 1) / BK * BK / 2; }

int64_t expanded_b_bytes(int64_t nbt, int64_t N, int64_t K) {
  return nbt * 2 * N * ((2 * K + BK - 1) / BK * BK) * 2;
}

// ------------------------------------------------------------ self-test
namespace {
__device__ __forceinline__ float hash_unit(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdULL;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ULL;
  x ^= x >> 33;
  return (float)((x >> 40) * (1.0 / 16777216.0)) * 2.0f - 1.0f;
}
template <class T2>
__global__ void fill_kernel(T2* p, int64_t n, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float re = hash_unit(seed * 0x9E3779B97F4A7C15ULL + 2 * i);
    float im = hash_unit(seed * 0x9E3779B97F4A7C15ULL + 2 * i + 1);
    T2 v;
    v.x = re;
    v.y = im;
    p[i] = v;
  }
}
// reference: plain FP32 complex GEMM from the same 16-bit inputs
template <class T2>
__global__ void ref_kernel(const T2* A, const T2* B, float2* C, int64_t nbt, int64_t M, int64_t N, int64_t K) {
  const int64_t total = nbt * M * N;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = x % N, m = (x / N) % M, bt = x / (N * M);
    float re = 0.f, im = 0.f;
    for (int64_t k = 0; k < K; ++k) {
      const T2 a = A[(bt * M + m) * K + k];
      const T2 b = B[(bt * K + k) * N + n];
      const float ar = (float)a.x, ai = (float)a.y, br = (float)b.x, bi = (float)b.y;
      re = fmaf(ar, br, re);
      re = fmaf(-ai, bi, re);
      im = fmaf(ar, bi, im);
      im = fmaf(ai, br, im);
    }
    C[x] = make_float2(re, im);
  }
}
__global__ void diff_kernel(const float2* a, const float2* b, int64_t n, unsigned* max_diff, unsigned* max_ref) {
  float md = 0.f, mr = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float dx = a[i].x - b[i].x, dy = a[i].y - b[i].y;
    md = fmaxf(md, sqrtf(dx * dx + dy * dy));
    mr = fmaxf(mr, sqrtf(b[i].x * b[i].x + b[i].y * b[i].y));
    if (!(a[i].x == a[i].x) || !(a[i].y == a[i].y)) md = 3.0e38f;
  }
  atomicMax(max_diff, __float_as_uint(md));
  atomicMax(max_ref, __float_as_uint(mr));
}
}  // namespace

double selftest_gemm_tc(int64_t nbt, int64_t M, int64_t N, int64_t K, bool bf16, uint64_t seed, cudaStream_t s,
                        int* d_err) {
  void *A = nullptr, *B = nullptr, *Bx = nullptr, *C = nullptr, *R = nullptr;
  unsigned* mx = nullptr;
  auto cleanup = [&] {
    for (void* q : {A, B, Bx, C, R, (void*)mx})
      if (q) cudaFree(q);
  };
  try {
    TN_CUDA(cudaMalloc(&A, nbt * M * K * 4));
    TN_CUDA(cudaMalloc(&B, nbt * K * N * 4));
    TN_CUDA(cudaMalloc(&Bx, expanded_b_bytes(nbt, N, K)));
    TN_CUDA(cudaMalloc(&C, nbt * M * N * 8));
    TN_CUDA(cudaMalloc(&R, nbt * M * N * 8));
    TN_CUDA(cudaMalloc(&mx, 8));
    TN_CUDA(cudaMemsetAsync(mx, 0, 8, s));
    TN_CUDA(cudaMemsetAsync(C, 0xff, nbt * M * N * 8, s));  // NaN pattern: unwritten outputs fail
    if (bf16) {
      fill_kernel<__nv_bfloat162><<<1024, 256, 0, s>>>((__nv_bfloat162*)A, nbt * M * K, seed);
      fill_kernel<__nv_bfloat162><<<1024, 256, 0, s>>>((__nv_bfloat162*)B, nbt * K * N, seed + 1);
    } else {
      fill_kernel<__half2><<<1024, 256, 0, s>>>((__half2*)A, nbt * M * K, seed);
      fill_kernel<__half2><<<1024, 256, 0, s>>>((__half2*)B, nbt * K * N, seed + 1);
    }
    // B stored [bt][k][n] (n contiguous): the expansion reads it strided
    launch_expand_b(B, single_run(nbt, K * N), single_run(K, N), single_run(N, 1), nbt, N, K, bf16, Bx, s);
    TcGemmParams p{};
    p.nbt = nbt;
    p.M = M;
    p.N = N;
    p.K = K;
    p.c_bt = single_run(nbt, M * N);
    p.c_m = single_run(M, N);
    p.c_n = single_run(N, 1);
    p.C = C;
    p.out_kind = 2;
    p.scale = 1.0f;
    p.err = d_err;
    p.bn = tc_gemm_bn(N);
    // both variants: one CTA per tile, and two-CTA clusters sharing B by multicast;
    // the second overwrites the first, then is compared; the first is compared below
    p.cluster2 = 0;
    launch_gemm_tc(A, nullptr, M * K, K, Bx, nullptr, p, bf16, s);
    if (bf16)
      ref_kernel<__nv_bfloat162><<<1024, 256, 0, s>>>((const __nv_bfloat162*)A, (const __nv_bfloat162*)B,
                                                     (float2*)R, nbt, M, N, K);
    else
      ref_kernel<__half2><<<1024, 256, 0, s>>>((const __half2*)A, (const __half2*)B, (float2*)R, nbt, M, N, K);
    diff_kernel<<<1024, 256, 0, s>>>((const float2*)C, (const float2*)R, nbt * M * N, mx, mx + 1);
    TN_CUDA(cudaMemsetAsync(C, 0xff, nbt * M * N * 8, s));
    p.cluster2 = 1;
    launch_gemm_tc(A, nullptr, M * K, K, Bx, nullptr, p, bf16, s);
    diff_kernel<<<1024, 256, 0, s>>>((const float2*)C, (const float2*)R, nbt * M * N, mx, mx + 1);
    unsigned h[2] = {0, 0};
    TN_CUDA(cudaMemcpyAsync(h, mx, 8, cudaMemcpyDeviceToHost, s));
    TN_CUDA(cudaStreamSynchronize(s));
    cleanup();
    float md, mr;
    std::memcpy(&md, &h[0], 4);
    std::memcpy(&mr, &h[1], 4);
    return mr > 0 ? (double)md / (double)mr : (double)md;
  } catch (...) {
    cudaStreamSynchronize(s);
    cleanup();
    throw;
  }
}

}  // namespace tn
