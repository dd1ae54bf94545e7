// Complex strided-gather GEMM on CUDA cores: the plain complex64 path, and
// the small steps of the reduced-precision path (FP32 arithmetic; complex64
// operands; complex64 or 16-bit complex results).
//
// One pairwise contraction of the tree (arXiv 2406.18889, Sec. III: the
// per-step tensor contraction the paper runs through cuTensor or
// transpose-transpose-GEMM-transpose) is C[bt][m][n] = sum_k A[bt][m][k] *
// B[bt][k][n].  Each index group of each tensor is addressed through its runs
// (tn_internal.h), so operands are read and results written in whatever
// layout the plan chose -- no separate transpose pass.  Each complex
// multiply-add is four FP32 fused multiply-adds.
//
// Two kernels:
//  * tiled: a CTA of 256 threads computes a TM x TN tile; per CTA the row and
//    column offsets of the tile are tabulated in shared memory once (and the k
//    offsets once per TK-deep slice); operands are staged through shared
//    memory with loads coalesced along whichever index is contiguous; each
//    thread keeps RM x RN complex accumulators.
//  * small-K: for K <= 4 (outer-product-like steps, bound by writing C).  A
//    CTA owns 2^P consecutive outputs of C's memory order; the A and B
//    entries those outputs use are staged in shared memory once per tile,
//    and every position map involved (output position -> A entry, B entry,
//    destination offset) is linear over the position's bits, so two small
//    per-CTA tables give each thread its operands and destination.  The
//    destination is C itself, or -- when the result is the expanded operand
//    of a tensor-core step -- that operand's real 2x2 form, written in place
//    of a separate expansion pass.
//  * direct: one thread per output element, for the remaining shapes too
//    small for a tile.
#include <algorithm>
#include <map>
#include <mutex>
#include <set>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tn_internal.h"

namespace tn {
namespace {

// storage <-> FP32 complex
struct C64 {
  using T = float2;
  static __device__ __forceinline__ float2 ld(const T& v) { return v; }
  static __device__ __forceinline__ T st(float2 v) { return v; }
};
struct F16 {
  using T = __half2;
  static __device__ __forceinline__ float2 ld(const T& v) { return __half22float2(v); }
  static __device__ __forceinline__ T st(float2 v) { return __floats2half2_rn(v.x, v.y); }
};
struct BF16 {
  using T = __nv_bfloat162;
  static __device__ __forceinline__ float2 ld(const T& v) { return __bfloat1622float2(v); }
  static __device__ __forceinline__ T st(float2 v) { return __floats2bfloat162_rn(v.x, v.y); }
};
// store v as a 16-bit pair plus its rounding residual (hi + lo)
template <class H>
__device__ __forceinline__ void store_out(typename H::T* C, typename H::T* C2, int64_t o, float2 v, bool hilo) {
  const typename H::T hi = H::st(v);
  C[o] = hi;
  if (hilo) {
    const float2 h = H::ld(hi);
    C2[o] = H::st(make_float2(v.x - h.x, v.y - h.y));
  }
}
template <>
__device__ __forceinline__ void store_out<C64>(float2* C, float2*, int64_t o, float2 v, bool) {
  C[o] = v;
}

__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

// flags: bit 0 = A loads run along k (A's k is contiguous), bit 1 = B loads run along n
template <int TM, int TN, int TK, int TY, int TX, class In, class Out>
__global__ void __launch_bounds__(256) gemm_tiled(GemmParams p, float scale, bool hilo, int flags) {
  static_assert(TY * TX == 256, "256 threads");
  constexpr int RM = TM / TY, RN = TN / TX;
  constexpr int LA = (TM * TK + 255) / 256, LB = (TN * TK + 255) / 256;  // loads per thread per k slice
  using TI = typename In::T;
  using TO = typename Out::T;
  __shared__ float2 As[2][TK][TM + 1];
  __shared__ float2 Bs[2][TK][TN + 1];
  __shared__ int64_t a_row[TM], b_col[TN], c_row[TM], c_col[TN];
  __shared__ int64_t a_kof[TK], b_kof[TK];
  const TI* __restrict__ A = (const TI*)p.A;
  const TI* __restrict__ Bm = (const TI*)p.B;
  TO* __restrict__ C = (TO*)p.C;
  TO* __restrict__ C2 = (TO*)p.C2;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  // blockIdx.x walks the (m tile, n tile) grid, n tile fastest
  const int64_t n_tiles = (p.N + TN - 1) / TN;
  const int64_t m0 = (int64_t)(blockIdx.x / n_tiles) * TM, n0 = (int64_t)(blockIdx.x % n_tiles) * TN;
  const bool a_kc = flags & 1;
  const bool b_nc = flags & 2;
  for (int i = tid; i < TM; i += 256) {
    a_row[i] = m0 + i < p.M ? run_offset(p.a_m, m0 + i) : 0;
    c_row[i] = m0 + i < p.M ? run_offset(p.c_m, m0 + i) : 0;
  }
  for (int i = tid; i < TN; i += 256) {
    b_col[i] = n0 + i < p.N ? run_offset(p.b_n, n0 + i) : 0;
    c_col[i] = n0 + i < p.N ? run_offset(p.c_n, n0 + i) : 0;
  }
  // k slices start at multiples of TK (a power of two), so a slice's contracted
  // offsets are its start's offset plus this CTA-constant table (run offsets
  // are linear over disjoint index bits)
  if (tid < TK) a_kof[tid] = run_offset(p.a_k, tid);
  if (tid >= 32 && tid < 32 + TK) b_kof[tid - 32] = run_offset(p.b_k, tid - 32);
  __syncthreads();
  // this thread's (row, k) and (k, col) slots of a slice, in the coalesced order
  int a_mm[LA], a_kk[LA], b_nn[LB], b_kk[LB];
#pragma unroll
  for (int q = 0; q < LA; ++q) {
    const int l = tid + q * 256;
    a_mm[q] = a_kc ? l / TK : l % TM;
    a_kk[q] = a_kc ? l % TK : l / TM;
  }
#pragma unroll
  for (int q = 0; q < LB; ++q) {
    const int l = tid + q * 256;
    b_nn[q] = b_nc ? l % TN : l / TK;
    b_kk[q] = b_nc ? l / TN : l % TK;
  }
  for (int64_t bt = blockIdx.z; bt < p.nbt; bt += gridDim.z) {
    const TI* Ab = A + run_offset(p.a_bt, bt);
    const TI* Bb = Bm + run_offset(p.b_bt, bt);
    float2 acc[RM][RN];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
      for (int j = 0; j < RN; ++j) acc[i][j] = make_float2(0.f, 0.f);
    float2 ra[LA], rb[LB];
    // operands of the slice starting at k0 into registers
    auto fetch = [&](int64_t k0) {
      const int64_t ab = run_offset(p.a_k, k0), bb = run_offset(p.b_k, k0);
#pragma unroll
      for (int q = 0; q < LA; ++q) {
        ra[q] = make_float2(0.f, 0.f);
        if (tid + q * 256 < TM * TK && m0 + a_mm[q] < p.M && k0 + a_kk[q] < p.K)
          ra[q] = In::ld(Ab[a_row[a_mm[q]] + ab + a_kof[a_kk[q]]]);
      }
#pragma unroll
      for (int q = 0; q < LB; ++q) {
        rb[q] = make_float2(0.f, 0.f);
        if (tid + q * 256 < TN * TK && n0 + b_nn[q] < p.N && k0 + b_kk[q] < p.K)
          rb[q] = In::ld(Bb[bb + b_kof[b_kk[q]] + b_col[b_nn[q]]]);
      }
    };
    auto stash = [&](int buf) {
#pragma unroll
      for (int q = 0; q < LA; ++q)
        if (tid + q * 256 < TM * TK) As[buf][a_kk[q]][a_mm[q]] = ra[q];
#pragma unroll
      for (int q = 0; q < LB; ++q)
        if (tid + q * 256 < TN * TK) Bs[buf][b_kk[q]][b_nn[q]] = rb[q];
    };
    __syncthreads();  // the previous batch entry's last slice is consumed
    fetch(0);
    stash(0);
    int buf = 0;
    for (int64_t k0 = 0; k0 < p.K; k0 += TK) {
      __syncthreads();  // slice k0 is in As/Bs[buf]; the other buffer is free
      const bool more = k0 + TK < p.K;
      if (more) fetch(k0 + TK);  // global loads in flight during the multiply-adds
#pragma unroll
      for (int kk = 0; kk < TK; ++kk) {
        float2 a[RM], b[RN];
#pragma unroll
        for (int i = 0; i < RM; ++i) a[i] = As[buf][kk][ty + i * TY];
#pragma unroll
        for (int j = 0; j < RN; ++j) b[j] = Bs[buf][kk][tx + j * TX];
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
          for (int j = 0; j < RN; ++j) cmac(acc[i][j], a[i], b[j]);
      }
      if (more) stash(buf ^ 1);
      buf ^= 1;
    }
    const int64_t cb = run_offset(p.c_bt, bt);
#pragma unroll
    for (int i = 0; i < RM; ++i) {
      const int mm = ty + i * TY;
      if (m0 + mm >= p.M) continue;
#pragma unroll
      for (int j = 0; j < RN; ++j) {
        const int nn = tx + j * TX;
        if (n0 + nn < p.N)
          store_out<Out>(C, C2, cb + c_row[mm] + c_col[nn], make_float2(acc[i][j].x * scale, acc[i][j].y * scale),
                         hilo);
      }
    }
  }
}

// one thread per output element, walking C in memory order (coalesced writes);
// (bt, m, n) are decoded from the output offset's bits.  I is the index type:
// 32-bit when every operand and the result hold fewer than 2^31 elements.
template <class I>
__device__ __forceinline__ I run_off(const Runs& R, I i) {
  I o = 0;
  for (int r = 0; r < R.n; ++r) {
    o += (i & ((I(1) << R.lg[r]) - 1)) * (I)R.st[r];
    i >>= R.lg[r];
  }
  return o;
}

constexpr int64_t kDirectVecMin = int64_t(152) * 256 * 4;  // outputs from which a thread takes four

template <class In, class Out, class I>
__global__ void __launch_bounds__(256) gemm_direct(GemmParams p, float scale, bool hilo) {
  using TI = typename In::T;
  using TO = typename Out::T;
  const TI* __restrict__ A = (const TI*)p.A;
  const TI* __restrict__ Bm = (const TI*)p.B;
  TO* __restrict__ C = (TO*)p.C;
  const I total = (I)(p.nbt * p.M * p.N);
  const int K = (int)p.K;
  // the contracted offsets of K <= 4 are the same for every output: tabulate them
  I ak[4] = {0, 0, 0, 0}, bk[4] = {0, 0, 0, 0};
  const bool small_k = K <= 4;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (k < K) {
      ak[k] = run_off<I>(p.a_k, (I)k);
      bk[k] = run_off<I>(p.b_k, (I)k);
    }
  // four consecutive outputs per thread when C's fastest run (pos 0) spans >= 4
  // elements: they differ only in that run's digit, i.e. in one group's index
  // (only when the grid is full anyway: small steps take one output per thread)
  const bool vec = p.c_dec.n > 0 && p.c_dec.pos[0] == 0 && p.c_dec.lg[0] >= 2 && (total & 3) == 0 &&
                   total >= (I)kDirectVecMin;
  const int g0 = p.c_dec.grp[0];
  const I step0 = I(1) << p.c_dec.shift[0];
  const I per = vec ? 4 : 1;
  for (I x = (blockIdx.x * (I)blockDim.x + threadIdx.x) * per; x < total; x += (I)gridDim.x * blockDim.x * per) {
    I i0 = 0, i1 = 0, i2 = 0;  // (bt, m, n) in registers (no dynamically indexed array)
    for (int e = 0; e < p.c_dec.n; ++e) {
      const I d = ((x >> p.c_dec.pos[e]) & ((I(1) << p.c_dec.lg[e]) - 1)) << p.c_dec.shift[e];
      const int g = p.c_dec.grp[e];
      i0 |= g == 0 ? d : I(0);
      i1 |= g == 1 ? d : I(0);
      i2 |= g == 2 ? d : I(0);
    }
    for (I v = 0; v < per; ++v) {
      const TI* a = A + run_off<I>(p.a_bt, i0) + run_off<I>(p.a_m, i1);
      const TI* b = Bm + run_off<I>(p.b_bt, i0) + run_off<I>(p.b_n, i2);
      float2 acc = make_float2(0.f, 0.f);
      if (small_k) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (k < K) cmac(acc, In::ld(a[ak[k]]), In::ld(b[bk[k]]));
      } else {
        // four k at a time, their eight loads issued before the multiply-adds
        int k = 0;
        for (; k + 4 <= K; k += 4) {
          TI av[4], bv[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            av[q] = a[run_off<I>(p.a_k, (I)(k + q))];
            bv[q] = b[run_off<I>(p.b_k, (I)(k + q))];
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) cmac(acc, In::ld(av[q]), In::ld(bv[q]));
        }
        for (; k < K; ++k)
          cmac(acc, In::ld(a[run_off<I>(p.a_k, (I)k)]), In::ld(b[run_off<I>(p.b_k, (I)k)]));
      }
      store_out<Out>(C, (TO*)p.C2, (int64_t)(x + v), make_float2(acc.x * scale, acc.y * scale), hilo);
      i0 += g0 == 0 ? step0 : I(0);
      i1 += g0 == 1 ? step0 : I(0);
      i2 += g0 == 2 ? step0 : I(0);
    }
  }
}

// ------------------------------------------------------------------ small K
constexpr int kSkMaxTileBits = 12;  // outputs per tile <= 4096
constexpr int kSkMaxStage = 2048;   // staged entries per operand (16 KB)

struct SmallK {
  const float2* A;
  const float2* B;
  void* C;
  void* C2;
  int K, lgK;    // contracted extent (1, 2 or 4)
  int nbits;     // log2 of the outputs
  int P;         // log2 of the outputs per tile
  int na, nb;    // bits of the staged A / B index
  int8_t a_rank[kSkMaxTileBits], b_rank[kSkMaxTileBits];  // tile bit -> staged-index bit (-1: none)
  int64_t a_wt[kSkMaxTileBits], b_wt[kSkMaxTileBits];     // staged-index bit -> operand offset
  int64_t a_w[kMaxBits], b_w[kMaxBits], o_w[kMaxBits];    // output-position bit -> offsets
  int64_t ak[4], bk[4];                                   // contracted-index offsets
  int64_t hp;    // expanded destination: row pitch in 16-bit pairs
  float scale;
};

// v into the expanded form at row pair (o, o + hp): [[Re, -Im], [Im, Re]];
// with Xlo also the rounding residual of every entry
template <class H>
__device__ __forceinline__ void store_expanded(typename H::T* X, typename H::T* Xlo, int64_t o, int64_t hp,
                                               float2 v) {
  X[o] = H::st(make_float2(v.x, -v.y));  // round-to-nearest is odd-symmetric: this is -(rounded Im)
  X[o + hp] = H::st(make_float2(v.y, v.x));
  if (Xlo) {
    const float2 h = H::ld(H::st(v));
    const float2 l = make_float2(v.x - h.x, v.y - h.y);
    Xlo[o] = H::st(make_float2(l.x, -l.y));
    Xlo[o + hp] = H::st(make_float2(l.y, l.x));
  }
}

// V adjacent results (V = 1 or 2) at element offset o of the destination
template <class Out, int MODE, int V>
__device__ __forceinline__ void store_v(const SmallK& p, int64_t o, const float2 (&v)[V], bool hilo) {
  using TO = typename Out::T;
  TO* C = reinterpret_cast<TO*>(p.C);
  TO* C2 = reinterpret_cast<TO*>(p.C2);
  if constexpr (V == 1) {
    if constexpr (MODE == 0)
      store_out<Out>(C, C2, o, v[0], hilo);
    else
      store_expanded<Out>(C, C2, o, p.hp, v[0]);
  } else if constexpr (MODE == 0 && std::is_same_v<Out, C64>) {
    *reinterpret_cast<float4*>(reinterpret_cast<float2*>(p.C) + o) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
  } else if constexpr (MODE == 0) {
    // two 16-bit complex values (8 bytes), and their residuals when split
    TO h[2] = {Out::st(v[0]), Out::st(v[1])};
    *reinterpret_cast<uint2*>(C + o) = *reinterpret_cast<const uint2*>(h);
    if (hilo) {
      const float2 f0 = Out::ld(h[0]), f1 = Out::ld(h[1]);
      TO l[2] = {Out::st(make_float2(v[0].x - f0.x, v[0].y - f0.y)), Out::st(make_float2(v[1].x - f1.x, v[1].y - f1.y))};
      *reinterpret_cast<uint2*>(C2 + o) = *reinterpret_cast<const uint2*>(l);
    }
  } else {
    // expanded rows o (Re, -Im) and o + hp (Im, Re), two columns each
    TO r0[2] = {Out::st(make_float2(v[0].x, -v[0].y)), Out::st(make_float2(v[1].x, -v[1].y))};
    TO r1[2] = {Out::st(make_float2(v[0].y, v[0].x)), Out::st(make_float2(v[1].y, v[1].x))};
    *reinterpret_cast<uint2*>(C + o) = *reinterpret_cast<const uint2*>(r0);
    *reinterpret_cast<uint2*>(C + o + p.hp) = *reinterpret_cast<const uint2*>(r1);
    if (C2) {
      float2 l[2];
      for (int i = 0; i < 2; ++i) {
        const float2 h = Out::ld(Out::st(v[i]));
        l[i] = make_float2(v[i].x - h.x, v[i].y - h.y);
      }
      TO q0[2] = {Out::st(make_float2(l[0].x, -l[0].y)), Out::st(make_float2(l[1].x, -l[1].y))};
      TO q1[2] = {Out::st(make_float2(l[0].y, l[0].x)), Out::st(make_float2(l[1].y, l[1].x))};
      *reinterpret_cast<uint2*>(C2 + o) = *reinterpret_cast<const uint2*>(q0);
      *reinterpret_cast<uint2*>(C2 + o + p.hp) = *reinterpret_cast<const uint2*>(q1);
    }
  }
}

// 8-byte asynchronous copy global -> shared (both 8-byte aligned)
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst))),
               "l"(gmem_src)
               : "memory");
}

// MODE 0: C[o] = result (Out storage, hi + lo when `hilo`); MODE 1: expanded
// destination.  KC: the contracted extent; V: adjacent outputs per thread (the
// tile's bit 0 is then a unit-stride bit of the destination).  Thread t of a
// tile takes outputs V*(t + 256*i) + v: the part of every map that depends on
// t is read once into registers, the part that depends on i is a broadcast.
// The staged A and B entries of tile n+1 are copied (cp.async) while tile n is
// computed, into the other half of a double buffer; staged entry
// s = t + 256 r of a tile has operand offset tile base + (thread part, in a
// register) + (part of r, a table of at most 8 entries).
template <class Out, int MODE, int KC, int V>
__global__ void __launch_bounds__(256) gemm_smallk(SmallK p, bool hilo) {
  extern __shared__ float2 staged[];
  __shared__ uint32_t sel_lo[256], sel_hi[16];
  __shared__ int64_t off_lo[256], off_hi[16];
  __shared__ int64_t a_hi[8], b_hi[8];
  __shared__ int64_t w_a[kMaxBits], w_b[kMaxBits], w_o[kMaxBits];  // position-bit weights (lanes read them per bit)
  constexpr int lgK = KC == 1 ? 0 : KC == 2 ? 1 : 2;
  for (int j = threadIdx.x; j < p.nbits; j += blockDim.x) {
    w_a[j] = p.a_w[j];
    w_b[j] = p.b_w[j];
    w_o[j] = p.o_w[j];
  }
  constexpr int sh = V - 1;  // tile bits below the thread index
  const int na_n = KC << p.na, nb_n = KC << p.nb;
  const int buf_n = na_n + nb_n;  // buffer q starts at staged + q * buf_n
  // tables over tile bits sh..sh+7 (thread index) and sh+8.. (iteration);
  // linear maps: OR / sum of the parts
  {
    const int j = threadIdx.x;
    uint32_t sel = 0;
    int64_t off = 0;
    for (int b = 0; b < 8 && b + sh < p.P; ++b)
      if ((j >> b) & 1) {
        if (p.a_rank[b + sh] >= 0) sel |= 1u << p.a_rank[b + sh];
        if (p.b_rank[b + sh] >= 0) sel |= 1u << (16 + p.b_rank[b + sh]);
        off += p.o_w[b + sh];
      }
    sel_lo[j] = sel;
    off_lo[j] = off;
    if (j < 16) {
      sel = 0;
      off = 0;
      for (int b = 0; b + 8 + sh < p.P; ++b)
        if ((j >> b) & 1) {
          if (p.a_rank[b + 8 + sh] >= 0) sel |= 1u << p.a_rank[b + 8 + sh];
          if (p.b_rank[b + 8 + sh] >= 0) sel |= 1u << (16 + p.b_rank[b + 8 + sh]);
          off += p.o_w[b + 8 + sh];
        }
      sel_hi[j] = sel;
      off_hi[j] = off;
    }
    // staged entry s = j + 256 r: u = s >> lgK takes bits 0..7-lgK from j and
    // the rest from r (256 is a multiple of KC)
    if (j < 8) {
      int64_t ah = 0, bh = 0;
      for (int b = 0; b < 3; ++b)
        if ((j >> b) & 1) {
          const int q = 8 - lgK + b;
          if (q < p.na) ah += p.a_wt[q];
          if (q < p.nb) bh += p.b_wt[q];
        }
      a_hi[j] = ah;
      b_hi[j] = bh;
    }
  }
  int64_t a_lo = p.ak[threadIdx.x & (KC - 1)], b_lo = p.bk[threadIdx.x & (KC - 1)];
  {
    const int u = threadIdx.x >> lgK;
    for (int b = 0; b < 8 - lgK; ++b)
      if ((u >> b) & 1) {
        if (b < p.na) a_lo += p.a_wt[b];
        if (b < p.nb) b_lo += p.b_wt[b];
      }
  }
  // tile bit 0 (V = 2): its staged-index bits (rank 0 when it is an A / B bit)
  const uint32_t a_v = (V == 2 && p.a_rank[0] >= 0) ? 1u : 0u;
  const uint32_t b_v = (V == 2 && p.b_rank[0] >= 0) ? 1u : 0u;
  const int64_t ntiles = int64_t(1) << (p.nbits - p.P);
  const int n_q = (1 << p.P) / V;
  // A, B and destination offsets of tile origins: warp 0 forms them two
  // tiles ahead (lanes take the tile index bits, then a warp reduction)
  __shared__ int64_t tile_base[2][3];
  const int lane = threadIdx.x & 31;
  auto bases = [&](int64_t t, int slot) {
    int64_t a = 0, b = 0, o = 0;
    for (int j = p.P + lane; j < p.nbits; j += 32)
      if ((t >> (j - p.P)) & 1) {
        a += w_a[j];
        b += w_b[j];
        o += w_o[j];
      }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, s);
      b += __shfl_xor_sync(0xffffffffu, b, s);
      o += __shfl_xor_sync(0xffffffffu, o, s);
    }
    if (lane == 0) {
      tile_base[slot][0] = a;
      tile_base[slot][1] = b;
      tile_base[slot][2] = o;
    }
  };
  // queue the asynchronous copies of one tile's staged entries into buffer q.
  // Entry s = (u << lgK) | k is read from global memory in s order and stored
  // k-major (k * 2^na + u), so that the lanes of a warp, which take
  // consecutive u, read shared memory without bank conflicts
  const int na_u = 1 << p.na, nb_u = 1 << p.nb;
  const int a_dst = (threadIdx.x & (KC - 1)) * na_u + (threadIdx.x >> lgK);
  const int b_dst = (threadIdx.x & (KC - 1)) * nb_u + (threadIdx.x >> lgK);
  auto stage = [&](int slot, int q) {
    const int64_t a0 = tile_base[slot][0] + a_lo, b0 = tile_base[slot][1] + b_lo;
    float2* As = staged + q * buf_n;
    float2* Bs = As + na_n;
    for (int r = 0, i = threadIdx.x; i < na_n; ++r, i += 256)
      cp_async8(As + a_dst + (r << (8 - lgK)), p.A + a0 + a_hi[r]);
    for (int r = 0, i = threadIdx.x; i < nb_n; ++r, i += 256)
      cp_async8(Bs + b_dst + (r << (8 - lgK)), p.B + b0 + b_hi[r]);
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  const int64_t G = gridDim.x;
  __syncthreads();  // the weight tables
  if (threadIdx.x < 32 && (int64_t)blockIdx.x < ntiles) bases(blockIdx.x, 0);
  __syncthreads();
  if ((int64_t)blockIdx.x < ntiles) stage(0, 0);
  if (threadIdx.x < 32 && blockIdx.x + G < ntiles) bases(blockIdx.x + G, 1);
  const uint32_t sel_t = sel_lo[threadIdx.x];
  const int64_t off_t = off_lo[threadIdx.x];
  int it = 0;
  for (int64_t t = blockIdx.x; t < ntiles; t += G, ++it) {
    const int cur = it & 1;
    __syncthreads();  // the next tile's bases visible; the other buffer consumed
    const int64_t o0 = tile_base[cur][2];
    if (t + G < ntiles) {
      stage(cur ^ 1, cur ^ 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();  // this tile's staged entries visible; every thread holds o0
    if (threadIdx.x < 32 && t + 2 * G < ntiles) bases(t + 2 * G, cur);
    const float2* As = staged + cur * buf_n;
    const float2* Bs = As + na_n;
    const int64_t ot = o0 + off_t;
#pragma unroll 2
    for (int q = threadIdx.x; q < n_q; q += blockDim.x) {
      const int h = q >> 8;
      const uint32_t sel = sel_t | sel_hi[h];
      const uint32_t ua = sel & 0xffffu, ub = sel >> 16;
      float2 r[V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const float2* a = As + (ua | (v ? a_v : 0u));
        const float2* b = Bs + (ub | (v ? b_v : 0u));
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < KC; ++k) cmac(acc, a[k * na_u], b[k * nb_u]);
        r[v] = make_float2(acc.x * p.scale, acc.y * p.scale);
      }
      store_v<Out, MODE, V>(p, ot + off_hi[h], r, hilo);
    }
  }
}

// ------------------------------------------------------------------ rows
// Small K with few outputs per row (K <= 4, N <= 8, the result written in
// place): thread t takes rows (bt, m) of the step, loads the row's K entries
// of A once (16-byte loads when they are contiguous), forms all N outputs in
// registers from B (held in registers when the step has one batch) and stores
// them (pairs when consecutive n are adjacent).  A thread takes 2 or 4 rows
// of a chunk and issues their loads together.  Row r = bt * M + m is
// addressed bit-linearly: its low bits (the thread and its row within the
// chunk) by a register part, the rest (the chunk) by a warp reduction over
// per-bit weights.
struct RowsK {
  const float2* A;
  const float2* B;
  void* C;
  void* C2;
  int nbits;                               // log2 of the rows
  int64_t a_w[kMaxBits], c_w[kMaxBits], b_w[kMaxBits];  // row bit -> A / C / B offset
  int64_t ak[4], bk[4];                    // contracted-index offsets
  int64_t cn[8], bn[8];                    // output / B offsets of n
  int a_vec;                               // a row's K entries contiguous and 16-byte aligned
  int b_fixed;                             // one batch: B the same for every row
  int c_pairs;                             // n = 2i, 2i + 1 adjacent and pair-aligned
  float scale;
};

template <class Out, int KC, int NC>
__global__ void __launch_bounds__(256, 2) gemm_rows(RowsK p, bool hilo) {
  __shared__ int64_t w[3][kMaxBits];
  for (int j = threadIdx.x; j < p.nbits; j += blockDim.x) {
    w[0][j] = p.a_w[j];
    w[1][j] = p.c_w[j];
    w[2][j] = p.b_w[j];
  }
  __syncthreads();
  using TO = typename Out::T;
  TO* C = reinterpret_cast<TO*>(p.C);
  TO* C2 = reinterpret_cast<TO*>(p.C2);
  const int lane = threadIdx.x & 31;
  // the thread's part of the row offsets (row bits 0..7)
  int64_t a_t = 0, c_t = 0, b_t = 0;
  for (int j = 0; j < 8 && j < p.nbits; ++j)
    if ((threadIdx.x >> j) & 1) {
      a_t += w[0][j];
      c_t += w[1][j];
      b_t += w[2][j];
    }
  float2 bf[KC][NC];
  if (p.b_fixed) {
#pragma unroll
    for (int k = 0; k < KC; ++k)
#pragma unroll
      for (int n = 0; n < NC; ++n) bf[k][n] = __ldg(p.B + p.bk[k] + p.bn[n]);
  }
  // a chunk is 256 R rows: thread t takes rows t + 256 q (q < R), the row
  // bits 8, 9 being q; their R A loads are issued before any arithmetic, so
  // each thread keeps several rows' loads in flight (R = 2 where the B
  // registers of a larger tile leave no room for four rows)
  constexpr int R = KC * NC <= 16 ? 4 : 2;
  constexpr int lgR = R == 4 ? 2 : 1;
  int64_t a_q[R], c_q[R], b_q[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    a_q[q] = a_t;
    c_q[q] = c_t;
    b_q[q] = b_t;
    for (int j = 0; j < lgR; ++j)
      if (((q >> j) & 1) && 8 + j < p.nbits) {
        a_q[q] += w[0][8 + j];
        c_q[q] += w[1][8 + j];
        b_q[q] += w[2][8 + j];
      }
  }
  const int64_t rows = int64_t(1) << p.nbits;
  const int lgC = 8 + lgR;
  const int64_t chunks = (rows + (256 * R - 1)) >> lgC;
  for (int64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
    // chunk offsets: lane j sums the weights of row bits lgC + j, lgC + 32 + j
    int64_t a0 = 0, c0 = 0, b0 = 0;
    for (int j = lgC + lane; j < p.nbits; j += 32)
      if ((c >> (j - lgC)) & 1) {
        a0 += w[0][j];
        c0 += w[1][j];
        b0 += w[2][j];
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      c0 += __shfl_xor_sync(0xffffffffu, c0, o);
      b0 += __shfl_xor_sync(0xffffffffu, b0, o);
    }
    float2 a[R][KC];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if ((c << lgC) + (q << 8) + threadIdx.x >= rows) continue;
      const int64_t ao = a0 + a_q[q];
      if (KC >= 2 && p.a_vec) {
#pragma unroll
        for (int k = 0; k < KC; k += 2) {
          const float4 v = __ldcs(reinterpret_cast<const float4*>(p.A + ao + k));
          a[q][k] = make_float2(v.x, v.y);
          a[q][k + 1] = make_float2(v.z, v.w);
        }
      } else {
#pragma unroll
        for (int k = 0; k < KC; ++k) a[q][k] = __ldcs(p.A + ao + p.ak[k]);
      }
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if ((c << lgC) + (q << 8) + threadIdx.x >= rows) continue;
      const int64_t co = c0 + c_q[q];
      float2 r[NC];
#pragma unroll
      for (int n = 0; n < NC; ++n) r[n] = make_float2(0.f, 0.f);
      if (p.b_fixed) {
#pragma unroll
        for (int k = 0; k < KC; ++k)
#pragma unroll
          for (int n = 0; n < NC; ++n) cmac(r[n], a[q][k], bf[k][n]);
      } else {
        const int64_t bo = b0 + b_q[q];
#pragma unroll
        for (int k = 0; k < KC; ++k)
#pragma unroll
          for (int n = 0; n < NC; ++n) cmac(r[n], a[q][k], __ldg(p.B + bo + p.bk[k] + p.bn[n]));
      }
#pragma unroll
      for (int n = 0; n < NC; ++n) r[n] = make_float2(r[n].x * p.scale, r[n].y * p.scale);
      if (NC >= 2 && p.c_pairs) {
        SmallK sq{};  // store_v reads only the destination pointers
        sq.C = p.C;
        sq.C2 = p.C2;
#pragma unroll
        for (int n = 0; n < NC; n += 2) {
          const float2 v2[2] = {r[n], r[n + 1]};
          store_v<Out, 0, 2>(sq, co + p.cn[n], v2, hilo);
        }
      } else {
#pragma unroll
        for (int n = 0; n < NC; ++n) store_out<Out>(C, C2, co + p.cn[n], r[n], hilo);
      }
    }
  }
}

// dynamic shared memory above 48 KB: opted in once per (function, device)
void set_max_dynamic_smem(const void* fn, int bytes) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  TN_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({fn, dev})) return;
  TN_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.insert({fn, dev});
}

// CTAs of 256 threads resident per SM for a function and its dynamic shared
// memory (cached: the launch sequence of a plan asks again and again)
int resident_blocks(const void* fn, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<const void*, size_t>, int> known;
  std::lock_guard<std::mutex> lock(mu);
  auto it = known.find({fn, smem});
  if (it != known.end()) return it->second;
  int n = 1;
  TN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, 256, smem));
  n = std::max(n, 1);
  known[{fn, smem}] = n;
  return n;
}

int ilog2_exact(int64_t x) {
  int r = 0;
  while ((int64_t(1) << r) < x) ++r;
  TN_CHECK((int64_t(1) << r) == x, TN_ERR_UNSUPPORTED, "extent is not a power of two");
  return r;
}

// group and natural bit of every position bit of a dense tensor decoded by d
// (groups 0..2 with extents ext[]); false when some bit is not covered
bool position_bits_impl(const RunDecode& d, int nbits, const int64_t ext[3], int8_t* grp, int8_t* nat) {
  for (int j = 0; j < nbits; ++j) grp[j] = -1;
  int lg_ext[3];
  for (int g = 0; g < 3; ++g) lg_ext[g] = ilog2_exact(ext[g]);
  for (int e = 0; e < d.n; ++e)
    for (int b = 0; b < d.lg[e]; ++b) {
      const int pos = d.pos[e] + b, q = d.shift[e] + b;
      if (pos >= nbits || q >= lg_ext[d.grp[e]]) break;
      if (grp[pos] >= 0) return false;
      grp[pos] = d.grp[e];
      nat[pos] = (int8_t)q;
    }
  for (int j = 0; j < nbits; ++j)
    if (grp[j] < 0) return false;
  return true;
}

bool fastest_unit(const Runs& r) { return r.n > 0 && r.st[0] == 1; }

template <int TM, int TN, int TK, int TY, int TX, class In, class Out>
void launch_tiled(const GemmParams& p, float scale, bool hilo, cudaStream_t s) {
  int64_t gx = (p.N + TN - 1) / TN, gy = (p.M + TM - 1) / TM;
  TN_CHECK(gx * gy < (1LL << 31), TN_ERR_UNSUPPORTED, "GEMM grid too large");
  unsigned gz = (unsigned)std::min<int64_t>(p.nbt, 65535);
  const int flags = (fastest_unit(p.a_k) || !fastest_unit(p.a_m) ? 1 : 0) | (fastest_unit(p.b_n) ? 2 : 0);
  gemm_tiled<TM, TN, TK, TY, TX, In, Out><<<dim3((unsigned)(gx * gy), 1, gz), 256, 0, s>>>(p, scale, hilo, flags);
}

// The row kernel for a small-K step written in place, when its rows suit it
// (A rows of K contiguous entries, rows written densely): false otherwise.
template <class Out>
bool launch_rows(const GemmParams& g, float scale, cudaStream_t s, bool hilo) {
  if (g.K > 4 || !(g.N == 2 || g.N == 4 || g.N == 8)) return false;
  const int64_t rows = g.nbt * g.M;
  if (rows < 256) return false;
  RowsK p{};
  p.A = (const float2*)g.A;
  p.B = (const float2*)g.B;
  p.C = g.C;
  p.C2 = g.C2;
  p.nbits = ilog2_exact(rows);
  const int lgM = ilog2_exact(g.M);
  if (p.nbits > kMaxBits) return false;
  for (int j = 0; j < p.nbits; ++j) {
    if (j < lgM) {
      const int64_t bit = int64_t(1) << j;
      p.a_w[j] = run_offset(g.a_m, bit);
      p.c_w[j] = run_offset(g.c_m, bit);
      p.b_w[j] = 0;
    } else {
      const int64_t bit = int64_t(1) << (j - lgM);
      p.a_w[j] = run_offset(g.a_bt, bit);
      p.c_w[j] = run_offset(g.c_bt, bit);
      p.b_w[j] = run_offset(g.b_bt, bit);
    }
  }
  for (int k = 0; k < 4; ++k) {
    p.ak[k] = k < g.K ? run_offset(g.a_k, k) : 0;
    p.bk[k] = k < g.K ? run_offset(g.b_k, k) : 0;
  }
  for (int n = 0; n < 8; ++n) {
    p.cn[n] = n < g.N ? run_offset(g.c_n, n) : 0;
    p.bn[n] = n < g.N ? run_offset(g.b_n, n) : 0;
  }
  // a warp's 32 rows: A read as one contiguous span, C written densely
  if (p.a_w[0] != g.K || p.c_w[0] > g.N) return false;
  bool a_vec = g.K >= 2 && (reinterpret_cast<uintptr_t>(g.A) & 15) == 0;
  for (int k = 0; k < g.K && a_vec; ++k) a_vec = p.ak[k] == k;
  for (int j = 0; j < p.nbits && a_vec; ++j) a_vec = p.a_w[j] % 2 == 0;
  p.a_vec = a_vec ? 1 : 0;
  bool b_fixed = true;
  for (int j = 0; j < p.nbits; ++j) b_fixed = b_fixed && p.b_w[j] == 0;
  p.b_fixed = b_fixed ? 1 : 0;
  const size_t pair_bytes = 2 * sizeof(typename Out::T);
  bool pairs = (reinterpret_cast<uintptr_t>(g.C) % pair_bytes) == 0 &&
               (!hilo || (reinterpret_cast<uintptr_t>(g.C2) % pair_bytes) == 0);
  for (int n = 0; n < g.N && pairs; n += 2) pairs = p.cn[n + 1] == p.cn[n] + 1 && p.cn[n] % 2 == 0;
  for (int j = 0; j < p.nbits && pairs; ++j) pairs = p.c_w[j] % 2 == 0;
  p.c_pairs = pairs ? 1 : 0;
  p.scale = scale;
  // every offset is a sum over a subset of these non-negative weights
  {
    int64_t sa = 0, sc = 0, sb = 0, ka = 0, kb = 0, nc = 0, nb = 0;
    for (int j = 0; j < p.nbits; ++j) {
      TN_CHECK(p.a_w[j] >= 0 && p.c_w[j] >= 0 && p.b_w[j] >= 0, TN_ERR_UNSUPPORTED, "negative stride");
      sa += p.a_w[j];
      sc += p.c_w[j];
      sb += p.b_w[j];
    }
    for (int k = 0; k < g.K; ++k) {
      ka = std::max(ka, p.ak[k]);
      kb = std::max(kb, p.bk[k]);
    }
    for (int n = 0; n < g.N; ++n) {
      nc = std::max(nc, p.cn[n]);
      nb = std::max(nb, p.bn[n]);
    }
    TN_CHECK(sa + ka < rows * g.K && sc + nc < rows * g.N && sb + kb + nb < g.nbt * g.K * g.N, TN_ERR_INVALID_ARG,
             "internal: row-kernel index maps exceed their tensors");
  }
  // at most two resident blocks per SM; chunks of up to 1024 rows
  const unsigned blocks = (unsigned)std::min<int64_t>((rows + 511) / 512, 152 * 4);
  auto go = [&](auto kc, auto nc) {
    constexpr int KC = decltype(kc)::value, NC = decltype(nc)::value;
    gemm_rows<Out, KC, NC><<<blocks, 256, 0, s>>>(p, hilo);
  };
  using I1 = std::integral_constant<int, 1>;
  using I2 = std::integral_constant<int, 2>;
  using I4 = std::integral_constant<int, 4>;
  using I8 = std::integral_constant<int, 8>;
  auto by_n = [&](auto kc) {
    if (g.N == 2) go(kc, I2{});
    else if (g.N == 4) go(kc, I4{});
    else go(kc, I8{});
  };
  if (g.K == 1) by_n(I1{});
  else if (g.K == 2) by_n(I2{});
  else by_n(I4{});
  return true;
}

// Small-K launch; `ex` non-null: the result goes to that expanded operand.
template <class Out>
void launch_smallk(const GemmParams& g, float scale, cudaStream_t s, bool hilo, const ExpandedDst* ex) {
  if (!ex && launch_rows<Out>(g, scale, s, hilo)) return;
  SmallK p{};
  p.A = (const float2*)g.A;
  p.B = (const float2*)g.B;
  p.K = (int)g.K;
  p.lgK = ilog2_exact(g.K);
  TN_CHECK(g.K <= 4, TN_ERR_UNSUPPORTED, "small-K kernel needs K <= 4");
  const int64_t total = g.nbt * g.M * g.N;
  p.nbits = ilog2_exact(total);
  TN_CHECK(p.nbits <= kMaxBits, TN_ERR_UNSUPPORTED, "result too large");
  int8_t grp[kMaxBits], nat[kMaxBits];
  const int64_t ext[3] = {g.nbt, g.M, g.N};
  TN_CHECK(position_bits_impl(g.c_dec, p.nbits, ext, grp, nat), TN_ERR_UNSUPPORTED, "result is not dense");
  for (int j = 0; j < p.nbits; ++j) {
    const int64_t bit = int64_t(1) << nat[j];
    p.a_w[j] = grp[j] == 0 ? run_offset(g.a_bt, bit) : grp[j] == 1 ? run_offset(g.a_m, bit) : 0;
    p.b_w[j] = grp[j] == 0 ? run_offset(g.b_bt, bit) : grp[j] == 2 ? run_offset(g.b_n, bit) : 0;
    p.o_w[j] = int64_t(1) << j;
  }
  if (ex) {
    // destination: expanded rows [bt][2N][hp] of the consuming step; this
    // tensor's position bits decoded through that step's index maps
    p.hp = expanded_half_pitch(ex->K);
    TN_CHECK(p.hp == ex->K, TN_ERR_UNSUPPORTED, "expanded destination needs K a multiple of the k tile");
    TN_CHECK(ex->nbt * ex->N * ex->K == total, TN_ERR_INVALID_ARG, "expanded destination size");
    int8_t g2[kMaxBits], n2[kMaxBits];
    const int64_t ext2[3] = {ex->nbt, ex->K, ex->N};
    TN_CHECK(position_bits_impl(decode_of(ex->b_bt, ex->b_k, ex->b_n), p.nbits, ext2, g2, n2), TN_ERR_UNSUPPORTED,
             "expanded destination is not dense");
    for (int j = 0; j < p.nbits; ++j) {
      const int64_t unit = g2[j] == 0 ? 2 * ex->N * p.hp : g2[j] == 1 ? 1 : 2 * p.hp;
      p.o_w[j] = unit << n2[j];
    }
    p.C = ex->Bx;
    p.C2 = ex->Bx_lo;
  } else {
    p.C = g.C;
    p.C2 = g.C2;
  }
  for (int k = 0; k < 4; ++k) {
    p.ak[k] = k < p.K ? run_offset(g.a_k, k) : 0;
    p.bk[k] = k < p.K ? run_offset(g.b_k, k) : 0;
  }
  // every offset the kernel forms is a sum over a subset of these non-negative
  // weights: bound the full sums by the (dense) tensors' sizes
  {
    int64_t sa = 0, sb = 0, so = 0, ka = 0, kb = 0;
    for (int j = 0; j < p.nbits; ++j) {
      TN_CHECK(p.a_w[j] >= 0 && p.b_w[j] >= 0 && p.o_w[j] >= 0, TN_ERR_UNSUPPORTED, "negative stride");
      sa += p.a_w[j];
      sb += p.b_w[j];
      so += p.o_w[j];
    }
    for (int k = 0; k < p.K; ++k) {
      ka = std::max(ka, p.ak[k]);
      kb = std::max(kb, p.bk[k]);
    }
    const int64_t dst = ex ? ex->nbt * 2 * ex->N * p.hp : total;
    TN_CHECK(sa + ka < g.nbt * g.M * g.K && sb + kb < g.nbt * g.K * g.N && so + (ex ? p.hp : 0) < dst,
             TN_ERR_INVALID_ARG, "internal: small-K index maps exceed their tensors");
  }
  // the widest tile whose staged A and B entries fit
  for (p.P = std::min(kSkMaxTileBits, p.nbits); p.P > 0; --p.P) {
    int na = 0, nb = 0;
    for (int j = 0; j < p.P; ++j) {
      na += grp[j] != 2;
      nb += grp[j] != 1;
    }
    if ((p.K << na) <= kSkMaxStage && (p.K << nb) <= kSkMaxStage) break;
  }
  p.na = p.nb = 0;
  for (int j = 0; j < kSkMaxTileBits; ++j) p.a_rank[j] = p.b_rank[j] = -1;
  for (int j = 0; j < p.P; ++j) {
    if (grp[j] != 2) {
      p.a_rank[j] = (int8_t)p.na;
      p.a_wt[p.na++] = p.a_w[j];
    }
    if (grp[j] != 1) {
      p.b_rank[j] = (int8_t)p.nb;
      p.b_wt[p.nb++] = p.b_w[j];
    }
  }
  p.scale = scale;
  const size_t smem = 2 * (size_t)((p.K << p.na) + (p.K << p.nb)) * sizeof(float2);  // double buffer
  const int64_t tiles = int64_t(1) << (p.nbits - p.P);
  // two adjacent outputs per thread when the tile's bit 0 has unit stride in the
  // destination and every other bit an even one (aligned vector stores)
  bool pair = p.P >= 1 && p.o_w[0] == 1 && (!ex || p.hp % 2 == 0);
  for (int j = 1; j < p.nbits && pair; ++j) pair = p.o_w[j] % 2 == 0;
  auto go = [&](auto kc, auto v) {
    constexpr int KC = decltype(kc)::value, V = decltype(v)::value;
    auto kern = ex ? gemm_smallk<Out, 1, KC, V> : gemm_smallk<Out, 0, KC, V>;
    // the double buffer (up to 64 KB) plus the static tables can pass the 48 KB
    // a launch may use without the opt-in
    set_max_dynamic_smem((const void*)kern, (int)(2 * kSkMaxStage * 2 * sizeof(float2)));
    // one wave: as many CTAs as are resident at once (a second, partial wave
    // would leave SMs idle at the end), each walking tiles grid-stride
    const int per_sm = resident_blocks((const void*)kern, smem);
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, (int64_t)152 * std::max(per_sm, 1));
    kern<<<grid, 256, smem, s>>>(p, hilo);
  };
  using I1 = std::integral_constant<int, 1>;
  using I2 = std::integral_constant<int, 2>;
  using I4 = std::integral_constant<int, 4>;
  if (pair) {
    if (p.K == 1) go(I1{}, I2{});
    else if (p.K == 2) go(I2{}, I2{});
    else go(I4{}, I2{});
  } else {
    if (p.K == 1) go(I1{}, I1{});
    else if (p.K == 2) go(I2{}, I1{});
    else go(I4{}, I1{});
  }
}

template <class In, class Out>
void launch_typed(const GemmParams& p, float scale, cudaStream_t s, bool hilo = false) {
  const int64_t outputs = p.nbt * p.M * p.N;
  if constexpr (std::is_same_v<In, C64>) {
    if (p.K <= 4) return launch_smallk<Out>(p, scale, s, hilo, nullptr);
  }
  if (p.K <= 4 || (p.M < 16 && p.N < 16) || outputs * p.K < (1 << 16)) {
    int64_t blocks = std::min<int64_t>((outputs >= kDirectVecMin ? outputs / 4 : outputs) / 256 + 1, 152 * 64);
    if (p.elems_max < (int64_t(1) << 31))
      gemm_direct<In, Out, int32_t><<<(unsigned)blocks, 256, 0, s>>>(p, scale, hilo);
    else
      gemm_direct<In, Out, int64_t><<<(unsigned)blocks, 256, 0, s>>>(p, scale, hilo);
    return;
  }
  if (p.M >= 64 && p.N >= 64)
    launch_tiled<64, 64, 16, 16, 16, In, Out>(p, scale, hilo, s);
  else if (p.M < 32 && p.N >= 128)
    launch_tiled<16, 128, 16, 8, 32, In, Out>(p, scale, hilo, s);
  else if (p.N < 32 && p.M >= 128)
    launch_tiled<128, 16, 16, 32, 8, In, Out>(p, scale, hilo, s);
  else
    launch_tiled<32, 32, 16, 16, 16, In, Out>(p, scale, hilo, s);
}

}  // namespace

void launch_gemm_c64(const GemmParams& p, int accumulate, cudaStream_t s) {
  (void)accumulate;
  if (p.nbt <= 0 || p.M <= 0 || p.N <= 0) return;
  launch_typed<C64, C64>(p, 1.0f, s);
}

// in_kind / out_kind: 0 = fp16 complex, 1 = bf16 complex, 2 = fp32 complex;
// out_hilo: a 16-bit output also stores its rounding residual in p.C2
void launch_gemm_simt(const GemmParams& p, int in_kind, int out_kind, float scale, cudaStream_t s, bool out_hilo,
                      const ExpandedDst* ex) {
  if (p.nbt <= 0 || p.M <= 0 || p.N <= 0) return;
  if (ex) {
    TN_CHECK(in_kind == 2 && p.K <= 4, TN_ERR_UNSUPPORTED, "expanded destination needs a complex64 small-K step");
    if (ex->bf16) return launch_smallk<BF16>(p, scale, s, false, ex);
    return launch_smallk<F16>(p, scale, s, false, ex);
  }
  if (in_kind == 2 && out_kind == 2) return launch_typed<C64, C64>(p, scale, s);
  if (in_kind == 2 && out_kind == 0) return launch_typed<C64, F16>(p, scale, s, out_hilo);
  if (in_kind == 2 && out_kind == 1) return launch_typed<C64, BF16>(p, scale, s, out_hilo);
  fail(TN_ERR_UNSUPPORTED, "GEMM storage combination");
}

bool output_position_bits(const RunDecode& d, int nbits, const int64_t ext[3], int8_t* grp, int8_t* nat) {
  return position_bits_impl(d, nbits, ext, grp, nat);
}

RunDecode decode_of(const Runs& bt, const Runs& m, const Runs& n) {
  RunDecode d{};
  d.n = 0;
  const Runs* gs[3] = {&bt, &m, &n};
  for (int g = 0; g < 3; ++g) {
    int shift = 0;
    for (int r = 0; r < gs[g]->n; ++r) {
      int64_t st = gs[g]->st[r];
      int pos = 0;
      while ((int64_t(1) << pos) < st) ++pos;
      TN_CHECK((int64_t(1) << pos) == st, TN_ERR_UNSUPPORTED, "output stride is not a power of two");
      d.pos[d.n] = (int8_t)pos;
      d.lg[d.n] = gs[g]->lg[r];
      d.grp[d.n] = (int8_t)g;
      d.shift[d.n] = (int8_t)shift;
      shift += gs[g]->lg[r];
      ++d.n;
    }
  }
  return d;
}

// one run covering any extent (the digit mask is wider than every index)
Runs single_run(int64_t extent, int64_t stride) {
  Runs r{};
  r.n = extent > 1 ? 1 : 0;
  r.lg[0] = 62;
  r.st[0] = stride;
  return r;
}

}  // namespace tn
