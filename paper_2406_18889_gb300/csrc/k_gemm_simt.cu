// Complex strided batched GEMM on CUDA cores: the plain complex64 path, and
// the small steps of the reduced-precision path (fp16/bf16 complex storage,
// FP32 arithmetic).
//
// One pairwise contraction of the tree (arXiv 2406.18889, Sec. III: the
// per-step tensor contraction the paper runs through cuTensor or
// transpose-transpose-GEMM-transpose) is C[bt][m][n] = sum_k A[bt][m][k] *
// B[bt][k][n] once the plan has put each operand's batch, free and contracted
// indices into contiguous blocks.  Each complex multiply-add is four FP32
// fused multiply-adds.
//
// Two kernels:
//  * tiled: a CTA of 256 threads computes a TM x TN tile, staging TK-deep
//    slices of A and B through shared memory (loads coalesced along whichever
//    of the operand's two indices is contiguous); each thread keeps RM x RN
//    complex accumulators.
//  * direct: one thread per output element, for shapes too small for a tile.
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

template <int TM, int TN, int TK, int TY, int TX, class In, class Out>
__global__ void __launch_bounds__(256) gemm_tiled(GemmParams p, float scale, bool hilo) {
  static_assert(TY * TX == 256, "256 threads");
  constexpr int RM = TM / TY, RN = TN / TX;
  __shared__ float2 As[TK][TM + 1];
  __shared__ float2 Bs[TK][TN + 1];
  using TI = typename In::T;
  using TO = typename Out::T;
  const TI* __restrict__ A = (const TI*)p.A;
  const TI* __restrict__ Bm = (const TI*)p.B;
  TO* __restrict__ C = (TO*)p.C;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int64_t m0 = (int64_t)blockIdx.y * TM, n0 = (int64_t)blockIdx.x * TN;
  const bool a_kc = p.sa_k == 1;  // A contiguous along k
  const bool b_nc = p.sb_n == 1;  // B contiguous along n
  for (int64_t bt = blockIdx.z; bt < p.nbt; bt += gridDim.z) {
    const TI* Ab = A + bt * p.sa_bt;
    const TI* Bb = Bm + bt * p.sb_bt;
    float2 acc[RM][RN];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
      for (int j = 0; j < RN; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int64_t k0 = 0; k0 < p.K; k0 += TK) {
      // stage A[m0 : m0+TM][k0 : k0+TK]
#pragma unroll
      for (int l = tid; l < TM * TK; l += 256) {
        int mm, kk;
        if (a_kc) {
          mm = l / TK;
          kk = l % TK;
        } else {
          kk = l / TM;
          mm = l % TM;
        }
        int64_t gm = m0 + mm, gk = k0 + kk;
        float2 v = make_float2(0.f, 0.f);
        if (gm < p.M && gk < p.K) v = In::ld(Ab[gm * p.sa_m + gk * p.sa_k]);
        As[kk][mm] = v;
      }
      // stage B[k0 : k0+TK][n0 : n0+TN]
#pragma unroll
      for (int l = tid; l < TN * TK; l += 256) {
        int nn, kk;
        if (b_nc) {
          kk = l / TN;
          nn = l % TN;
        } else {
          nn = l / TK;
          kk = l % TK;
        }
        int64_t gn = n0 + nn, gk = k0 + kk;
        float2 v = make_float2(0.f, 0.f);
        if (gn < p.N && gk < p.K) v = In::ld(Bb[gk * p.sb_k + gn * p.sb_n]);
        Bs[kk][nn] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < TK; ++kk) {
        float2 a[RM], b[RN];
#pragma unroll
        for (int i = 0; i < RM; ++i) a[i] = As[kk][ty + i * TY];
#pragma unroll
        for (int j = 0; j < RN; ++j) b[j] = Bs[kk][tx + j * TX];
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
          for (int j = 0; j < RN; ++j) cmac(acc[i][j], a[i], b[j]);
      }
      __syncthreads();
    }
    TO* Cb = C + bt * p.sc_bt;
#pragma unroll
    for (int i = 0; i < RM; ++i) {
      int64_t gm = m0 + ty + i * TY;
      if (gm >= p.M) continue;
#pragma unroll
      for (int j = 0; j < RN; ++j) {
        int64_t gn = n0 + tx + j * TX;
        if (gn < p.N)
          store_out<Out>(Cb, (TO*)p.C2 + bt * p.sc_bt, gm * p.sc_m + gn * p.sc_n,
                         make_float2(acc[i][j].x * scale, acc[i][j].y * scale), hilo);
      }
    }
  }
}

// one thread per output element (bt, m, n), n fastest
template <class In, class Out>
__global__ void __launch_bounds__(256) gemm_direct(GemmParams p, float scale, bool hilo) {
  using TI = typename In::T;
  using TO = typename Out::T;
  const TI* __restrict__ A = (const TI*)p.A;
  const TI* __restrict__ Bm = (const TI*)p.B;
  TO* __restrict__ C = (TO*)p.C;
  const int64_t total = p.nbt * p.M * p.N;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
       x += (int64_t)gridDim.x * blockDim.x) {
    int64_t n = x % p.N;
    int64_t t = x / p.N;
    int64_t m = t % p.M;
    int64_t bt = t / p.M;
    const TI* a = A + bt * p.sa_bt + m * p.sa_m;
    const TI* b = Bm + bt * p.sb_bt + n * p.sb_n;
    float2 acc = make_float2(0.f, 0.f);
    for (int64_t k = 0; k < p.K; ++k) cmac(acc, In::ld(a[k * p.sa_k]), In::ld(b[k * p.sb_k]));
    store_out<Out>(C, (TO*)p.C2, bt * p.sc_bt + m * p.sc_m + n * p.sc_n,
                   make_float2(acc.x * scale, acc.y * scale), hilo);
  }
}

template <int TM, int TN, int TK, int TY, int TX, class In, class Out>
void launch_tiled(const GemmParams& p, float scale, bool hilo, cudaStream_t s) {
  int64_t gx = (p.N + TN - 1) / TN, gy = (p.M + TM - 1) / TM;
  TN_CHECK(gx < (1LL << 31) && gy < 65536, TN_ERR_UNSUPPORTED, "GEMM grid too large");
  unsigned gz = (unsigned)std::min<int64_t>(p.nbt, 65535);
  gemm_tiled<TM, TN, TK, TY, TX, In, Out><<<dim3((unsigned)gx, (unsigned)gy, gz), 256, 0, s>>>(p, scale, hilo);
}

template <class In, class Out>
void launch_typed(const GemmParams& p, float scale, cudaStream_t s, bool hilo = false) {
  const int64_t outputs = p.nbt * p.M * p.N;
  if (p.K <= 4 || (p.M < 16 && p.N < 16) || outputs * p.K < (1 << 16)) {
    int64_t blocks = std::min<int64_t>((outputs + 255) / 256, 152 * 64);
    gemm_direct<In, Out><<<(unsigned)blocks, 256, 0, s>>>(p, scale, hilo);
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
void launch_gemm_simt(const GemmParams& p, int in_kind, int out_kind, float scale, cudaStream_t s, bool out_hilo) {
  if (p.nbt <= 0 || p.M <= 0 || p.N <= 0) return;
  if (in_kind == 2 && out_kind == 2) return launch_typed<C64, C64>(p, scale, s);
  if (in_kind == 2 && out_kind == 0) return launch_typed<C64, F16>(p, scale, s, out_hilo);
  if (in_kind == 2 && out_kind == 1) return launch_typed<C64, BF16>(p, scale, s, out_hilo);
  if (in_kind == 0 && out_kind == 0) return launch_typed<F16, F16>(p, scale, s, out_hilo);
  if (in_kind == 0 && out_kind == 2) return launch_typed<F16, C64>(p, scale, s);
  if (in_kind == 1 && out_kind == 1) return launch_typed<BF16, BF16>(p, scale, s, out_hilo);
  if (in_kind == 1 && out_kind == 2) return launch_typed<BF16, C64>(p, scale, s);
  fail(TN_ERR_UNSUPPORTED, "GEMM storage combination");
}

}  // namespace tn
