// Small per-batch steps in one launch.
//
// Near the sliced leaves the contraction tree has many pairwise steps whose
// results hold only a few thousand elements (arXiv 2406.18889, Sec. III: the
// per-step contractions of the sliced sub-network); launched one by one, each
// costs a kernel launch and a prologue for microseconds of work.  Here every
// maximal subtree of such steps is executed by ONE CTA, step after step
// (topological order), with a block barrier between steps; distinct subtrees
// run on distinct CTAs of the same launch.  Each step is the same
// strided-gather complex GEMM as the CUDA-core kernels, C[x] = scale *
// sum_k A[a(x) + ak[k]] * B[b(x) + bk[k]] over C's memory order x, where the
// operand offsets a(x), b(x) are linear over the bits of x: two 128-entry
// tables (bits 0..6 and 7..13) give them per output.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>
#include <set>

#include "tn_internal.h"

namespace tn {
namespace {

__device__ __forceinline__ void cmac_m(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

template <class T2>
__device__ __forceinline__ void store16(char* C, char* C2, int x, float2 v, bool hilo);
template <>
__device__ __forceinline__ void store16<__half2>(char* C, char* C2, int x, float2 v, bool hilo) {
  const __half2 h = __floats2half2_rn(v.x, v.y);
  reinterpret_cast<__half2*>(C)[x] = h;
  if (hilo) {
    const float2 f = __half22float2(h);
    reinterpret_cast<__half2*>(C2)[x] = __floats2half2_rn(v.x - f.x, v.y - f.y);
  }
}
template <>
__device__ __forceinline__ void store16<__nv_bfloat162>(char* C, char* C2, int x, float2 v, bool hilo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
  reinterpret_cast<__nv_bfloat162*>(C)[x] = h;
  if (hilo) {
    const float2 f = __bfloat1622float2(h);
    reinterpret_cast<__nv_bfloat162*>(C2)[x] = __floats2bfloat162_rn(v.x - f.x, v.y - f.y);
  }
}

constexpr int kMicroThreads = 512;

__global__ void __launch_bounds__(kMicroThreads) micro_kernel(const MicroStep* __restrict__ steps,
                                                              const MicroGroup* __restrict__ groups,
                                                              const MicroLoad* __restrict__ loads,
                                                              const char* plan_base, char* ws_base) {
  extern __shared__ __align__(16) char sm[];  // [descriptors | operands and inner results]
  __shared__ int2 tab[256];  // [0, 128): output bits 0..6; [128, 256): bits 7..13
  const MicroGroup G = groups[blockIdx.x];
  const MicroStep* ds = steps + G.first_step;
  // one round of loads before the first step: the group's descriptors and the
  // operands it reads from outside (gate tensors, gathered leaves); inner
  // results then stay in shared memory, so a step costs no global round trip
  if (G.desc_in_smem) {
    const int4* src = reinterpret_cast<const int4*>(ds);
    int4* dst = reinterpret_cast<int4*>(sm);
    const int n16 = G.n_steps * (int)(sizeof(MicroStep) / 16);
    for (int i = threadIdx.x; i < n16; i += kMicroThreads) dst[i] = src[i];
    ds = reinterpret_cast<const MicroStep*>(sm);
  }
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int l = G.first_load + warp; l < G.first_load + G.n_loads; l += kMicroThreads / 32) {
      const MicroLoad L = loads[l];
      const float2* src = reinterpret_cast<const float2*>((L.src_loc ? ws_base : plan_base) + L.src_off);
      float2* dst = reinterpret_cast<float2*>(sm + L.smem_off);
      for (int i = lane; i < L.elems; i += 32) dst[i] = src[i];
    }
  }
  __syncthreads();
  for (int s = 0; s < G.n_steps; ++s) {
    const MicroStep& d = ds[s];
    const int nb = d.nbits;
    for (int j = threadIdx.x; j < 256; j += blockDim.x) {
      const int lo = j < 128 ? 0 : 7, idx = j & 127;
      int a = 0, b = 0;
      for (int q = 0; q < 7; ++q)
        if (((idx >> q) & 1) && lo + q < nb) {
          a += d.a_w[lo + q];
          b += d.b_w[lo + q];
        }
      tab[j] = make_int2(a, b);
    }
    __syncthreads();
    auto base = [&](int loc) -> const char* { return loc == 2 ? sm : loc == 1 ? ws_base : plan_base; };
    const float2* A = reinterpret_cast<const float2*>(base(d.a_loc) + d.a_off);
    const float2* B = reinterpret_cast<const float2*>(base(d.b_loc) + d.b_off);
    char* C = (d.c_loc == 2 ? sm : ws_base) + d.c_off;
    char* C2 = ws_base + d.c2_off;
    const int K = d.K, total = 1 << nb, kind = d.out_kind;
    const bool hilo = d.out_hilo != 0;
    const float scale = d.scale;
    int ak[4], bk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ak[k] = d.ak[k];
      bk[k] = d.bk[k];
    }
    // kU outputs per thread per pass, all of their operand loads issued before
    // any arithmetic: a step is a few dependent memory round trips, not one
    // per output
    constexpr int kU = 4;
    for (int x0 = threadIdx.x; x0 < total; x0 += kU * kMicroThreads) {
      float2 av[kU][4], bv[kU][4];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int x = x0 + u * kMicroThreads;
        const int xs = x < total ? x : 0;
        const int2 l = tab[xs & 127], h = tab[128 + (xs >> 7)];
        const int ao = l.x + h.x, bo = l.y + h.y;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const bool on = k < K && x < total;
          av[u][k] = on ? A[ao + ak[k]] : make_float2(0.f, 0.f);
          bv[u][k] = on ? B[bo + bk[k]] : make_float2(0.f, 0.f);
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int x = x0 + u * kMicroThreads;
        if (x >= total) break;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (k < K) cmac_m(acc, av[u][k], bv[u][k]);
        acc.x *= scale;
        acc.y *= scale;
        if (kind == 2)
          reinterpret_cast<float2*>(C)[x] = acc;
        else if (kind == 0)
          store16<__half2>(C, C2, x, acc, hilo);
        else
          store16<__nv_bfloat162>(C, C2, x, acc, hilo);
      }
    }
    __syncthreads();  // this step's results are visible to the group's next step
  }
}

}  // namespace

void fill_micro_weights(const GemmParams& g, MicroStep& d) {
  const int64_t total = g.nbt * g.M * g.N;
  int nbits = 0;
  while ((int64_t(1) << nbits) < total) ++nbits;
  TN_CHECK((int64_t(1) << nbits) == total && nbits <= kMicroMaxBits, TN_ERR_INVALID_ARG,
           "internal: micro step output size");
  TN_CHECK(g.K >= 1 && g.K <= 4, TN_ERR_INVALID_ARG, "internal: micro step K");
  int8_t grp[kMaxBits], nat[kMaxBits];
  const int64_t ext[3] = {g.nbt, g.M, g.N};
  TN_CHECK(output_position_bits(g.c_dec, nbits, ext, grp, nat), TN_ERR_INVALID_ARG,
           "internal: micro step result is not dense");
  int64_t sa = 0, sb = 0, ka = 0, kb = 0;
  for (int j = 0; j < kMicroMaxBits; ++j) d.a_w[j] = d.b_w[j] = 0;
  for (int j = 0; j < nbits; ++j) {
    const int64_t bit = int64_t(1) << nat[j];
    const int64_t a = grp[j] == 0 ? run_offset(g.a_bt, bit) : grp[j] == 1 ? run_offset(g.a_m, bit) : 0;
    const int64_t b = grp[j] == 0 ? run_offset(g.b_bt, bit) : grp[j] == 2 ? run_offset(g.b_n, bit) : 0;
    sa += a;
    sb += b;
    d.a_w[j] = (int32_t)a;
    d.b_w[j] = (int32_t)b;
  }
  for (int k = 0; k < 4; ++k) {
    d.ak[k] = k < g.K ? (int32_t)run_offset(g.a_k, k) : 0;
    d.bk[k] = k < g.K ? (int32_t)run_offset(g.b_k, k) : 0;
    ka = std::max<int64_t>(ka, d.ak[k]);
    kb = std::max<int64_t>(kb, d.bk[k]);
  }
  // every offset formed is a sum over a subset of these non-negative weights
  TN_CHECK(sa + ka < g.nbt * g.M * g.K && sb + kb < g.nbt * g.K * g.N && sa + ka < (int64_t(1) << 31) &&
               sb + kb < (int64_t(1) << 31),
           TN_ERR_INVALID_ARG, "internal: micro step index maps exceed their tensors");
  d.nbits = (int8_t)nbits;
  d.K = (int8_t)g.K;
}

void launch_micro(const MicroStep* d_steps, const MicroGroup* d_groups, const MicroLoad* d_loads, int n_groups,
                  int smem_bytes, const char* plan_base, char* ws_base, cudaStream_t s) {
  if (n_groups <= 0) return;
  TN_CHECK(smem_bytes >= 0 && smem_bytes <= kMicroSmemBytes, TN_ERR_INVALID_ARG, "internal: fused launch smem");
  {
    // dynamic shared memory above 48 KB: opted in once per device
    static std::mutex mu;
    static std::set<int> done;
    int dev = 0;
    TN_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (!done.count(dev)) {
      TN_CUDA(cudaFuncSetAttribute((const void*)micro_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kMicroSmemBytes));
      done.insert(dev);
    }
  }
  micro_kernel<<<(unsigned)n_groups, kMicroThreads, (size_t)smem_bytes, s>>>(d_steps, d_groups, d_loads, plan_base,
                                                                              ws_base);
}

}  // namespace tn
