// Data-movement kernels: bit-permutation transpose, sliced-leaf gather, leaf
// upload, and the FP64 cross-slice accumulation.
//
// Every tensor here has 2^r complex elements (all edge dimensions are powers
// of two), so a change of dimension order is a permutation of the r index
// bits.  These kernels are HBM-bound: each element is read once and written
// once.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "tn_internal.h"

namespace tn {

// ------------------------------------------------------------ bit permute
// A tile is 2^nt elements (nt <= 12): the input's fastest bits (coalesced
// reads) together with the input bits that become the output's fastest bits
// (coalesced writes), staged through shared memory.  The remaining bits index
// the tiles; each CTA walks tiles with a grid stride.  Per-element offsets come
// from two 64-entry tables per direction (low and high 6 bits of the tile
// index), so the inner loops are two shared-memory loads and an add.
namespace {

constexpr int kTileMaxBits = 12;

struct PermTile {
  int nt;                   // tile bits
  int tin[kTileMaxBits];    // input bit position of tile bit i (read order)
  int tpos_w[kTileMaxBits]; // tile bit index of the i-th write-order bit
  int tout_w[kTileMaxBits]; // output bit position of the i-th write-order bit
  int ng;                   // tile-index bits
  int gin[kMaxBits];
  int gout[kMaxBits];
};

__device__ __forceinline__ int pad(int t) { return t + (t >> 6); }

template <class W>
__global__ void __launch_bounds__(256) bit_permute_kernel(const W* __restrict__ in, W* __restrict__ out,
                                                          PermTile pt) {
  __shared__ W tile[(1 << kTileMaxBits) + (1 << kTileMaxBits) / 64];
  __shared__ int64_t in_lo[64], in_hi[64], out_lo[64], out_hi[64];
  __shared__ int t_lo[64], t_hi[64];
  const int tid = threadIdx.x;
  if (tid < 64) {
    int64_t a = 0, b = 0, c = 0, d = 0;
    int e = 0, f = 0;
    for (int i = 0; i < pt.nt; ++i) {
      const int bit_lo = i < 6 ? (tid >> i) & 1 : 0;
      const int bit_hi = i >= 6 ? (tid >> (i - 6)) & 1 : 0;
      a |= (int64_t)bit_lo << pt.tin[i];
      b |= (int64_t)bit_hi << pt.tin[i];
      c |= (int64_t)bit_lo << pt.tout_w[i];
      d |= (int64_t)bit_hi << pt.tout_w[i];
      e |= bit_lo << pt.tpos_w[i];
      f |= bit_hi << pt.tpos_w[i];
    }
    in_lo[tid] = a;
    in_hi[tid] = b;
    out_lo[tid] = c;
    out_hi[tid] = d;
    t_lo[tid] = e;
    t_hi[tid] = f;
  }
  __syncthreads();
  const int n = 1 << pt.nt;
  const int64_t n_tiles = int64_t(1) << pt.ng;
  for (int64_t blk = blockIdx.x; blk < n_tiles; blk += gridDim.x) {
    int64_t base_in = 0, base_out = 0;
    for (int j = 0; j < pt.ng; ++j) {
      const int64_t bit = (blk >> j) & 1;
      base_in |= bit << pt.gin[j];
      base_out |= bit << pt.gout[j];
    }
    // eight loads per thread issued before their shared-memory stores (one
    // round trip for the thread's share of the tile instead of one per element)
    for (int t0 = tid; t0 < n; t0 += 256 * 8) {
      W v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int t = t0 + q * 256;
        if (t < n) v[q] = in[base_in + in_lo[t & 63] + in_hi[t >> 6]];
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int t = t0 + q * 256;
        if (t < n) tile[pad(t)] = v[q];
      }
    }
    __syncthreads();
    for (int u = tid; u < n; u += 256)
      out[base_out + out_lo[u & 63] + out_hi[u >> 6]] = tile[pad(t_lo[u & 63] | t_hi[u >> 6])];
    __syncthreads();
  }
}

template <class W>
__global__ void copy_kernel(const W* __restrict__ in, W* __restrict__ out, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) out[i] = in[i];
}

}  // namespace

void launch_bit_permute(const void* in, void* out, const BitPermute& bp, int elem_bytes, cudaStream_t s) {
  const int R = bp.nbits;
  bool identity = true;
  for (int i = 0; i < R; ++i) identity &= bp.out_bit[i] == i;
  if (identity) {
    int64_t n = int64_t(1) << R;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    if (elem_bytes == 8)
      copy_kernel<uint2><<<blocks, 256, 0, s>>>((const uint2*)in, (uint2*)out, n);
    else
      copy_kernel<uint32_t><<<blocks, 256, 0, s>>>((const uint32_t*)in, (uint32_t*)out, n);
    return;
  }
  const int a = std::min(6, R);
  int in_of_out[kMaxBits];
  for (int i = 0; i < R; ++i) in_of_out[bp.out_bit[i]] = i;
  bool in_tile[kMaxBits] = {};
  PermTile pt{};
  pt.nt = 0;
  for (int i = 0; i < a; ++i) {
    in_tile[i] = true;
    pt.tin[pt.nt++] = i;
  }
  for (int o = 0; o < a; ++o) {
    int i = in_of_out[o];
    if (!in_tile[i]) {
      in_tile[i] = true;
      pt.tin[pt.nt++] = i;
    }
  }
  // widen the tile to 2^12 elements with the next input bits (more work per tile)
  for (int i = a; i < R && pt.nt < kTileMaxBits; ++i)
    if (!in_tile[i]) {
      in_tile[i] = true;
      pt.tin[pt.nt++] = i;
    }
  // write order: tile bits sorted by output position
  int order[kTileMaxBits];
  for (int i = 0; i < pt.nt; ++i) order[i] = i;
  for (int i = 0; i < pt.nt; ++i)
    for (int j = i + 1; j < pt.nt; ++j)
      if (bp.out_bit[pt.tin[order[j]]] < bp.out_bit[pt.tin[order[i]]]) std::swap(order[i], order[j]);
  for (int i = 0; i < pt.nt; ++i) {
    pt.tpos_w[i] = order[i];
    pt.tout_w[i] = bp.out_bit[pt.tin[order[i]]];
  }
  pt.ng = 0;
  for (int i = 0; i < R; ++i)
    if (!in_tile[i]) {
      pt.gin[pt.ng] = i;
      pt.gout[pt.ng] = bp.out_bit[i];
      ++pt.ng;
    }
  const int64_t tiles = int64_t(1) << pt.ng;
  const unsigned blocks = (unsigned)std::min<int64_t>(tiles, 152 * 8);
  if (elem_bytes == 8)
    bit_permute_kernel<uint2><<<blocks, 256, 0, s>>>((const uint2*)in, (uint2*)out, pt);
  else
    bit_permute_kernel<uint32_t><<<blocks, 256, 0, s>>>((const uint32_t*)in, (uint32_t*)out, pt);
}

void launch_bit_permute_c64(const void* in, void* out, const BitPermute& bp, cudaStream_t s) {
  launch_bit_permute(in, out, bp, 8, s);
}

// ------------------------------------------------------------ leaf upload
namespace {
// out_kind: 0 = fp16 complex, 1 = bf16 complex, 2 = fp32 complex; values are
// multiplied by `scale` (a power of two) in FP64 before rounding
__global__ void strided_copy_c128_kernel(const double2* __restrict__ in, void* __restrict__ out,
                                         StridedCopy sc, int64_t n, int out_kind, double scale) {
  int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= n) return;
  int64_t rem = o, off = 0;
  for (int d = sc.nd - 1; d >= 0; --d) {
    int64_t c = rem % sc.dims[d];
    rem /= sc.dims[d];
    off += c * sc.in_stride[d];
  }
  double2 v = in[off];
  const double re = v.x * scale, im = v.y * scale;
  if (out_kind == 2)
    ((float2*)out)[o] = make_float2((float)re, (float)im);
  else if (out_kind == 1)
    ((__nv_bfloat162*)out)[o] = __nv_bfloat162(__double2bfloat16(re), __double2bfloat16(im));
  else
    ((__half2*)out)[o] = __halves2half2(__double2half(re), __double2half(im));
}
}  // namespace

void launch_strided_copy_c128(const void* in, void* out, const StridedCopy& sc, int64_t n_out, int out_kind,
                              double scale, cudaStream_t s) {
  if (n_out <= 0) return;
  int64_t blocks = (n_out + 255) / 256;
  strided_copy_c128_kernel<<<(unsigned)blocks, 256, 0, s>>>((const double2*)in, out, sc, n_out, out_kind, scale);
}

void launch_strided_copy_c128_to_c64(const void* in, void* out, const StridedCopy& sc, int64_t n_out,
                                     cudaStream_t s) {
  launch_strided_copy_c128(in, out, sc, n_out, 2, 1.0, s);
}

// ------------------------------------------------------------ slice gather
namespace {
template <class W>
__global__ void gather_kernel(const GatherLeaf* __restrict__ tab, const int64_t* __restrict__ ids, int B,
                              const char* __restrict__ pbase, char* __restrict__ wbase) {
  const GatherLeaf& g = tab[blockIdx.y];
  const int64_t total = g.rest * B;
  const W* src = (const W*)(pbase + g.src_off);
  W* dst = (W*)(wbase + g.dst_off);
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
       x += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = x / g.rest, r = x % g.rest;
    int64_t sid = ids[b];
    int64_t sel = 0;
    for (int i = 0; i < g.n_sel; ++i) sel += ((sid >> g.slice_bit[i]) & 1) * g.sel_stride[i];
    int64_t o = (r / g.inner) * B * g.inner + b * g.inner + r % g.inner;
    dst[o] = src[sel + r];
  }
}
}  // namespace

void launch_gather_leaves(const GatherLeaf* d_table, int n_leaves, int64_t max_rest,
                          const int64_t* d_slice_ids, int B, const char* plan_base, char* ws_base,
                          cudaStream_t s, int elem_bytes) {
  if (n_leaves == 0) return;
  int64_t per = max_rest * B;
  unsigned bx = (unsigned)std::min<int64_t>((per + 255) / 256, 64);
  TN_CHECK(n_leaves <= 65535, TN_ERR_UNSUPPORTED, "too many sliced leaves");
  if (elem_bytes == 8)
    gather_kernel<uint2><<<dim3(bx, n_leaves), 256, 0, s>>>(d_table, d_slice_ids, B, plan_base, ws_base);
  else
    gather_kernel<uint32_t><<<dim3(bx, n_leaves), 256, 0, s>>>(d_table, d_slice_ids, B, plan_base, ws_base);
}

// ------------------------------------------------------------ accumulate
// amps[g][j] = (accumulate ? amps[g][j] : 0) + sum_{b < n_valid} root[b][g][j]
// in FP64 (the cross-slice sum of paper Sec. III slicing), in a fixed order:
// four threads per output each sum a contiguous quarter of the batch in batch
// order, then the four partial sums are added in quarter order.  (GB300's
// FP64 rate is low; four threads per output hide the latency of the add chains.)
namespace {
constexpr int kAccParts = 4;
constexpr int kAccOut = 64;  // outputs per 256-thread block
__global__ void __launch_bounds__(kAccParts * kAccOut)
    accumulate_kernel(const float2* __restrict__ root, int64_t sb, int64_t sg, int64_t sj, int64_t G, int64_t J,
                      const int32_t* __restrict__ n_valid, double2* __restrict__ amps, int accumulate,
                      double scale) {
  __shared__ double2 part[kAccParts][kAccOut];
  const int q = threadIdx.x / kAccOut, o = threadIdx.x % kAccOut;  // a warp: one quarter, 32 outputs
  const int64_t x = blockIdx.x * (int64_t)kAccOut + o;
  const int nv = *n_valid;
  double re = 0.0, im = 0.0;
  if (x < G * J) {
    const int64_t g = x / J, j = x % J;
    const float2* p = root + g * sg + j * sj;
    const int b1 = (int)((int64_t)nv * (q + 1) / kAccParts);
    int b = (int)((int64_t)nv * q / kAccParts);
    // loads issued eight at a time (independent), summed in batch order
    for (; b + 8 <= b1; b += 8) {
      float2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = p[(b + u) * sb];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        re += (double)v[u].x;
        im += (double)v[u].y;
      }
    }
    for (; b < b1; ++b) {
      const float2 v = p[b * sb];
      re += (double)v.x;
      im += (double)v.y;
    }
  }
  part[q][o] = make_double2(re, im);
  __syncthreads();
  if (q != 0 || x >= G * J) return;
  re = part[0][o].x;
  im = part[0][o].y;
#pragma unroll
  for (int r = 1; r < kAccParts; ++r) {
    re += part[r][o].x;
    im += part[r][o].y;
  }
  re *= scale;  // power of two: exact
  im *= scale;
  if (accumulate) {
    double2 a = amps[x];
    re = a.x + re;
    im = a.y + im;
  }
  amps[x] = make_double2(re, im);
}
__global__ void zero_kernel(uint4* p, int64_t n16) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = make_uint4(0, 0, 0, 0);
}
}  // namespace

void launch_accumulate_c64(const void* root, int64_t sb, int64_t sg, int64_t sj, int64_t G, int64_t J,
                           const int32_t* d_n_valid, int B, void* amps, int accumulate, cudaStream_t s,
                           double scale) {
  (void)B;
  int64_t n = G * J;
  accumulate_kernel<<<(unsigned)((n + kAccOut - 1) / kAccOut), kAccParts * kAccOut, 0, s>>>(
      (const float2*)root, sb, sg, sj, G, J, d_n_valid, (double2*)amps, accumulate, scale);
}

// ------------------------------------------------------------ amax
// out[slot] = max(out[slot], max |re|, |im| over a complex64 tensor)  (calibration)
namespace {
__global__ void amax_kernel(const float2* __restrict__ x, int64_t n, unsigned* out) {
  float m = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fmaxf(fabsf(x[i].x), fabsf(x[i].y)));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}
}  // namespace

void launch_amax_c64(const void* x, int64_t n, unsigned* out, cudaStream_t s) {
  if (n <= 0) return;
  unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8);
  amax_kernel<<<blocks, 256, 0, s>>>((const float2*)x, n, out);
}

void launch_zero(void* p, size_t bytes, cudaStream_t s) {
  // bytes is a multiple of 16 (complex128 buffers)
  int64_t n16 = (int64_t)(bytes / 16);
  if (n16 == 0) return;
  unsigned blocks = (unsigned)std::min<int64_t>((n16 + 255) / 256, 4096);
  zero_kernel<<<blocks, 256, 0, s>>>((uint4*)p, n16);
}

// ------------------------------------------------------------ slice ids
// Slice ids of one batch travel as kernel parameters (no host staging copy,
// no stream synchronisation): each launch writes up to kIdsPerLaunch ids.
namespace {
constexpr int kIdsPerLaunch = 256;
struct SliceIdChunk {
  int64_t ids[kIdsPerLaunch];
  int32_t count, n_valid, write_n_valid;
};
__global__ void set_ids_kernel(int64_t* dst, int32_t* n_valid, SliceIdChunk c) {
  if ((int)threadIdx.x < c.count) dst[threadIdx.x] = c.ids[threadIdx.x];
  if (threadIdx.x == 0 && c.write_n_valid) *n_valid = c.n_valid;
}
}  // namespace

void launch_set_slice_ids(int64_t* d_ids, int32_t* d_n_valid, const int64_t* ids, int B, int32_t n_valid,
                          cudaStream_t s) {
  for (int off = 0; off < B; off += kIdsPerLaunch) {
    SliceIdChunk c{};
    c.count = std::min(kIdsPerLaunch, B - off);
    for (int i = 0; i < c.count; ++i) c.ids[i] = ids[off + i];
    c.n_valid = n_valid;
    c.write_n_valid = off == 0 ? 1 : 0;
    set_ids_kernel<<<1, kIdsPerLaunch, 0, s>>>(d_ids + off, d_n_valid, c);
  }
}

}  // namespace tn
