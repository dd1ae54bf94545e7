// Tensor-core GEMM, host side: tensor maps, shape checks and dispatch to the
// per-tile-width kernels (tc_kernel.cuh, instantiated in k_gemm_tc_bn*.cu);
// the expansion of the B operand into its real 2x2 form; and a self-test
// against a plain FP32 complex GEMM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "tc_kernel.cuh"

namespace tn {

extern template void launch_tc_tiles<32>(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&,
                                         const CUtensorMap&, const TcGemmParams&, bool, bool, cudaStream_t);
extern template void launch_tc_tiles<64>(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&,
                                         const CUtensorMap&, const TcGemmParams&, bool, bool, cudaStream_t);
extern template void launch_tc_tiles<128>(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&,
                                          const CUtensorMap&, const TcGemmParams&, bool, bool, cudaStream_t);
extern template void launch_tc_tiles<256>(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&,
                                          const CUtensorMap&, const TcGemmParams&, bool, bool, cudaStream_t);

namespace {

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
  // a 16-bit output has the operands' type (with its residual when out_hilo)
  TN_CHECK(p.out_kind == 2 || p.out_kind == (bf16 ? 1 : 0), TN_ERR_UNSUPPORTED,
           "tensor-core output storage must match the operand precision");
  TN_CHECK((p.out_hilo != 0) == (p.C2 != nullptr) && !(p.out_hilo && p.out_kind == 2), TN_ERR_UNSUPPORTED,
           "tensor-core output residual: C2 exactly for a split 16-bit output");
  const int bn = p.bn;
  TN_CHECK(p.acc_split >= 0, TN_ERR_UNSUPPORTED, "negative accumulation chunk");
  TN_CHECK(p.m_halves == 0 || p.m_halves == 1 || (p.m_halves == 2 && bn == 256 && !p.acc_split),
           TN_ERR_UNSUPPORTED, "256-row tiles: tile width 256, one accumulator per tile");
  {
    // stage the epilogue when n is the output's more contiguous index
    const int64_t big = int64_t(1) << 62;
    const int64_t sn = p.c_n.n > 0 ? p.c_n.st[0] : big, sm = p.c_m.n > 0 ? p.c_m.st[0] : big;
    // only for write-heavy tiles (up to four k tiles); deeper tiles hide the per-row stores
    p.stage_n = (sn < sm && 2 * p.K <= 4 * BK && p.m_halves != 2) ? 1 : 0;
    // 16-byte stores along n instead: n's first run has unit stride and holds
    // whole groups of VN outputs, and every other stride keeps groups 16-byte
    // aligned.  Rows one group apart: each lane stores its own row (a warp's
    // 32 rows write one span of 512 bytes per store).  Rows further apart:
    // the pieces go through shared memory and L lanes store L consecutive
    // pieces of one row (L = the pieces in n's first run, at most a chunk
    // row's 16 / VN), so that every store fills whole 32-byte sectors.
    const int64_t VN = p.out_kind == 2 ? 2 : 4, ES = p.out_kind == 2 ? 8 : 4;
    bool vec = p.c_n.n > 0 && p.c_n.st[0] == 1 && (int64_t(1) << p.c_n.lg[0]) % VN == 0 && p.acc_split == 0;
    for (const Runs* R : {&p.c_n, &p.c_m, &p.c_bt})
      for (int r = (R == &p.c_n ? 1 : 0); r < R->n && vec; ++r) vec = R->st[r] % VN == 0;
    vec = vec && (reinterpret_cast<uintptr_t>(p.C) & 15) == 0 &&
          (!p.out_hilo || (reinterpret_cast<uintptr_t>(p.C2) & 15) == 0);
    // (staging shortens the operand ring: write-heavy tiles only, as above)
    p.vec = 0;
    p.vec_staged = 0;
    p.vec_lpr_lg = 0;
    const int64_t pieces = vec ? std::min<int64_t>((int64_t(1) << p.c_n.lg[0]) / VN, 16 / VN) : 0;
    if (vec && sm * ES <= 16) {
      p.vec = 1;
      p.stage_n = 0;
    } else if (vec && pieces >= 2 && p.m_halves != 2 && 2 * p.K <= 4 * BK) {
      int lg = 0;
      while ((int64_t(2) << lg) <= pieces) ++lg;
      p.vec = 1;
      p.vec_staged = 1;
      p.vec_lpr_lg = lg;
      p.stage_n = 1;
    } else if (vec && sm * ES <= 32) {
      p.vec = 1;  // two stores fill each 32-byte span
      p.stage_n = 0;
    }
  }
  const int64_t tbm = (p.m_halves == 2 ? 2 : 1) * (int64_t)BM;  // rows per tile
  TN_CHECK(p.nbt * ((p.M + tbm - 1) / tbm) * ((2 * p.N + bn - 1) / bn) < (int64_t(1) << 31) &&
               p.nbt < (int64_t(1) << 31) && p.M < (int64_t(1) << 31) && p.N < (int64_t(1) << 31),
           TN_ERR_UNSUPPORTED, "tensor-core GEMM: tile count or an extent reaches 2^31");
  {
    // offsets inside a tile are at most those of its all-ones row and column indices
    const int64_t local_max = run_offset(p.c_m, tbm - 1) + run_offset(p.c_n, bn / 2 - 1);
    p.off32 = local_max < (int64_t(1) << 31) ? 1 : 0;
  }
  const uint64_t pitch = (uint64_t)((2 * p.K + BK - 1) / BK * BK);
  CUtensorMap ma, ma2, mb, mb2;
  const uint64_t a_row = (uint64_t)sa_m * 4, a_bt = p.nbt > 1 ? (uint64_t)sa_bt * 4 : a_row * (uint64_t)p.M;
  make_map(&ma, A, bf16, (uint64_t)(2 * p.K), (uint64_t)p.M, (uint64_t)p.nbt, a_row, (a_bt + 15) / 16 * 16, BM);
  const uint32_t b_box = (uint32_t)bn;
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
  switch (bn) {
    case 32:
      launch_tc_tiles<32>(ma, ma2, mb, mb2, p, bf16, hilo, s);
      break;
    case 64:
      launch_tc_tiles<64>(ma, ma2, mb, mb2, p, bf16, hilo, s);
      break;
    case 128:
      launch_tc_tiles<128>(ma, ma2, mb, mb2, p, bf16, hilo, s);
      break;
    case 256:
      launch_tc_tiles<256>(ma, ma2, mb, mb2, p, bf16, hilo, s);
      break;
    default:
      fail(TN_ERR_UNSUPPORTED, "bad tensor-core tile");
  }
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
// pair = 1: the block-diagonal operand of a row-paired step, [[B, 0], [0, B]]
// (N, K are twice B's extents; entry (k', n') is B[k' mod K/2][n' mod N/2]
// when k' and n' fall in the same half, else 0)
// Four consecutive k per thread (half_pitch is a multiple of 32), so each of
// the two rows gets one 16-byte store.  P2: half_pitch, N and K are powers of
// two (lg.x, lg.y their logs), so the index splits are shifts and masks.
template <class T2>
struct alignas(16) Quad {
  T2 v[4];
};

template <class T2, class T, class TIN, class I, bool P2>
__global__ void expand_b_kernel(const TIN* __restrict__ B, Runs b_bt, Runs b_k, Runs b_n, int64_t nbt, int64_t N,
                                int64_t K, int64_t half_pitch, T2* __restrict__ Bx, T2* __restrict__ Bx_lo,
                                float bscale, int pair, int4 lg) {
  const I hq = (I)(half_pitch >> 2), NN = (I)N, KK = (I)K;
  const I total = (I)nbt * NN * hq;
  const I Nh = NN >> pair, Kh = KK >> pair;  // B's own extents
  for (I x = blockIdx.x * (I)blockDim.x + threadIdx.x; x < total; x += (I)gridDim.x * blockDim.x) {
    const I k0 = (P2 ? (x & (hq - 1)) : x % hq) << 2;
    const I t = P2 ? (x >> (lg.x - 2)) : x / hq;
    const I n = P2 ? (t & (NN - 1)) : t % NN, bt = P2 ? (t >> lg.y) : t / NN;
    const I ns = !pair ? n : P2 ? (n & (Nh - 1)) : n % Nh;
    const I base = run_off_i<I>(b_bt, bt) + run_off_i<I>(b_n, ns);
    Quad<T2> h0, h1, l0, l1;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const I k = k0 + j;
      float re = 0.f, im = 0.f;
      if (k < KK && (!pair || (n >= Nh) == (k >= Kh))) {
        const I ks = !pair ? k : P2 ? (k & (Kh - 1)) : k % Kh;
        const TIN v = B[base + run_off_i<I>(b_k, ks)];
        re = (float)v.x * bscale;  // power of two: exact unless out of range
        im = (float)v.y * bscale;
      }
      const T hre = T(re), him = T(im);
      h0.v[j].x = hre;
      h0.v[j].y = neg16<T>(him);
      h1.v[j].x = him;
      h1.v[j].y = hre;
      const T lre = T(re - (float)hre), lim = T(im - (float)him);
      l0.v[j].x = lre;
      l0.v[j].y = neg16<T>(lim);
      l1.v[j].x = lim;
      l1.v[j].y = lre;
    }
    const int64_t row0 = ((int64_t)bt * 2 * N + 2 * (int64_t)n) * half_pitch + k0;
    *reinterpret_cast<Quad<T2>*>(Bx + row0) = h0;
    *reinterpret_cast<Quad<T2>*>(Bx + row0 + half_pitch) = h1;
    if (Bx_lo) {
      *reinterpret_cast<Quad<T2>*>(Bx_lo + row0) = l0;
      *reinterpret_cast<Quad<T2>*>(Bx_lo + row0 + half_pitch) = l1;
    }
  }
}

template <class I, bool P2>
void expand_typed(const void* B, const Runs& b_bt, const Runs& b_k, const Runs& b_n, int64_t nbt, int64_t N,
                  int64_t K, int64_t half_pitch, bool bf16, void* Bx, cudaStream_t s, bool in_c64, void* Bx_lo,
                  float bscale, unsigned blocks, int pair, int4 lg) {
  if (bf16) {
    if (in_c64)
      expand_b_kernel<__nv_bfloat162, __nv_bfloat16, float2, I, P2><<<blocks, 256, 0, s>>>(
          (const float2*)B, b_bt, b_k, b_n, nbt, N, K, half_pitch, (__nv_bfloat162*)Bx, (__nv_bfloat162*)Bx_lo,
          bscale, pair, lg);
    else
      expand_b_kernel<__nv_bfloat162, __nv_bfloat16, __nv_bfloat162, I, P2><<<blocks, 256, 0, s>>>(
          (const __nv_bfloat162*)B, b_bt, b_k, b_n, nbt, N, K, half_pitch, (__nv_bfloat162*)Bx,
          (__nv_bfloat162*)Bx_lo, bscale, pair, lg);
  } else {
    if (in_c64)
      expand_b_kernel<__half2, __half, float2, I, P2><<<blocks, 256, 0, s>>>(
          (const float2*)B, b_bt, b_k, b_n, nbt, N, K, half_pitch, (__half2*)Bx, (__half2*)Bx_lo, bscale, pair,
          lg);
    else
      expand_b_kernel<__half2, __half, __half2, I, P2><<<blocks, 256, 0, s>>>(
          (const __half2*)B, b_bt, b_k, b_n, nbt, N, K, half_pitch, (__half2*)Bx, (__half2*)Bx_lo, bscale,
          pair, lg);
  }
}

// log2 of x, or -1 when x is not a power of two
int log2_or_neg(int64_t x) {
  if (x <= 0 || (x & (x - 1))) return -1;
  int r = 0;
  while ((int64_t(1) << r) < x) ++r;
  return r;
}
}  // namespace

void launch_expand_b(const void* B, const Runs& b_bt, const Runs& b_k, const Runs& b_n, int64_t nbt, int64_t N,
                     int64_t K, bool bf16, void* Bx, cudaStream_t s, bool in_c64, void* Bx_lo, float bscale,
                     bool pair) {
  // pair: the operand of the row-paired GEMM, extents 2N x 2K
  const int64_t Ne = pair ? 2 * N : N, Ke = pair ? 2 * K : K;
  const int64_t half_pitch = (2 * Ke + BK - 1) / BK * BK / 2;
  const int64_t total = nbt * Ne * half_pitch;
  if (total <= 0) return;
  TN_CHECK(half_pitch % 4 == 0 && (uintptr_t)Bx % 16 == 0 && (uintptr_t)Bx_lo % 16 == 0, TN_ERR_UNSUPPORTED,
           "expanded operand not 16-byte aligned");
  const unsigned blocks = (unsigned)std::min<int64_t>((total / 4 + 255) / 256, 152 * 32);
  const int4 lg = make_int4(log2_or_neg(half_pitch), log2_or_neg(Ne), log2_or_neg(pair ? K : Ke), 0);
  const bool p2 = lg.x >= 0 && lg.y >= 0 && lg.z >= 0;
  // 32-bit indices when every index and offset of B and the expanded copy fits
  const bool i32 = 2 * total < (int64_t(1) << 31) && nbt * Ne * Ke < (int64_t(1) << 30);
  const int pr = pair ? 1 : 0;
  if (i32 && p2)
    expand_typed<int32_t, true>(B, b_bt, b_k, b_n, nbt, Ne, Ke, half_pitch, bf16, Bx, s, in_c64, Bx_lo, bscale,
                                blocks, pr, lg);
  else if (i32)
    expand_typed<int32_t, false>(B, b_bt, b_k, b_n, nbt, Ne, Ke, half_pitch, bf16, Bx, s, in_c64, Bx_lo, bscale,
                                 blocks, pr, lg);
  else if (p2)
    expand_typed<int64_t, true>(B, b_bt, b_k, b_n, nbt, Ne, Ke, half_pitch, bf16, Bx, s, in_c64, Bx_lo, bscale,
                                blocks, pr, lg);
  else
    expand_typed<int64_t, false>(B, b_bt, b_k, b_n, nbt, Ne, Ke, half_pitch, bf16, Bx, s, in_c64, Bx_lo, bscale,
                                 blocks, pr, lg);
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
// the same for a result stored [bt][n][m] (m contiguous) against b = [bt][m][n]
__global__ void diff_t_kernel(const float2* a, const float2* b, int64_t nbt, int64_t M, int64_t N,
                              unsigned* max_diff) {
  float md = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nbt * M * N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t bt = i / (M * N), r = i - bt * M * N, m = r / N, n = r - m * N;
    const float2 x = a[bt * M * N + n * M + m];
    const float dx = x.x - b[i].x, dy = x.y - b[i].y;
    md = fmaxf(md, sqrtf(dx * dx + dy * dy));
    if (!(x.x == x.x) || !(x.y == x.y)) md = 3.0e38f;
  }
  atomicMax(max_diff, __float_as_uint(md));
}
// the same for a result stored [bt][n / 2][m][n % 2] (pairs of n outputs
// contiguous, rows two apart: the 16-byte store layout of fp32 outputs)
__global__ void diff_il_kernel(const float2* a, const float2* b, int64_t nbt, int64_t M, int64_t N,
                               unsigned* max_diff) {
  float md = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nbt * M * N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t bt = i / (M * N), r = i - bt * M * N, m = r / N, n = r - m * N;
    const float2 x = a[bt * M * N + (n / 2) * 2 * M + m * 2 + (n % 2)];
    const float dx = x.x - b[i].x, dy = x.y - b[i].y;
    md = fmaxf(md, sqrtf(dx * dx + dy * dy));
    if (!(x.x == x.x) || !(x.y == x.y)) md = 3.0e38f;
  }
  atomicMax(max_diff, __float_as_uint(md));
}
// a 16-bit result with its rounding residual, stored [bt][n / g][m][n % g]
// (g = N: [bt][m][n]), compared as hi + lo
template <class T2>
__global__ void diff_hl_kernel(const T2* hi, const T2* lo, const float2* b, int64_t nbt, int64_t M, int64_t N,
                               int64_t g, unsigned* max_diff) {
  float md = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nbt * M * N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t bt = i / (M * N), r = i - bt * M * N, m = r / N, n = r - m * N;
    const int64_t o = bt * M * N + (n / g) * g * M + m * g + (n % g);
    const float xr = (float)hi[o].x + (float)lo[o].x, xi = (float)hi[o].y + (float)lo[o].y;
    const float dx = xr - b[i].x, dy = xi - b[i].y;
    md = fmaxf(md, sqrtf(dx * dx + dy * dy));
    if (!(xr == xr) || !(xi == xi)) md = 3.0e38f;
  }
  atomicMax(max_diff, __float_as_uint(md));
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
    // one CTA per tile, K in one accumulator
    launch_gemm_tc(A, nullptr, M * K, K, Bx, nullptr, p, bf16, s);
    if (bf16)
      ref_kernel<__nv_bfloat162><<<1024, 256, 0, s>>>((const __nv_bfloat162*)A, (const __nv_bfloat162*)B,
                                                     (float2*)R, nbt, M, N, K);
    else
      ref_kernel<__half2><<<1024, 256, 0, s>>>((const __half2*)A, (const __half2*)B, (float2*)R, nbt, M, N, K);
    diff_kernel<<<1024, 256, 0, s>>>((const float2*)C, (const float2*)R, nbt * M * N, mx, mx + 1);
    // and K accumulated in chunks summed in FP32 registers
    TN_CUDA(cudaMemsetAsync(C, 0xff, nbt * M * N * 8, s));
    p.acc_split = 2;
    launch_gemm_tc(A, nullptr, M * K, K, Bx, nullptr, p, bf16, s);
    diff_kernel<<<1024, 256, 0, s>>>((const float2*)C, (const float2*)R, nbt * M * N, mx, mx + 1);
    // and 256-row tiles (two m halves sharing each B tile; tile width 256)
    if (p.bn == 256) {
      TN_CUDA(cudaMemsetAsync(C, 0xff, nbt * M * N * 8, s));
      p.acc_split = 0;
      p.m_halves = 2;
      launch_gemm_tc(A, nullptr, M * K, K, Bx, nullptr, p, bf16, s);
      diff_kernel<<<1024, 256, 0, s>>>((const float2*)C, (const float2*)R, nbt * M * N, mx, mx + 1);
    }
    // and an m-contiguous result ([bt][n][m], the direct epilogue's usual
    // layout) under each tile form
    p.c_m = single_run(M, 1);
    p.c_n = single_run(N, M);
    for (int v = 0; v < 2; ++v) {
      if (v == 1 && p.bn != 256) break;
      TN_CUDA(cudaMemsetAsync(C, 0xff, nbt * M * N * 8, s));
      p.acc_split = 0;
      p.m_halves = v == 1 ? 2 : 1;
      launch_gemm_tc(A, nullptr, M * K, K, Bx, nullptr, p, bf16, s);
      diff_t_kernel<<<1024, 256, 0, s>>>((const float2*)C, (const float2*)R, nbt, M, N, mx);
    }
    // and (M, N powers of two) pairs of n outputs contiguous with rows two
    // apart, which the epilogue writes with 16-byte stores
    auto pow2 = [](int64_t x) { return x > 0 && (x & (x - 1)) == 0; };
    if (pow2(M) && pow2(N) && N >= 2) {
      int lgM = 0, lgN = 0;
      while ((int64_t(1) << lgM) < M) ++lgM;
      while ((int64_t(1) << lgN) < N) ++lgN;
      p.c_m = single_run(M, 2);
      p.c_n.n = lgN > 1 ? 2 : 1;
      p.c_n.lg[0] = 1;
      p.c_n.st[0] = 1;
      if (lgN > 1) {
        p.c_n.lg[1] = (int8_t)(lgN - 1);
        p.c_n.st[1] = 2 * M;
      }
      p.c_bt = single_run(nbt, M * N);
      for (int v = 0; v < 2; ++v) {
        if (v == 1 && p.bn != 256) break;
        TN_CUDA(cudaMemsetAsync(C, 0xff, nbt * M * N * 8, s));
        p.acc_split = 0;
        p.m_halves = v == 1 ? 2 : 1;
        launch_gemm_tc(A, nullptr, M * K, K, Bx, nullptr, p, bf16, s);
        diff_il_kernel<<<1024, 256, 0, s>>>((const float2*)C, (const float2*)R, nbt, M, N, mx);
      }
    }
    // and 16-bit results with their residuals (M, N powers of two, N >= 8):
    // rows of 8 consecutive n outputs 32 bytes apart, and [bt][m][n] (the
    // 16-byte pieces staged through shared memory, two and four lanes per row)
    if (pow2(M) && pow2(N) && N >= 8) {
      int lgN = 0;
      while ((int64_t(1) << lgN) < N) ++lgN;
      char* lo = reinterpret_cast<char*>(C) + nbt * M * N * 4;
      for (int gi = 0; gi < (N > 8 ? 2 : 1); ++gi) {
        const int64_t g = gi ? N : 8;
        p.out_kind = bf16 ? 1 : 0;
        p.out_hilo = 1;
        p.C2 = lo;
        p.acc_split = 0;
        p.m_halves = 0;
        p.c_bt = single_run(nbt, M * N);
        p.c_m = single_run(M, g);
        p.c_n = single_run(g, 1);
        if (g < N) {
          p.c_n.n = 2;
          p.c_n.lg[0] = 3;
          p.c_n.lg[1] = (int8_t)(lgN - 3);
          p.c_n.st[1] = 8 * M;
        }
        TN_CUDA(cudaMemsetAsync(C, 0xff, nbt * M * N * 8, s));
        launch_gemm_tc(A, nullptr, M * K, K, Bx, nullptr, p, bf16, s);
        if (bf16)
          diff_hl_kernel<__nv_bfloat162><<<1024, 256, 0, s>>>((const __nv_bfloat162*)C, (const __nv_bfloat162*)lo,
                                                              (const float2*)R, nbt, M, N, g, mx);
        else
          diff_hl_kernel<__half2><<<1024, 256, 0, s>>>((const __half2*)C, (const __half2*)lo, (const float2*)R, nbt,
                                                       M, N, g, mx);
      }
    }
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

