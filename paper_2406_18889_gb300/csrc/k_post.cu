// Post-processing kernels (arXiv 2406.18889, Sec. III "Composition of our
// algorithm" and "Post-processing method and XEB amplification").
//
// * top-k: p(s) = |phi(s)|^2 / f evaluated as (re*re + im*im) * inv_f in FP64
//   with every operation rounded separately; keep the k largest ordered by
//   (p descending, full n-bit index ascending).  One CTA of 1024 threads per
//   block of 2^l candidates (or one CTA over all candidates in global mode):
//   each thread holds one candidate in registers; slots [0, k) carry the best
//   so far and slots [k, 1024) take the next chunk; a bitonic sort of the 1024
//   keys runs its strides below 32 with warp shuffles and the larger strides
//   through shared memory.
// * XEB (Eq. 1): 2^n / |S| * sum q - 1 with the sum in FP64 in a fixed order.
#include "tn_internal.h"

namespace tn {
namespace {

constexpr int kSortN = 1024;

struct Key {
  double p;
  long long idx;
};

// a is ordered before b: p descending, then index ascending.  Every p is a
// non-negative double or the -1 sentinel, and such values order exactly as
// their bit patterns read as signed 64-bit integers, so the comparison runs
// on the integer pipe (a NaN p has already raised the numeric flag).
__device__ __forceinline__ bool before(const Key& a, const Key& b) {
  const long long pa = __double_as_longlong(a.p), pb = __double_as_longlong(b.p);
  return pa > pb || (pa == pb && a.idx < b.idx);
}

__device__ __forceinline__ long long full_index(long long base, long long j, const TopkParams& tp) {
  long long part = 0;
  for (int i = 0; i < tp.l; ++i) part |= ((j >> (tp.l - 1 - i)) & 1LL) << tp.open_pos[i];
  return base | part;
}

__device__ __forceinline__ Key load_key(const double2* amps, long long x, long long g, long long j,
                                        const int64_t* base, const TopkParams& tp, int* flag) {
  double2 a = amps[x];
  double p = __dmul_rn(__dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y)), tp.inv_f);
  if (isnan(p) && flag) atomicExch(flag, 1);
  Key k;
  k.p = p;
  k.idx = full_index(base[g], j, tp);
  return k;
}

__device__ void bitonic_sort_1024(Key& mine, Key* sh) {
  const int i = threadIdx.x;
  for (int size = 2; size <= kSortN; size <<= 1) {
    const bool dir = (i & size) == 0;  // this run is sorted into `before` order
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      Key other;
      if (stride >= 32) {
        sh[i] = mine;
        __syncthreads();
        other = sh[i ^ stride];
        __syncthreads();
      } else {
        other.p = __shfl_xor_sync(0xffffffffu, mine.p, stride);
        other.idx = __shfl_xor_sync(0xffffffffu, mine.idx, stride);
      }
      const bool lower = (i & stride) == 0;
      const bool mine_first = before(mine, other);
      // lower slot keeps the element that comes first when dir, else the later
      const bool keep_mine = (lower == dir) ? mine_first : !mine_first;
      if (!keep_mine) mine = other;
    }
  }
}

__global__ void __launch_bounds__(kSortN) topk_kernel(const double2* __restrict__ amps, TopkParams tp,
                                                      const int64_t* __restrict__ base,
                                                      int64_t* __restrict__ out_idx,
                                                      double* __restrict__ out_p, int* flag) {
  __shared__ Key sh[kSortN];
  const int i = threadIdx.x;
  const int k = tp.k;
  const long long n_total = tp.global_mode ? tp.G * tp.Bsz : tp.Bsz;
  const long long g0 = tp.global_mode ? 0 : blockIdx.x;
  Key mine;
  mine.p = -1.0;
  mine.idx = 0x7fffffffffffffffLL;
  // the first pass fills all kSortN slots; later passes refill slots [k, kSortN)
  // while slots [0, k) carry the best so far (a block of <= kSortN strings: one sort)
  const int chunk = kSortN - k;
  for (long long start = 0; start < n_total; start += (start == 0 ? kSortN : chunk)) {
    if (start == 0 || i >= k) {
      long long e = start == 0 ? i : start + (i - k);
      if (e < n_total) {
        long long g = tp.global_mode ? e / tp.Bsz : g0;
        long long j = tp.global_mode ? e % tp.Bsz : e;
        mine = load_key(amps, g * tp.Bsz + j, g, j, base, tp, flag);
      } else {
        mine.p = -1.0;
        mine.idx = 0x7fffffffffffffffLL;
      }
    }
    bitonic_sort_1024(mine, sh);
  }
  if (i < k) {
    long long o = (tp.global_mode ? 0 : g0 * k) + i;
    out_idx[o] = mine.idx;
    out_p[o] = mine.p;
  }
}

__global__ void __launch_bounds__(1024) xeb_kernel(const double* __restrict__ q, int64_t n, int n_qubits,
                                                   double* out) {
  __shared__ double sh[1024];
  double s = 0.0;
  for (int64_t x = threadIdx.x; x < n; x += 1024) s += q[x];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    out[0] = __dsub_rn(__dmul_rn(__ddiv_rn(ldexp(1.0, n_qubits), (double)n), sh[0]), 1.0);
}

}  // namespace

void launch_topk(const double2* amps, const TopkParams& tp, const int64_t* block_base, int64_t* out_idx,
                 double* out_p, int* d_flag, cudaStream_t s) {
  unsigned grid = tp.global_mode ? 1u : (unsigned)tp.G;
  topk_kernel<<<grid, kSortN, 0, s>>>(amps, tp, block_base, out_idx, out_p, d_flag);
}

void launch_xeb(const double* q, int64_t n, int n_qubits, double* d_out, cudaStream_t s) {
  xeb_kernel<<<1, 1024, 0, s>>>(q, n, n_qubits, d_out);
}

}  // namespace tn
