// Global top-k over many candidates (arXiv 2406.18889, Sec. III "Composition of
// our algorithm": the k strings of largest p among all candidates S~; the
// Sycamore run keeps k = 3e6 of 3e6 * 2^10, the 30-qubit study k = 2^15 of 2^30).
//
// Exact selection by (p descending, full n-bit index ascending), p evaluated as
// (re*re + im*im) * inv_f in FP64 with every operation rounded separately:
//  1. radix select on p's 64 IEEE bits (non-negative doubles order as their bit
//     patterns): passes of 12 bits (then 4), each a histogram of the next digit
//     over the candidates that match the digits chosen so far, and a one-CTA
//     scan that picks the digit where the count from the top reaches k; this
//     fixes the k-th largest value T and how many candidates equal to T to take;
//  2. only if more candidates equal T than are needed, the same select on their
//     full indices (the smallest ones are taken);
//  3. the chosen candidates are gathered (order of arrival) and bitonic-sorted
//     into (p desc, index asc): shared-memory stages for strides below 2048,
//     one launch per stride above.
// After the first digit the candidates in its chosen bucket (usually few) are
// compacted once and the remaining passes run over them; all other decisions
// stay on the device (one host read of the bucket's size).
#include <cuda_runtime.h>

#include <algorithm>

#include "tn_internal.h"

namespace tn {
namespace {

constexpr int kDigitBits = 12;
constexpr int kBins = 1 << kDigitBits;
constexpr int kLocal = 2048;  // elements sorted per CTA in shared memory
constexpr unsigned long long kMaxCompact = 1ull << 26;  // candidates kept in the top digit's bucket

struct SelState {
  unsigned long long prefix, mask;  // decided key bits
  unsigned long long need;          // candidates still to take among those matching prefix
  unsigned long long n_eq;          // candidates equal to the final threshold
  unsigned long long tie;           // 1: more candidates equal T than needed
  unsigned long long idx_prefix, idx_mask, idx_need;
  unsigned long long n_out;         // gathered so far
  unsigned long long n_bucket;      // candidates in the digit chosen by the last pick
  unsigned long long n_comp;        // compacted candidates
};

// a candidate of the threshold bucket: p's key and its position
struct Comp {
  unsigned long long key;
  long long x;
};

struct Cand {
  double p;
  long long idx;
};

__device__ __forceinline__ double prob(const double2* amps, long long x, double inv_f) {
  const double2 a = amps[x];
  return __dmul_rn(__dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y)), inv_f);
}

__device__ __forceinline__ long long full_index(long long base, long long j, const TopkParams& tp) {
  long long part = 0;
  for (int i = 0; i < tp.l; ++i) part |= ((j >> (tp.l - 1 - i)) & 1LL) << tp.open_pos[i];
  return base | part;
}

__device__ __forceinline__ unsigned long long key_of(double p) {
  return (unsigned long long)__double_as_longlong(p);
}

// histogram of key digit [shift, shift + width) over candidates whose decided bits
// match; idx_mode: the key is the full index, restricted to p's key == T
__global__ void __launch_bounds__(256) hist_kernel(const double2* __restrict__ amps, TopkParams tp,
                                                   const int64_t* __restrict__ base, const SelState* st,
                                                   unsigned long long* hist, int shift, int width, int idx_mode,
                                                   int* flag) {
  __shared__ unsigned int h[kBins];
  if (idx_mode && !st->tie) return;
  for (int b = threadIdx.x; b < kBins; b += blockDim.x) h[b] = 0;
  __syncthreads();
  const long long n = tp.G * tp.Bsz;
  const unsigned long long pm = idx_mode ? st->idx_mask : st->mask;
  const unsigned long long pp = idx_mode ? st->idx_prefix : st->prefix;
  const unsigned long long T = st->prefix;
  const unsigned long long dmask = (1ull << width) - 1;
  const int lane = threadIdx.x & 31;
  // warp-uniform loop; lanes with the same digit add once per warp (the digits
  // of p crowd into a few exponent bins)
  for (long long wb = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); wb < n;
       wb += (long long)gridDim.x * blockDim.x) {
    const long long x = wb + lane;
    bool match = false;
    unsigned bin = 0xffffffffu;
    if (x < n) {
      const double p = prob(amps, x, tp.inv_f);
      if (!idx_mode && flag && isnan(p)) atomicExch(flag, 1);
      unsigned long long key = key_of(p);
      bool take = true;
      if (idx_mode) {
        take = key == T;
        if (take) key = (unsigned long long)full_index(base[x / tp.Bsz], x % tp.Bsz, tp);
      }
      match = take && (key & pm) == pp;
      if (match) bin = (unsigned)((key >> shift) & dmask);
    }
    const unsigned same = __match_any_sync(0xffffffffu, bin);
    if (match && lane == __ffs(same) - 1) atomicAdd(&h[bin], (unsigned)__popc(same));
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kBins; b += blockDim.x)
    if (h[b]) atomicAdd(&hist[b], (unsigned long long)h[b]);
}

// one CTA: pick the digit where the running count reaches `need` (from the top
// for p, from the bottom for indices), update the state, clear the histogram
__global__ void __launch_bounds__(1024) pick_kernel(SelState* st, unsigned long long* hist, int shift, int width,
                                                    int idx_mode, int last) {
  __shared__ unsigned long long part[1024];
  if (idx_mode && !st->tie) return;
  const int nb = 1 << width;
  const int per = (nb + 1023) / 1024;
  // chunk sums in pick order (descending digits for p, ascending for indices)
  unsigned long long s = 0;
  for (int q = 0; q < per; ++q) {
    const int r = threadIdx.x * per + q;
    if (r < nb) s += hist[idx_mode ? r : nb - 1 - r];
  }
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long need = idx_mode ? st->idx_need : st->need;
    const int n_chunks = (nb + per - 1) / per;
    unsigned long long cum = 0;
    int c = 0;
    while (c < n_chunks - 1 && cum + part[c] < need) cum += part[c++];
    int r = c * per;  // <= nb - 1
    int digit = 0;
    unsigned long long cnt = 0;
    for (;; ++r) {
      digit = idx_mode ? r : nb - 1 - r;
      cnt = hist[digit];
      if (cum + cnt >= need || r >= nb - 1) break;
      cum += cnt;
    }
    const unsigned long long dm = ((1ull << width) - 1) << shift;
    st->n_bucket = cnt;
    if (idx_mode) {
      st->idx_prefix |= (unsigned long long)digit << shift;
      st->idx_mask |= dm;
      st->idx_need = need - cum;
    } else {
      st->prefix |= (unsigned long long)digit << shift;
      st->mask |= dm;
      st->need = need - cum;
      if (last) {
        st->n_eq = cnt;
        st->tie = cnt > need - cum ? 1ull : 0ull;
        st->idx_need = need - cum;
      }
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kBins; b += blockDim.x) hist[b] = 0;
}

// gather the chosen candidates: p's key above T, or equal to T (all of them, or
// with index at most the selected index threshold when ties straddle T)
__global__ void __launch_bounds__(256) gather_kernel(const double2* __restrict__ amps, TopkParams tp,
                                                     const int64_t* __restrict__ base, SelState* st,
                                                     Cand* __restrict__ out, unsigned long long cap) {
  const long long n = tp.G * tp.Bsz;
  const unsigned long long T = st->prefix;
  const bool tie = st->tie != 0;
  const unsigned long long I = st->idx_prefix;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
    const double p = prob(amps, x, tp.inv_f);
    const unsigned long long key = key_of(p);
    if (key < T) continue;
    const long long idx = full_index(base[x / tp.Bsz], x % tp.Bsz, tp);
    if (key == T && tie && (unsigned long long)idx > I) continue;
    const unsigned long long slot = atomicAdd(&st->n_out, 1ull);
    if (slot < cap) out[slot] = Cand{p, idx};
  }
}

// after the first digit: candidates above the chosen top digit go straight to
// the output; those in it are compacted (key, position) for the later passes
__global__ void __launch_bounds__(256) compact_kernel(const double2* __restrict__ amps, TopkParams tp,
                                                      const int64_t* __restrict__ base, SelState* st,
                                                      Cand* __restrict__ out, unsigned long long cap_out,
                                                      Comp* __restrict__ comp, unsigned long long cap_comp,
                                                      int shift) {
  const long long n = tp.G * tp.Bsz;
  const unsigned long long top = st->prefix >> shift;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
    const double p = prob(amps, x, tp.inv_f);
    const unsigned long long key = key_of(p);
    const unsigned long long d = key >> shift;
    if (d > top) {
      const unsigned long long slot = atomicAdd(&st->n_out, 1ull);
      if (slot < cap_out) out[slot] = Cand{p, full_index(base[x / tp.Bsz], x % tp.Bsz, tp)};
    } else if (d == top) {
      const unsigned long long slot = atomicAdd(&st->n_comp, 1ull);
      if (slot < cap_comp) comp[slot] = Comp{key, x};
    }
  }
}

// hist_kernel over the compacted candidates
__global__ void __launch_bounds__(256) hist_comp_kernel(const Comp* __restrict__ comp, unsigned long long m,
                                                        TopkParams tp, const int64_t* __restrict__ base,
                                                        const SelState* st, unsigned long long* hist, int shift,
                                                        int width, int idx_mode) {
  __shared__ unsigned int h[kBins];
  if (idx_mode && !st->tie) return;
  for (int b = threadIdx.x; b < kBins; b += blockDim.x) h[b] = 0;
  __syncthreads();
  const unsigned long long pm = idx_mode ? st->idx_mask : st->mask;
  const unsigned long long pp = idx_mode ? st->idx_prefix : st->prefix;
  const unsigned long long T = st->prefix;
  const unsigned long long dmask = (1ull << width) - 1;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < m;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned long long key = comp[i].key;
    if (idx_mode) {
      if (key != T) continue;
      const long long x = comp[i].x;
      key = (unsigned long long)full_index(base[x / tp.Bsz], x % tp.Bsz, tp);
    }
    if ((key & pm) == pp) atomicAdd(&h[(key >> shift) & dmask], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kBins; b += blockDim.x)
    if (h[b]) atomicAdd(&hist[b], (unsigned long long)h[b]);
}

// gather_kernel over the compacted candidates (those above the bucket are out already)
__global__ void __launch_bounds__(256) gather_comp_kernel(const Comp* __restrict__ comp, unsigned long long m,
                                                          const double2* __restrict__ amps, TopkParams tp,
                                                          const int64_t* __restrict__ base, SelState* st,
                                                          Cand* __restrict__ out, unsigned long long cap) {
  const unsigned long long T = st->prefix;
  const bool tie = st->tie != 0;
  const unsigned long long I = st->idx_prefix;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < m;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long key = comp[i].key;
    if (key < T) continue;
    const long long x = comp[i].x;
    const long long idx = full_index(base[x / tp.Bsz], x % tp.Bsz, tp);
    if (key == T && tie && (unsigned long long)idx > I) continue;
    const unsigned long long slot = atomicAdd(&st->n_out, 1ull);
    if (slot < cap) out[slot] = Cand{prob(amps, x, tp.inv_f), idx};
  }
}

__device__ __forceinline__ bool before(const Cand& a, const Cand& b) {
  return a.p > b.p || (a.p == b.p && a.idx < b.idx);
}

__global__ void pad_kernel(Cand* buf, unsigned long long from, unsigned long long to) {
  for (unsigned long long i = from + blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < to;
       i += (unsigned long long)gridDim.x * blockDim.x)
    buf[i] = Cand{-1.0, 0x7fffffffffffffffLL};
}

// bitonic stages with strides < 2048 inside a CTA's chunk: a full sort of the
// chunk (size_hi == 0) or the tail of the merge at `size`
__global__ void __launch_bounds__(1024) bitonic_local(Cand* buf, unsigned long long size) {
  __shared__ Cand sh[kLocal];
  const unsigned long long base = (unsigned long long)blockIdx.x * kLocal;
  for (int t = threadIdx.x; t < kLocal; t += blockDim.x) sh[t] = buf[base + t];
  __syncthreads();
  auto stage = [&](unsigned long long sz, int j) {
    for (int t = threadIdx.x; t < kLocal / 2; t += blockDim.x) {
      const int lo = 2 * j * (t / j) + (t % j), hi = lo + j;
      const unsigned long long gi = base + lo;
      const bool asc = (gi & sz) == 0;  // this run goes into `before` order
      Cand a = sh[lo], b = sh[hi];
      if (before(b, a) == asc) {
        sh[lo] = b;
        sh[hi] = a;
      }
    }
    __syncthreads();
  };
  if (size == 0) {
    for (unsigned long long sz = 2; sz <= (unsigned long long)kLocal; sz <<= 1)
      for (int j = (int)(sz >> 1); j > 0; j >>= 1) stage(sz, j);
  } else {
    for (int j = kLocal / 2; j > 0; j >>= 1) stage(size, j);
  }
  for (int t = threadIdx.x; t < kLocal; t += blockDim.x) buf[base + t] = sh[t];
}

__global__ void bitonic_global(Cand* buf, unsigned long long n, unsigned long long size, unsigned long long j) {
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < n / 2;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long lo = 2 * j * (t / j) + (t % j), hi = lo + j;
    const bool asc = (lo & size) == 0;
    Cand a = buf[lo], b = buf[hi];
    if (before(b, a) == asc) {
      buf[lo] = b;
      buf[hi] = a;
    }
  }
}

__global__ void write_kernel(const Cand* buf, int64_t k, int64_t* out_idx, double* out_p) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
    out_idx[i] = buf[i].idx;
    out_p[i] = buf[i].p;
  }
}

__global__ void init_state(SelState* st, unsigned long long k) {
  SelState z{};
  z.need = k;
  *st = z;
}

}  // namespace

void topk_global(const double2* amps, const TopkParams& tp, const int64_t* block_base, int64_t* out_idx,
                 double* out_p, int* d_flag, cudaStream_t s) {
  const unsigned long long k = (unsigned long long)tp.k;
  unsigned long long P = kLocal;
  while (P < k) P <<= 1;
  void* scratch = nullptr;
  const size_t hist_bytes = sizeof(unsigned long long) * kBins;
  const size_t bytes = 256 + hist_bytes + sizeof(Cand) * P;
  TN_CUDA(cudaMalloc(&scratch, bytes));
  SelState* st = reinterpret_cast<SelState*>(scratch);
  unsigned long long* hist = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(scratch) + 256);
  Cand* buf = reinterpret_cast<Cand*>(reinterpret_cast<char*>(hist) + hist_bytes);
  Comp* comp = nullptr;
  try {
    TN_CUDA(cudaMemsetAsync(hist, 0, hist_bytes, s));
    init_state<<<1, 1, 0, s>>>(st, k);
    const long long n = tp.G * tp.Bsz;
    const unsigned grid = (unsigned)std::min<long long>((n + 255) / 256, 152 * 8);
    // digits of the 64-bit key from the top: 12, 12, 12, 12, 12, 4 bits
    const int shifts[6] = {52, 40, 28, 16, 4, 0}, widths[6] = {12, 12, 12, 12, 12, 4};
    hist_kernel<<<grid, 256, 0, s>>>(amps, tp, block_base, st, hist, shifts[0], widths[0], 0, d_flag);
    pick_kernel<<<1, 1024, 0, s>>>(st, hist, shifts[0], widths[0], 0, 0);
    // the top digit's bucket usually holds few candidates: compact it once and
    // run the remaining passes over the compacted set (else over everything)
    unsigned long long n_bucket = 0;
    TN_CUDA(cudaMemcpyAsync(&n_bucket, &st->n_bucket, sizeof(n_bucket), cudaMemcpyDeviceToHost, s));
    TN_CUDA(cudaStreamSynchronize(s));
    if (n_bucket <= kMaxCompact) {
      TN_CUDA(cudaMalloc(&comp, sizeof(Comp) * std::max<unsigned long long>(n_bucket, 1)));
      compact_kernel<<<grid, 256, 0, s>>>(amps, tp, block_base, st, buf, P, comp, n_bucket, shifts[0]);
      const unsigned cgrid = (unsigned)std::min<unsigned long long>((n_bucket + 255) / 256 + 1, 152 * 8);
      for (int mode = 0; mode < 2; ++mode)
        for (int d = mode == 0 ? 1 : 0; d < 6; ++d) {
          hist_comp_kernel<<<cgrid, 256, 0, s>>>(comp, n_bucket, tp, block_base, st, hist, shifts[d], widths[d],
                                                 mode);
          pick_kernel<<<1, 1024, 0, s>>>(st, hist, shifts[d], widths[d], mode, d == 5 ? 1 : 0);
        }
      gather_comp_kernel<<<cgrid, 256, 0, s>>>(comp, n_bucket, amps, tp, block_base, st, buf, P);
    } else {
      for (int mode = 0; mode < 2; ++mode)
        for (int d = mode == 0 ? 1 : 0; d < 6; ++d) {
          hist_kernel<<<grid, 256, 0, s>>>(amps, tp, block_base, st, hist, shifts[d], widths[d], mode,
                                           mode == 0 ? d_flag : nullptr);
          pick_kernel<<<1, 1024, 0, s>>>(st, hist, shifts[d], widths[d], mode, d == 5 ? 1 : 0);
        }
      gather_kernel<<<grid, 256, 0, s>>>(amps, tp, block_base, st, buf, P);
    }
    pad_kernel<<<(unsigned)std::min<unsigned long long>((P + 255) / 256, 4096), 256, 0, s>>>(buf, k, P);
    const unsigned chunks = (unsigned)(P / kLocal);
    bitonic_local<<<chunks, 1024, 0, s>>>(buf, 0);
    for (unsigned long long size = 2 * kLocal; size <= P; size <<= 1) {
      for (unsigned long long j = size >> 1; j >= (unsigned long long)kLocal; j >>= 1)
        bitonic_global<<<(unsigned)std::min<unsigned long long>(P / 2 / 256 + 1, 152 * 16), 256, 0, s>>>(buf, P,
                                                                                                         size, j);
      bitonic_local<<<chunks, 1024, 0, s>>>(buf, size);
    }
    write_kernel<<<(unsigned)std::min<unsigned long long>((k + 255) / 256, 4096), 256, 0, s>>>(buf, (int64_t)k,
                                                                                             out_idx, out_p);
    TN_CUDA(cudaGetLastError());
    TN_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    cudaStreamSynchronize(s);
    cudaFree(scratch);
    if (comp) cudaFree(comp);
    throw;
  }
  TN_CUDA(cudaFree(scratch));
  if (comp) TN_CUDA(cudaFree(comp));
}

}  // namespace tn
