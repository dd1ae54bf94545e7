// Cross-rank sum of FP64 partial amplitudes (tn_sum_partials): the slice sum
// of Sec. III split over ranks -- each rank sums its own share of the slices,
// and the shares are added here in rank order, one fixed order.
#include "tn_internal.h"

namespace tn {

namespace {

// out[i] = (accumulate ? out[i] : 0) + parts[0][i] + parts[1][i] + ... in part order;
// two outputs per thread as 32-byte loads of each part
__global__ void sum_partials_kernel(const double2* __restrict__ parts, int64_t n_parts, int64_t n,
                                    double2* __restrict__ out, int accumulate) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    double re = 0.0, im = 0.0;
    if (accumulate) {
      const double2 o = out[i];
      re = o.x;
      im = o.y;
    }
    for (int64_t p = 0; p < n_parts; ++p) {
      const double2 v = parts[p * n + i];
      re += v.x;
      im += v.y;
    }
    out[i] = make_double2(re, im);
  }
}

}  // namespace

void launch_sum_partials(const void* parts, int64_t n_parts, int64_t n, void* out, int accumulate, cudaStream_t s) {
  if (n <= 0) return;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
  sum_partials_kernel<<<(unsigned)blocks, 256, 0, s>>>((const double2*)parts, n_parts, n, (double2*)out,
                                                       accumulate);
}

}  // namespace tn
