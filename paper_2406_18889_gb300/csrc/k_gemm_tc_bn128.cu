// Tensor-core GEMM kernels of tile width 128 real columns (every precision and
// epilogue variant), compiled as a translation unit of their own.
#include "tc_kernel.cuh"

namespace tn {
template void launch_tc_tiles<128>(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const CUtensorMap&,
                                   const TcGemmParams&, bool, bool, cudaStream_t);
}  // namespace tn
