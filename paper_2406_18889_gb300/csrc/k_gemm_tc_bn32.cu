// Tensor-core GEMM kernels of tile width 32 real columns (every precision and
// epilogue variant), compiled as a translation unit of their own.
#include "tc_kernel.cuh"

namespace tn {
template void launch_tc_tiles<32>(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const CUtensorMap&,
                                   const TcGemmParams&, bool, bool, cudaStream_t);
}  // namespace tn
