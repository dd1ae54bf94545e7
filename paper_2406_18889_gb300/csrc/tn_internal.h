// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/tn.h"

namespace tn {

// ---------------------------------------------------------------- errors
struct Error {
  tn_status code;
  std::string msg;
};
void set_error(const std::string& msg);
[[noreturn]] void fail(tn_status code, const std::string& msg);

#define TN_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      ::tn::fail(TN_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define TN_CHECK(cond, code, msg) \
  do {                            \
    if (!(cond)) ::tn::fail(code, msg); \
  } while (0)

// ------------------------------------------------------------ kernel params
constexpr int kMaxBits = 48;

// Index map of one index group of one tensor: the group's linear index i is
// split into digits, run 0 the fastest; digit r has 2^lg[r] values and stride
// st[r] (elements).  offset(i) = sum_r digit_r(i) * st[r].  The digit order is
// the group's canonical order, shared by every tensor holding the group, so a
// group may sit in memory as several separate runs in any order.
constexpr int kMaxRuns = 16;
struct Runs {
  int n;
  int8_t lg[kMaxRuns];
  int64_t st[kMaxRuns];
};

__host__ __device__ inline int64_t run_offset(const Runs& R, int64_t i) {
  int64_t o = 0;
  for (int r = 0; r < R.n; ++r) {
    o += (i & ((int64_t(1) << R.lg[r]) - 1)) * R.st[r];
    i >>= R.lg[r];
  }
  return o;
}

// Inverse of C's runs: output offset o -> (bt, m, n).  Entry e takes the
// digit (o >> pos[e]) & (2^lg[e] - 1) into group grp[e] (0 bt, 1 m, 2 n) at
// bit `shift[e]` of that group's index.  Valid when C is dense (it holds
// exactly nbt * M * N elements), which every contraction result is.
struct RunDecode {
  int n;
  int8_t pos[3 * kMaxRuns], lg[3 * kMaxRuns], grp[3 * kMaxRuns], shift[3 * kMaxRuns];
};

// C[bt][m][n] = scale * sum_k A[bt][m][k] * B[bt][k][n] with every index group
// addressed through its runs (any layout of A, B and C).
struct GemmParams {
  int64_t nbt, M, N, K;
  Runs a_bt, a_m, a_k;
  Runs b_bt, b_k, b_n;
  Runs c_bt, c_m, c_n;
  RunDecode c_dec;  // memory-order walk of C (small-K kernel)
  int64_t elems_max;  // largest of A, B, C in elements (index width selection)
  const void* A;
  const void* B;
  void* C;
  void* C2;  // low part of a hi+lo output (reduced precision), else unused
};

// out[pi(x)] = in[x] for a tensor of 2^nbits elements; out_bit[i] is the
// output bit position of input bit i (bit 0 = fastest varying).
struct BitPermute {
  int nbits;
  int out_bit[kMaxBits];
};

// Per-call gather of one sliced leaf into its batched copy (offsets in bytes
// from the plan-memory and workspace bases):
// dst[(r / inner) * B * inner + b * inner + r % inner] =
//   src[sel_off(slice_ids[b]) + r],  r in [0, rest), b in [0, B)
// sel_off(s) = sum_i ((s >> slice_bit[i]) & 1) * sel_stride[i]  (elements).
struct GatherLeaf {
  int64_t src_off;
  int64_t dst_off;
  int64_t rest, inner;
  int32_t n_sel;
  int32_t slice_bit[8];
  int64_t sel_stride[8];
};

// Generic strided copy used for leaf upload: out element o (row-major over
// dims[0..nd) ) = in[sum_d coord_d * in_stride[d]], converting complex128 to
// complex64 (or copying complex64).
struct StridedCopy {
  int nd;
  int64_t dims[kMaxBits];
  int64_t in_stride[kMaxBits];
};

// real k per stage of the tensor-core GEMM (one 128-byte row of 16-bit values)
constexpr int kTcKTile = 64;

// Tensor-core GEMM on interleaved 16-bit complex data (stacked 4M lowering):
// C[bt][m][n] = scale * sum_k A[bt][m][k] B[bt][k][n]; extents in complex elements.
struct TcGemmParams {
  int64_t nbt, M, N, K;
  Runs c_bt, c_m, c_n;        // output index maps
  void* C;
  int out_kind;               // 0 = fp16 complex, 1 = bf16 complex, 2 = fp32 complex
  int out_hilo;               // 16-bit output also writes its rounding residual to C2
  void* C2;
  float scale;                // power of two applied to the FP32 accumulators
  int* err;                   // device flag raised when a bounded wait times out
  int bn;                     // real-column tile (32, 64, 128 or 256)
  int stage_n;                // write tiles out along n (n is the output's contiguous index)
  int acc_split;              // > 0: accumulate K in chunks of this many k tiles, summed in FP32 registers
  int off32;                  // every offset inside a tile (from its base) fits in 32 bits (set by the launcher)
  int vec;                    // 16-byte stores of consecutive n outputs (set by the launcher)
  int vec_staged;             // with vec and stage_n: the 16-byte pieces go through shared memory and
  int vec_lpr_lg;             // 2^vec_lpr_lg lanes store consecutive pieces of one row together (launcher)
  int m_halves;              // 2: 256-row tiles, two 128-row MMAs sharing each B tile (tile width 256 only)
};

// ------------------------------------------------------------ launchers
void launch_gemm_c64(const GemmParams& p, int accumulate, cudaStream_t s);
void launch_bit_permute_c64(const void* in, void* out, const BitPermute& bp, cudaStream_t s);
void launch_strided_copy_c128_to_c64(const void* in, void* out, const StridedCopy& sc,
                                     int64_t n_out, cudaStream_t s);
void launch_gather_leaves(const GatherLeaf* d_table, int n_leaves, int64_t max_rest,
                          const int64_t* d_slice_ids, int B, const char* plan_base, char* ws_base,
                          cudaStream_t s, int elem_bytes = 8);
void launch_accumulate_c64(const void* root, int64_t sb, int64_t sg, int64_t sj, int64_t G,
                           int64_t J, const int32_t* d_n_valid, int B, void* amps, int accumulate,
                           cudaStream_t s, double scale = 1.0);
void launch_bit_permute(const void* in, void* out, const BitPermute& bp, int elem_bytes, cudaStream_t s);
void launch_strided_copy_c128(const void* in, void* out, const StridedCopy& sc, int64_t n_out, int out_kind,
                              double scale, cudaStream_t s);
// Destination of a CUDA-core step whose result is the expanded (real 2x2)
// operand of the tensor-core step that consumes it: the result is written
// straight into that step's expanded copy, [bt][2N][2K] 16-bit reals.
struct ExpandedDst {
  Runs b_bt, b_k, b_n;   // the consuming step's index maps of this tensor
  int64_t nbt, N, K;     // the consuming step's extents (K: a multiple of the k tile)
  void* Bx;
  void* Bx_lo;           // rounding residuals (split precision), else null
  bool bf16;
};
void launch_gemm_simt(const GemmParams& p, int in_kind, int out_kind, float scale, cudaStream_t s,
                      bool out_hilo = false, const ExpandedDst* ex = nullptr);
// row pitch of an expanded operand, in 16-bit pairs (2K rounded up to the k tile, halved)
int64_t expanded_half_pitch(int64_t K);
// group (0 bt, 1 m, 2 n) and natural bit of every position bit of a dense
// result decoded by d (group extents ext[]); false when a bit is not covered
bool output_position_bits(const RunDecode& d, int nbits, const int64_t ext[3], int8_t* grp, int8_t* nat);

// One small step run inside the fused small-step kernel (k_micro.cu): result
// C (dense, 2^nbits elements, memory order x) with operand offsets linear
// over the bits of x.
constexpr int kMicroMaxBits = 14;
struct MicroStep {
  int64_t a_off, b_off;          // operand byte offsets from their memory's base
  int64_t c_off, c2_off;         // result (and residual) byte offsets from their memory's base
  int32_t a_w[kMicroMaxBits];    // element offset in A of output bit j
  int32_t b_w[kMicroMaxBits];    // element offset in B of output bit j
  int32_t ak[4], bk[4];          // contracted-index offsets
  float scale;
  int8_t a_loc, b_loc;           // operand memory: 0 plan memory, 1 workspace, 2 the group's shared memory
  int8_t c_loc;                  // result memory: 1 workspace, 2 the group's shared memory (complex64)
  int8_t nbits, K, out_kind, out_hilo;
  int8_t pad_[5];
};
static_assert(sizeof(MicroStep) % 16 == 0, "micro step descriptors are copied in 16-byte pieces");
// complex64 operand copied into the group's shared memory before its first step
struct MicroLoad {
  int64_t src_off;               // byte offset from the source memory's base
  int32_t smem_off, elems;       // destination byte offset, complex64 elements
  int32_t src_loc, pad_;         // 0 plan memory, 1 workspace
};
// one CTA of the fused launch: steps [first_step, first_step + n_steps) in order
struct MicroGroup {
  int32_t first_step, n_steps, first_load, n_loads;
  int32_t desc_in_smem, pad_[3]; // descriptors copied to shared memory offset 0 first
};
constexpr int kMicroSmemBytes = 160 * 1024;  // dynamic shared memory of a fused launch, at most
void fill_micro_weights(const GemmParams& g, MicroStep& d);
// group g of [0, n_groups) runs on CTA g with smem_bytes of dynamic shared memory
void launch_micro(const MicroStep* d_steps, const MicroGroup* d_groups, const MicroLoad* d_loads, int n_groups,
                  int smem_bytes, const char* plan_base, char* ws_base, cudaStream_t s);
void launch_amax_c64(const void* x, int64_t n, unsigned* out, cudaStream_t s);
// d_ids[0..B) = ids, *d_n_valid = n_valid, through kernel parameters (asynchronous)
void launch_set_slice_ids(int64_t* d_ids, int32_t* d_n_valid, const int64_t* ids, int B, int32_t n_valid,
                          cudaStream_t s);
void launch_zero(void* p, size_t bytes, cudaStream_t s);
// out (+)= sum over p in order of parts[p] (complex128 [n_parts][n])
void launch_sum_partials(const void* parts, int64_t n_parts, int64_t n, void* out, int accumulate, cudaStream_t s);
struct TopkParams {
  int64_t G, Bsz;   // blocks and entries per block
  int k, l, global_mode;
  double inv_f;
  int8_t open_pos[64];  // bit position of open edge i (i = 0 most significant in j)
};
void launch_topk(const double2* amps, const TopkParams& tp, const int64_t* block_base,
                 int64_t* out_idx, double* out_p, int* d_flag, cudaStream_t s);
void launch_xeb(const double* q, int64_t n, int n_qubits, double* d_out, cudaStream_t s);
// exact global top-k over all G * Bsz candidates (radix select + bitonic sort),
// synchronous on s; d_flag is raised on a NaN probability
void topk_global(const double2* amps, const TopkParams& tp, const int64_t* block_base, int64_t* out_idx,
                 double* out_p, int* d_flag, cudaStream_t s);
bool tc_gemm_supported(int64_t nbt, int64_t M, int64_t N, int64_t K, int64_t sa_bt, int64_t sa_m, int64_t sa_k);
int tc_gemm_bn(int64_t N);
// A/A_lo: 16-bit complex [bt][M][K] (k contiguous); Bx/Bx_lo: expanded operand.
// With A_lo and Bx_lo non-null the product is A*B + A*B_lo + A_lo*B (hi+lo split).
void launch_gemm_tc(const void* A, const void* A_lo, int64_t sa_bt, int64_t sa_m, const void* Bx,
                    const void* Bx_lo, const TcGemmParams& p, bool bf16, cudaStream_t s);
// expand a complex operand B[bt][k][n] (index maps b_bt, b_k, b_n) stored as fp32
// (in_c64) or 16-bit complex into its real 2x2 form; with Bx_lo non-null also
// the rounding residual of every entry
// pair: write the block-diagonal [[B, 0], [0, B]] of a row-paired step (2N x 2K)
void launch_expand_b(const void* B, const Runs& b_bt, const Runs& b_k, const Runs& b_n, int64_t nbt, int64_t N,
                     int64_t K, bool bf16, void* Bx, cudaStream_t s, bool in_c64 = false, void* Bx_lo = nullptr,
                     float bscale = 1.0f, bool pair = false);
Runs single_run(int64_t extent, int64_t stride);
// true when a wait on a barrier nothing completes gave up after limit_ns and raised its flag
bool selftest_bounded_wait(uint64_t limit_ns, cudaStream_t s);
// measured FP32 FMA throughput of the device (TFLOP/s, 2 flops per FMA)
double selftest_fp32_peak(cudaStream_t s);
RunDecode decode_of(const Runs& bt, const Runs& m, const Runs& n);
int64_t expanded_b_bytes(int64_t nbt, int64_t N, int64_t K);
double selftest_gemm_tc(int64_t nbt, int64_t M, int64_t N, int64_t K, bool bf16, uint64_t seed, cudaStream_t s,
                        int* d_err);

}  // namespace tn
