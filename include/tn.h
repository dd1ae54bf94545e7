/*
 * tn.h -- C ABI of the sliced tensor-network contraction library for
 * random-circuit sampling on one GB300 (sm_103a).
 *
 * Method (arXiv 2406.18889, "Leapfrogging Sycamore"):
 *   - Sec. III "Composition of our algorithm": amplitudes of k groups of 2^l
 *     correlated bitstrings are computed by contracting a fraction f of the
 *     sliced sub-networks; the top-k strings by p(s) = |phi(s)|^2 / f are kept.
 *   - Sec. III "Optimizing tensor contraction": slicing fixes the values of
 *     chosen edges; the network is the sum of its sub-networks over all value
 *     assignments; each sub-network is a sequence of pairwise contractions.
 *   - Eq. (1): linear XEB of a selection.
 *
 * Conventions
 *   - Every call returns a tn_status; TN_OK is 0.  On failure
 *     tn_last_error() returns a message for the calling host thread.
 *   - Arguments are validated before any device work is queued; an invalid
 *     call leaves device memory untouched.
 *   - Device pointers are caller-owned (the library never frees them).  The
 *     plan owns only its own device copy of the network and its step table.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls queue work on it and return without synchronising,
 *     except where a function says it synchronises.
 *   - A plan is immutable after creation, except for the tensor-core launch
 *     forms that tn_plan_autotune and tn_plan_set_tuning set (no other call
 *     may run on the plan meanwhile), and may be shared by host threads;
 *     concurrent calls must use distinct workspaces and output buffers.
 *   - Complex numbers are interleaved (re, im); complex64 = 2 x float,
 *     complex128 = 2 x double.
 *   - Bit order: qubit 0 is the most significant bit of an n-bit index.
 */
#ifndef TN_H_
#define TN_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TN_OK = 0,
  TN_ERR_INVALID_ARG = 1, /* bad pointer, size, id or descriptor */
  TN_ERR_OOM = 2,         /* device or host allocation failed */
  TN_ERR_CUDA = 3,        /* a CUDA runtime call failed (message has the code) */
  TN_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
  TN_ERR_UNSUPPORTED = 5, /* valid but not supported (e.g. a non power-of-two dim) */
  TN_ERR_NUMERIC = 6      /* a NaN or infinity was detected */
} tn_status;

typedef enum {
  TN_PREC_C64 = 0,  /* complex64 storage, FP32 complex multiply-add on CUDA cores */
  TN_PREC_BF16 = 1, /* bf16 complex storage, real tensor-core GEMMs, FP32 accumulate */
  TN_PREC_FP16 = 2  /* fp16 complex storage, real tensor-core GEMMs, FP32 accumulate */
} tn_precision;

/* Host-side fault injection (tests of callers' failure handling; no device
 * work is done by a call that fails this way): the environment variable
 * TN_FAULT=alloc makes tn_plan_create return TN_ERR_OOM, TN_FAULT=invalid_plan
 * makes it return TN_ERR_INVALID_ARG, and TN_FAULT=stream makes the
 * tn_contract_slices* calls return TN_ERR_CUDA, each before any device work. */

/* tn_plan_options.flags */
#define TN_FLAG_HOIST_INVARIANT 0x1u /* contract slice-independent subtrees once, at plan creation */
#define TN_FLAG_NO_GRAPH 0x2u        /* launch kernels directly instead of replaying a CUDA graph */
#define TN_FLAG_PLAN_ONLY 0x4u       /* host-side planning only: no device memory is touched and
                                        contraction calls on the plan fail (for inspection) */
#define TN_FLAG_HILO 0x8u            /* reduced precision: every tensor-core step multiplies
                                        split-precision operands (hi + lo, three passes) */
#define TN_FLAG_FINE_ACC 0x20u       /* reduced precision: tensor-core steps accumulate K one k tile
                                        (64 real products) at a time, summed in FP32 registers;
                                        with TN_FLAG_HILO the result has complex64 accuracy (without
                                        it, TN_FLAG_HILO accumulates 4 k tiles at a time) */
#define TN_FLAG_HILO_AUTO 0x40u      /* reduced precision: split-precision (hi + lo) products only on
                                        the tensor-core steps whose 16-bit rounding moves the
                                        calibration batch's amplitudes most, until their relative L2
                                        against a complex64 pass is within hilo_tol (selection at
                                        tn_plan_create, see tn_plan_precision) */
#define TN_FLAG_SERIAL_GRAPH 0x80u   /* the batch graph runs every launch in one chain.  Default:
                                        the launches are spread over concurrent graph branches, each
                                        waiting only for the launches whose workspace ranges it
                                        shares (its operands, or memory they freed), so that the
                                        slice-independent subtrees -- which have a workspace region
                                        of their own -- overlap the rest of the batch */

typedef struct tn_plan_s* tn_plan_t;

/*
 * Host-side tensor network (paper Sec. III: gate tensors, initial states and
 * projectors; all edges have power-of-two dimensions).
 *   n_leaves, n_edges : counts (n_leaves >= 1, n_edges >= 1).
 *   leaf_rank[n_leaves]: number of edges of each leaf (0..32).
 *   leaf_edges        : concatenated edge ids, leaf-major; within a leaf the
 *                       first edge is the slowest-varying axis of its data.
 *   edge_dim[n_edges] : dimension of each edge (power of two, >= 2).
 *   leaf_data         : host complex128, the leaves' elements concatenated in
 *                       leaf order, each row-major in its leaf_edges order.
 *                       Copied during tn_plan_create.
 *   n_open, open_edges: output edges of one block; element j of a block packs
 *                       them with open_edges[0] most significant.
 *   block_edge        : the block (group) hyper-edge g, shared by every
 *                       closed-qubit projector and kept to the output; -1 when
 *                       there is a single block.
 * Every edge other than open/block edges must appear in exactly two leaves.
 */
typedef struct {
  int32_t n_leaves;
  int32_t n_edges;
  const int32_t* leaf_rank;
  const int32_t* leaf_edges;
  const int64_t* edge_dim;
  const void* leaf_data;
  int32_t n_open;
  const int32_t* open_edges;
  int32_t block_edge;
} tn_network_desc;

/*
 * Contraction tree and slicing set (paper Sec. III: pairwise contraction
 * path; sliced edges).
 *   n_steps, pairs[2*n_steps]: SSA pairs -- leaf i has id i, step t creates
 *                       id n_leaves + t; every id is consumed exactly once and
 *                       the last step is the root (n_steps = n_leaves - 1).
 *   n_sliced, sliced_edges: bit i of a slice id is the value of
 *                       sliced_edges[i]; each must be a dimension-2 bond (two
 *                       leaves, not an output edge).  0 <= n_sliced <= 62.
 */
typedef struct {
  int32_t n_steps;
  const int32_t* pairs;
  int32_t n_sliced;
  const int32_t* sliced_edges;
} tn_tree_desc;

/*
 * prec            : arithmetic of the per-slice contractions (tn_precision).
 * flags           : TN_FLAG_* bits.
 * max_slice_batch : slices contracted together per launch sequence (power of
 *                   two, 1..65536); the workspace scales with it.  0 = chosen
 *                   from memory: the largest power of two, at most the number
 *                   of slices and 65536, whose device memory (plan memory plus
 *                   workspace, and the complex64 calibration pass of a
 *                   reduced-precision plan) fits mem_cap_bytes, or half of the
 *                   device's free memory at creation when mem_cap_bytes = 0
 *                   (a TN_FLAG_PLAN_ONLY plan then needs mem_cap_bytes > 0);
 *                   1 if none fits (then TN_ERR_OOM when the workspace exceeds
 *                   mem_cap_bytes).  tn_plan_slice_batch reports the choice.
 * mem_cap_bytes   : reject the plan (TN_ERR_OOM) if the workspace exceeds this
 *                   (0 = no cap).
 * hilo_steps      : NULL, or host [n_steps] of 0/1: 1 asks for a split-precision
 *                   (hi + lo) product on that step; it takes effect on the
 *                   tensor-core steps of a reduced-precision plan and is
 *                   ignored elsewhere.  NULL: TN_FLAG_HILO decides for every
 *                   step (or TN_FLAG_HILO_AUTO selects them).  Not combined
 *                   with TN_FLAG_HILO or TN_FLAG_HILO_AUTO.
 * hilo_tol        : TN_FLAG_HILO_AUTO's target relative L2 (0 < hilo_tol < 1;
 *                   0 selects 3e-3).
 */
typedef struct {
  int32_t prec;
  uint32_t flags;
  int32_t max_slice_batch;
  int64_t mem_cap_bytes;
  const uint8_t* hilo_steps;
  double hilo_tol;
} tn_plan_options;

/*
 * Build a plan: validates the network and tree, assigns every intermediate a
 * memory layout (contracted dimensions of both operands in one order, free
 * dimensions in the output's order, so most steps need no transpose), plans
 * workspace offsets, and copies the leaves to the device.
 * Reduced precision (TN_PREC_BF16 / TN_PREC_FP16): large steps run on the
 * tensor cores as one real GEMM with FP32 accumulation; the operand read by
 * the tensor cores as stored is kept as 16-bit complex pairs scaled by a
 * per-tensor power of two 2^-e (so that amplitudes far below the 16-bit normal
 * range do not underflow), the other operand is rounded to 16 bits when it is
 * expanded; with TN_FLAG_HILO both are split into hi + lo 16-bit parts.  Every
 * other tensor, the small steps (CUDA cores, FP32) and the root stay in
 * complex64.  e is fixed at creation by one complex64 calibration batch
 * (B seeded pseudo-random slice ids, splitmix64) as the exponent of the
 * tensor's largest component.
 * Creation temporarily needs a complex64 workspace for the calibration.
 * Synchronises `stream`.  *out is set only on success; destroy with
 * tn_plan_destroy.
 */
tn_status tn_plan_create(const tn_network_desc* net, const tn_tree_desc* tree,
                         const tn_plan_options* opt, void* stream, tn_plan_t* out);

tn_status tn_plan_destroy(tn_plan_t plan);

/* The plan's slice batch (max_slice_batch as given, or as chosen when it was
 * 0; 1 for a network without sliced edges). */
tn_status tn_plan_slice_batch(tn_plan_t plan, int32_t* batch);

/*
 * Precision record of a reduced-precision plan (split-precision products
 * only on the contractions whose error measurably moves the result).
 * With TN_FLAG_HILO_AUTO, tn_plan_create contracts the calibration slices
 * (the plan's seeded calibration batch) once in complex64 and, in the plan's
 * 16-bit precision, with every candidate placement it tries: no split; each
 * tensor-core step alone left unsplit (all others split) to size each step's
 * share of the error; then the steps with the largest shares split first
 * until the relative L2 of the calibration amplitudes is at most hilo_tol.
 *   rel_l2_chosen : relative L2 of the calibration amplitudes with the chosen
 *                   placement (-1 when no selection ran);
 *   rel_l2_none   : the same with no split product (-1 when not measured);
 *   n_tc_steps    : tensor-core steps; n_hilo_steps: of those, split.
 * Any output pointer may be NULL.
 */
tn_status tn_plan_precision(tn_plan_t plan, double* rel_l2_chosen, double* rel_l2_none, int32_t* n_tc_steps,
                            int32_t* n_hilo_steps);

/*
 * Cost model of one slice (paper Table I conventions):
 *   useful_flops_per_slice : 8 * sum over per-slice steps of batch*M*N*K
 *                            ("8 is the complex number product factor").
 *   algo_bytes_per_slice   : sum over per-slice steps of the bytes of both
 *                            operands and the result at the plan's precision.
 *   peak_intermediate_bytes: largest single intermediate for one slice.
 *   workspace_bytes        : device workspace tn_contract_slices needs.
 * Any output pointer may be NULL.
 */
tn_status tn_plan_query(tn_plan_t plan, int64_t* useful_flops_per_slice,
                        int64_t* algo_bytes_per_slice, int64_t* peak_intermediate_bytes,
                        int64_t* workspace_bytes);

/* Per-step description for profiling and tests: the step's GEMM shape and
 * whether it runs once per slice batch (variant) or once per plan.  kinds[t]
 * bit 0 = variant, bit 1 = needs an output transpose, bit 2 = hoisted (runs
 * at plan creation), bit 3 = tensor-core GEMM (reduced precision), bit 4 =
 * split-precision (hi + lo) tensor-core GEMM, bit 5 = writes its result
 * directly as the expanded operand of the tensor-core step consuming it,
 * bit 6 = tensor-core step whose expanded operand its producer wrote,
 * bit 7 = small step run inside the one fused launch of small steps. */
tn_status tn_plan_steps(tn_plan_t plan, int32_t max_steps, int64_t* batch, int64_t* m,
                        int64_t* n, int64_t* k, int32_t* kinds, int32_t* n_steps_out);

/*
 * Synchronise `stream` and report whether a bounded device-side wait of an
 * earlier call on this plan timed out (TN_ERR_TIMEOUT; the flag is then
 * cleared).  The contraction calls are asynchronous and cannot report it
 * themselves.
 */
tn_status tn_plan_status(tn_plan_t plan, void* stream);

/*
 * Per-step launch-form tuning of the tensor-core steps (paper Sec. III: each
 * step's contraction kernel is chosen by timing the candidates).  Every
 * tensor-core step that runs per batch tries each of its launch forms on one
 * batch of the given slices and keeps the fastest.  The forms are: tile width
 * (the widest for the step's N, or half of it), and at width 256 also 256-row
 * tiles (not with split-precision chunked accumulation).
 * Each form gets `reps` profiled passes, and the minimum event time per step
 * decides.  Every form computes each output with the same MMAs over K in the
 * same order, so tuning changes speed, not results.  The plan's captured batch
 * graph is dropped and rebuilt on the next call.
 *   plan      : created without TN_FLAG_PLAN_ONLY; a complex64 plan has no
 *               tensor-core steps (nothing is tuned, TN_OK).
 *   slice_ids : host [n_slices], 1 <= n_slices <= the plan's slice batch.
 *   amps, workspace, ws_bytes, stream : as for tn_contract_slices (amps is
 *               overwritten with the sum over the slices).
 *   reps      : 1..64 timed passes per form.
 *   forms     : host [2 * n_steps] (n_steps from tn_plan_steps) or NULL: per
 *               step the chosen (tile width, row halves); zeros for steps
 *               that are not tuned.
 * Errors: INVALID_ARG before any device work; CUDA_ERROR; TIMEOUT (a bounded
 * device wait gave up).  On an error the plan keeps its previous forms.
 * Synchronises `stream`.
 */
tn_status tn_plan_autotune(tn_plan_t plan, const int64_t* slice_ids, int64_t n_slices, void* amps,
                           void* workspace, size_t ws_bytes, void* stream, int32_t reps, int32_t* forms);

/*
 * Set the launch forms of the tensor-core steps, e.g. those tn_plan_autotune
 * returned, read back from a cache.  forms: host [2 * n_steps] with n_steps
 * the plan's step count; per step (0, 0) selects the default form, anything
 * else must be one of the forms tn_plan_autotune may try for that step; steps
 * that are not tuned take (0, 0).  Validated in full before anything changes
 * (INVALID_ARG).  Host-only: also valid on a TN_FLAG_PLAN_ONLY plan.
 */
tn_status tn_plan_set_tuning(tn_plan_t plan, const int32_t* forms, int32_t n_steps);

/*
 * Contract the sub-networks `slice_ids[0..n_slices)` (host array; each id in
 * [0, 2^n_sliced), duplicates allowed and counted twice) and add them into
 * amps.  amps: device complex128 [G][2^l] (G = block edge dimension or 1);
 * accumulate = 0 overwrites amps with the sum, 1 adds to it.  Each slice is
 * computed in the plan's precision and summed across slices in FP64 in a fixed
 * order: within a batch, four contiguous quarters of the batch each summed in
 * slice order, then the quarters in order; batch by batch (deterministic).  workspace: device,
 * >= workspace_bytes of tn_plan_query, 256-byte aligned.  n_slices = 0 with
 * accumulate = 0 zeroes amps.  The plan's device (current at tn_plan_create)
 * must be current (TN_ERR_INVALID_ARG otherwise).
 */
tn_status tn_contract_slices(tn_plan_t plan, const int64_t* slice_ids, int64_t n_slices,
                             void* amps, int accumulate, void* workspace, size_t ws_bytes,
                             void* stream);

/*
 * Several plans (e.g. many small circuits with uneven trees) in one call: plan p contracts slice_ids[p][0..n_slices[p]) into
 * amps[p], with the semantics of tn_contract_slices for each.  All of the
 * plans' slice batches are captured into ONE CUDA graph whose up to 8
 * concurrent branches each run a share of the plans one after another
 * (longest work first onto the least-loaded branch) in their own region of
 * `workspace`; a region is as large as the largest workspace_bytes among its
 * plans.  When ws_bytes does not hold 8 regions, fewer branches are used (one
 * branch needs the largest workspace_bytes of all plans);
 * tn_batched_workspace_bytes gives the size for a number of branches.  A plan
 * listed twice makes the call run on one branch.  The graph is kept (up to 4
 * per process) and replayed while the plans, their launch forms, slice ids,
 * outputs, workspace and accumulate flag repeat; otherwise it is captured
 * again.  Every plan must live on the current device.  Arguments of every
 * plan are validated before any work is queued.
 */
tn_status tn_contract_slices_batched(const tn_plan_t* plans, int32_t n_plans,
                                     const int64_t* const* slice_ids, const int64_t* n_slices,
                                     void* const* amps, int accumulate, void* workspace,
                                     size_t ws_bytes, void* stream);

/* Workspace bytes tn_contract_slices_batched needs for these plans and slice
 * counts on up to max_branches (>= 1) concurrent branches. */
tn_status tn_batched_workspace_bytes(const tn_plan_t* plans, int32_t n_plans, const int64_t* n_slices,
                                     int32_t max_branches, int64_t* bytes);

/*
 * Sum of FP64 partial amplitudes over ranks (paper Sec. III: the sum over
 * sliced sub-networks, split into independent subtasks whose partial sums are
 * reduced once; the paper's cross-node reduction).  Each rank contracts its own
 * share of the slice ids into a partial [G][2^l]; the partials, gathered on
 * one device, are added here in part order, a fixed order, so the sum does not
 * depend on how the gather was carried out.
 *   parts     : device complex128 [n_parts][n_amps], part p = rank p's partial.
 *   out       : device complex128 [n_amps]; accumulate = 0 overwrites it with
 *               the sum, 1 adds the sum to it (the old value first).
 * n_parts = 0 with accumulate = 0 zeroes out.  Asynchronous on `stream`.
 */
tn_status tn_sum_partials(const void* parts, int64_t n_parts, int64_t n_amps, void* out, int accumulate,
                          void* stream);

/*
 * Top-k post-processing (paper Sec. III): p = (re*re + im*im) * inv_f in FP64
 * (each product and the sum rounded separately, no fused multiply-add), then
 * the k largest p ordered by (p descending, full index ascending).
 *   amps          : device complex128 [G][B], B = 2^l.
 *   global_mode   : 0 = k per block (outputs [G][k]); 1 = k over all G*B
 *                   (outputs [k]).
 *   block_base_idx: device int64 [G], the closed bits of each block as an
 *                   n-bit index with every open bit 0.
 *   open_bit_pos  : host int64 [l], bit position (0 = LSB) of open edge i
 *                   (open edge 0 is the most significant bit of j).
 *   out_idx, out_p: device int64 / double outputs.
 * Constraints: per block, 1 <= k <= B, k <= 512, B <= 2^16; global, 1 <= k
 * <= G*B, k <= 2^26, B <= 2^40, G*B <= 2^40.  The global selection is exact (a
 * radix select on the FP64 bit patterns of p, then on the full indices of
 * candidates tied at the threshold) and allocates scratch of about 16 bytes per
 * selected string for the final sort.  A NaN probability makes the call return
 * TN_ERR_NUMERIC after synchronising the stream.
 */
tn_status tn_topk_postprocess(const void* amps, int64_t G, int64_t B, int32_t k, double inv_f,
                              int global_mode, const int64_t* block_base_idx,
                              const int64_t* open_bit_pos, int32_t l, int64_t* out_idx,
                              double* out_p, void* stream);

/*
 * Linear XEB, Eq. (1): 2^n_qubits / n_sel * sum(q) - 1, the sum in FP64 in a
 * fixed order.  q: device double [n_sel] (ideal probabilities of the selected
 * strings).  Synchronises `stream` and writes *out_xeb (host).
 */
tn_status tn_xeb(const double* q, int64_t n_sel, int32_t n_qubits, double* out_xeb, void* stream);

/*
 * Profiling form of tn_contract_slices: the same work launched directly (no
 * graph) with a CUDA event pair around every kernel; synchronises `stream`
 * and reports, per kernel launch in launch order, its class (0 = CUDA-core
 * GEMM, 1 = transpose, 2 = slice gather, 3 = FP64 accumulate, 4 = operand
 * expansion for the tensor cores, 5 = tensor-core GEMM), its duration in
 * milliseconds, and its algorithmic FLOPs (8 * batch*M*N*K for a GEMM, else 0)
 * and bytes (operands + result for a GEMM; bytes read + written otherwise).
 * Arrays hold max_records entries; *n_records is set to the number of
 * launches (which may exceed max_records: the rest are dropped).
 */
tn_status tn_contract_slices_profile(tn_plan_t plan, const int64_t* slice_ids, int64_t n_slices,
                                     void* amps, int accumulate, void* workspace, size_t ws_bytes,
                                     void* stream, int32_t max_records, int32_t* kind, float* ms,
                                     double* flops, double* bytes, int32_t* n_records);

/*
 * tn_contract_slices_noalloc -- tn_contract_slices without device allocation.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc, for example a host application whose device memory
 * is owned entirely by another allocator (a framework's caching pool reserved
 * up front), or a latency-critical loop where an allocation and the device
 * synchronisation it may imply are not allowed.  The caller still passes the
 * slice ids (host) and the output amps (device complex128 [G][2^l]), with the
 * same meaning as in tn_contract_slices.
 *
 * The workspace is a library-owned static device array of
 * TN_STATIC_WORKSPACE_BYTES (64 MiB), which every GPU that loads the library
 * keeps until the process exits.  A plan whose workspace_bytes
 * (tn_plan_query) exceeds it is rejected with TN_ERR_INVALID_ARG before any
 * work is queued; build such plans with a smaller max_slice_batch or use
 * tn_contract_slices.  The plan's device must be the current device (the
 * array used is that device's); otherwise TN_ERR_INVALID_ARG.  Argument
 * checks, TN_FAULT injection and batching are those of tn_contract_slices.  The first call on each device looks up the array's
 * device address (which also loads the library's device code on that device)
 * with that device current; make that first call before any stream capture.
 * Kernels are launched directly; no CUDA graph is built.  All calls share the
 * one array, which keeps the previous call's contents: calls whose work
 * overlaps on the GPU (different streams, or different host threads) race
 * and give wrong results -- serialise them.  No part of the array needs to
 * start at zero.  Calls no cudaMalloc, cudaFree or other allocating routine.
 */
#define TN_STATIC_WORKSPACE_BYTES (64ull << 20)
tn_status tn_contract_slices_noalloc(tn_plan_t plan, const int64_t* slice_ids, int64_t n_slices,
                                     void* amps, int accumulate, void* stream);

/*
 * Self-test of the tensor-core GEMM on this device: random complex operands
 * in fp16 (prec = TN_PREC_FP16) or bf16 (TN_PREC_BF16), A [nbt][M][K] and
 * B [nbt][K][N] (complex extents), multiplied by the tcgen05 kernel (after
 * expanding B to its real 2x2 form) in each of its tile forms -- one
 * accumulator per tile, K accumulated in chunks, and (tile width 256) 256-row
 * tiles; results stored n-contiguous and m-contiguous -- and by a plain FP32
 * CUDA-core reference from the same 16-bit inputs.  *max_rel_err = max over
 * the forms of max |C_tc - C_ref| / max |C_ref|.  Allocates and frees its own buffers; synchronises `stream`.
 * Returns TN_ERR_TIMEOUT if a bounded device wait gave up.
 */
tn_status tn_selftest_gemm_tc(int64_t nbt, int64_t M, int64_t N, int64_t K, int32_t prec, uint64_t seed,
                              double* max_rel_err, void* stream);

/*
 * Failure detection self-test: one device thread waits, bounded by limit_ns
 * nanoseconds of the global timer, on an mbarrier that nothing completes --
 * the same bounded wait every persistent kernel of the library uses.  The
 * wait must give up and raise its error flag: the call returns
 * TN_ERR_TIMEOUT (the expected outcome) or TN_OK if the barrier completed.
 * 1000 <= limit_ns <= 1e9.  Synchronises the stream; no GPU fault, no hang.
 */
tn_status tn_selftest_bounded_wait(uint64_t limit_ns, void* stream);

/*
 * Measured FP32 fused multiply-add throughput of the current device (the
 * roofline of the complex64 CUDA-core path: 4 FMAs per complex
 * multiply-add): *tflops = 2 flops per FMA / time, from CUDA events around
 * 8 independent FMA chains per thread over 8 CTAs of 256 threads per SM.
 */
tn_status tn_selftest_fp32_peak(double* tflops, void* stream);

/*
 * Index permutation of a tensor with power-of-two dimensions (paper Sec. III:
 * the order of dimensions, and transposes between contraction steps).  The
 * contraction path itself never calls it -- every GEMM reads and writes any
 * layout in place -- but layouts fixed by a caller can be converted with it.
 * in/out: device arrays of 2^nbits elements of elem_bytes (4 or 8) bytes,
 * not overlapping; element x of `in` goes to the index whose bit out_bit[i]
 * is bit i of x (out_bit a permutation of 0..nbits-1, host array).
 * 1 <= nbits <= 40.
 */
tn_status tn_permute(const void* in, void* out, int32_t nbits, const int32_t* out_bit, int32_t elem_bytes,
                     void* stream);

/* Message of the last failed call on this host thread ("" if none). */
const char* tn_last_error(void);

/* Library version string. */
const char* tn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TN_H_ */
