// Plan: the network, its contraction tree and slicing, every intermediate's
// memory layout, the workspace map and the per-step kernel parameters.
#pragma once

#include <functional>
#include <map>
#include <memory>
#include <vector>

#include "tn_internal.h"

namespace tn {

// storage kinds (also the kernels' in/out kinds)
enum : int { KIND_F16 = 0, KIND_BF16 = 1, KIND_C64 = 2 };

struct Node {
  std::vector<int> edges;   // edge set of this tensor in one sub-network (+ batch edge if variant)
  std::vector<int> layout;  // storage order, slowest first
  int64_t elems = 1;
  bool variant = false;     // depends on the slice (carries the slice-batch edge)
  bool leaf = false;
  int leaf_id = -1;
  int consumer = -1;        // step consuming this node; -1 for the root
  int exp2 = 0;             // stored value = true value * 2^-exp2 (reduced precision)
  int kind = 2;             // storage: KIND_C64, or KIND_F16 / KIND_BF16 (tensor-core operands)
  bool hilo = false;        // 16-bit value followed by its 16-bit rounding residual
};

// Launch form of a tensor-core step: tile width in real columns, 128-row
// halves per tile.
struct TcForm {
  int bn, mh;
};

struct Step {
  int a = -1, b = -1, c = -1;          // node ids: operands and result
  std::vector<int> bt, m, n, k;        // ordered index groups
  std::vector<int> lc_nat;             // layout the GEMM writes
  bool post_perm = false;              // lc_nat differs from node c's layout
  bool variant = false;
  bool hoisted = false;                // runs once at plan creation
  GemmParams gp{};                     // sizes and strides (pointers filled at launch)
  BitPermute perm{};                   // lc_nat -> node c layout
  bool tc = false;                     // tensor-core GEMM in reduced precision
  bool tc_swap = false;                // tensor-core A operand is node b (else node a)
  bool hilo = false;                   // split-precision product (A, B as hi + lo)
  int hilo_group = -1;                 // tensor-core steps that split together (see build_plan)
  int bexp = 0;                        // the expanded operand is scaled by 2^-bexp into 16 bits
  bool fuse_expand = false;            // writes its result as the consumer's expanded operand
  bool b_fused = false;                // tensor-core step whose expanded operand its producer wrote
  bool micro = false;                  // small per-batch step run inside the fused small-step launch
  bool pair_rows = false;              // tensor-core step run with row pairs (see tc_roles in plan.cu)
  int tc_bn = 0, tc_mh = 0;            // tuned tensor-core launch form (tc_bn 0: the default heuristics)
  double cost = 0;                     // complex MACs with the batch edge at its planned size
  double cost_one = 0;                 // complex MACs of one sub-network
};

// Where every tensor lives for one storage precision.
struct MemPlan {
  bool c64 = true;                      // complex64 everywhere (else 16-bit, root in complex64)
  bool micro = false;                   // small steps run fused (their results never share memory)
  std::vector<int64_t> off;             // per node: byte offset
  std::vector<char> in_plan;            // per node: plan memory (1) or workspace (0)
  std::vector<int64_t> wsz;             // per node: workspace bytes it occupies (0 in plan memory)
  std::vector<int64_t> tmp_off;         // per step: natural-layout result before the transpose
  std::vector<int64_t> tmp_sz;
  std::vector<int64_t> bx_off;          // per step: expanded operand of a tensor-core GEMM
  std::vector<int64_t> bx_sz;           // (0 when the producer writes it into its own result)
  int64_t inv_bytes = 0;                // workspace [0, inv_bytes): slice-independent steps of a batch
  std::vector<GatherLeaf> gather;       // per sliced leaf
  std::vector<int> gather_node;
  int64_t gather_max_rest = 0;
  int64_t plan_bytes = 0, ws_bytes = 0;
  int64_t create_scratch = 0;           // transposes of hoisted steps (creation only)
};

struct Plan {
  int device = -1;                      // CUDA device the plan lives on (-1: plan-only)
  uint64_t serial = 0;                  // unique per plan in this process (graph caches)
  uint64_t generation = 0;              // bumped whenever launch forms change (graph caches)
  // network
  int n_leaves = 0, n_edges = 0;
  std::vector<int64_t> dim;             // edge dims; index n_edges is the slice-batch edge
  std::vector<std::vector<int>> leaf_edges;
  std::vector<int64_t> leaf_off;        // element offset of each leaf in leaf_data
  std::vector<int> open_edges;
  int block_edge = -1;
  int64_t G = 1, J = 1;
  // tree
  std::vector<int> sliced;              // sliced edge ids, bit i <-> sliced[i]
  int batch_edge = -1;                  // = n_edges
  int B = 1;                            // slice batch (power of two)
  std::vector<Node> nodes;
  std::vector<Step> steps;
  int root = -1;
  // options
  int prec = TN_PREC_C64;
  int skind = KIND_C64;                 // storage kind of intermediates
  uint32_t flags = 0;
  // memory
  MemPlan mem;                          // execution
  void* d_plan = nullptr;               // leaves + hoisted results
  int64_t* d_slice_ids = nullptr;       // [B]
  int32_t* d_n_valid = nullptr;
  GatherLeaf* d_gather = nullptr;       // gather table (device)
  int* d_err = nullptr;                 // raised by a timed-out device wait
  // fused small steps: subtrees of micro steps, each in topological order (one CTA each)
  std::vector<std::vector<int>> micro_groups;  // slice-independent groups first
  int n_micro_inv = 0;                  // how many groups are slice-independent
  MicroStep* d_micro = nullptr;
  MicroGroup* d_micro_groups = nullptr;
  MicroLoad* d_micro_loads = nullptr;
  int micro_smem = 0;                   // dynamic shared memory of the fused launches
  double micro_flops = 0, micro_bytes = 0;
  // root readout strides (elements)
  int64_t root_sb = 0, root_sg = 0, root_sj = 1;
  // statistics
  double useful_flops_per_slice = 0, algo_bytes_per_slice = 0, peak_intermediate_bytes = 0;
  int64_t calib_bytes = 0;              // device memory of the complex64 calibration pass (reduced precision)
  // split-precision selection (TN_FLAG_HILO_AUTO): calibration relative L2 errors, -1 = not measured
  double calib_err_chosen = -1, calib_err_none = -1;
  // CUDA graph cache
  cudaGraphExec_t graph = nullptr;
  void* graph_ws = nullptr;
  void* graph_amps = nullptr;
  int graph_acc = -1;
  cudaStream_t capture_stream = nullptr;
  // concurrent batch graph: the batch's launch units (gather, fused small
  // steps, steps), each with its branch and the units of other branches it
  // waits for (from the workspace ranges they touch)
  std::vector<int> unit_kind, unit_step, unit_branch;
  std::vector<std::vector<int>> unit_waits;
  std::vector<cudaStream_t> branch_streams;  // branches 1.. (branch 0 is the capturing stream)
  std::vector<cudaEvent_t> unit_events;      // one per unit, then the fork and the joins

  ~Plan();
};

// One plan for the given options; hilo_mask (per step, 1 = split product on a
// tensor-core step) overrides TN_FLAG_HILO when given.  max_slice_batch >= 1.
std::unique_ptr<Plan> build_plan(const tn_network_desc* net, const tn_tree_desc* tree,
                                 const tn_plan_options* opt, cudaStream_t stream,
                                 const std::vector<char>* hilo_mask = nullptr);
// tn_plan_create: resolves max_slice_batch = 0 (from memory), hilo_steps and
// TN_FLAG_HILO_AUTO (calibrated placement of split products), then builds.
std::unique_ptr<Plan> create_plan(const tn_network_desc* net, const tn_tree_desc* tree,
                                  const tn_plan_options* opt, cudaStream_t stream);
// Several plans in one captured graph (tn_contract_slices_batched).
struct BatchedLayout {
  int branches = 1;                // concurrent branches
  std::vector<int> branch_of;      // per plan
  std::vector<int64_t> offset;     // per branch: workspace offset (bytes)
  int64_t bytes = 0;               // workspace the layout needs
};
// Pack plans into at most max_branches branches whose workspace regions fit
// ws_bytes (fewer branches when they do not; one when a plan repeats).
BatchedLayout batched_layout(const std::vector<Plan*>& plans, const int64_t* n_slices, size_t ws_bytes,
                             int max_branches);
void contract_batched(const std::vector<Plan*>& plans, const int64_t* const* slice_ids, const int64_t* n_slices,
                      void* const* amps, int accumulate, void* workspace, size_t ws_bytes, cudaStream_t stream);
// Forget cached batched graphs that refer to the plan with this serial.
void drop_batched_graphs(uint64_t serial);

// The seeded calibration slice ids of a plan with batch B over n_sliced edges.
std::vector<int64_t> calibration_ids(int B, int n_sliced);

// Per-launch profiling record (tn_contract_slices_profile).
struct LaunchRecord {
  int kind;
  double flops, bytes;
  cudaEvent_t start, stop;
};

// The launch forms the tuner may try for step t (the default first); empty
// unless t is a tensor-core step that runs per batch.
std::vector<TcForm> tc_step_forms(const Plan& P, size_t t);
// Forget the captured batch graph (its kernels' launch forms changed).
void drop_graph(Plan& P);

// Queue one batch (n_valid <= B slice ids already in d_slice_ids) into amps.
// With `rec`, launches directly and brackets every kernel with an event pair.
void run_batch(Plan& P, void* ws, void* amps, int accumulate, cudaStream_t stream,
               std::vector<LaunchRecord>* rec = nullptr);
// The same with direct launches only (no graph is built or replayed).
void run_batch_direct(Plan& P, void* ws, void* amps, int accumulate, cudaStream_t stream);

// How one batch is queued once its slice ids are on the device.
using BatchRunner = std::function<void(Plan&, void* ws, void* amps, int accumulate, cudaStream_t)>;
// Validate a contraction call (before any device work), then queue its
// batches: slice-id upload + run(...) per batch of up to P.B slices.
void contract_checked(Plan& P, const int64_t* ids, int64_t n, void* amps, int accumulate, void* ws,
                      size_t ws_bytes, cudaStream_t s, const BatchRunner& run);

}  // namespace tn
