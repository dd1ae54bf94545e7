// tn_contract_slices_batched: many plans (e.g. many small circuits with uneven
// trees) in one captured CUDA graph.
//
// The plans are packed into up to kMaxBranches concurrent branches (longest
// work first onto the least-loaded branch); each branch owns one region of
// the caller's workspace, as large as the largest workspace among its plans,
// and runs its plans one after another.  Branches fork from and join back to
// one capture stream, so one graph holds every plan's slice batches, and
// replaying it runs small circuits side by side on the GPU instead of one
// launch sequence after another.  The graph is cached by the call's
// arguments (plans with their launch-form generation, slice ids, outputs,
// workspace) and replayed while they repeat.
#include <algorithm>
#include <cstring>
#include <list>
#include <map>
#include <mutex>
#include <numeric>
#include <string>

#include "plan.h"

namespace tn {

namespace {

constexpr int kMaxBranches = 8;

struct BatchedKey {
  std::vector<uint64_t> words;
  bool operator==(const BatchedKey& o) const { return words == o.words; }
};

struct BatchedEntry {
  BatchedKey key;
  std::vector<uint64_t> serials;  // plans the graph refers to
  int device = -1;
  cudaGraphExec_t exec = nullptr;
};

struct BatchedCache {
  std::mutex mu;
  std::list<BatchedEntry> entries;  // most recent first
  std::map<int, std::vector<cudaStream_t>> streams;  // per device: capture streams
  std::map<int, std::vector<cudaEvent_t>> events;    // per device: fork/join events
};

BatchedCache& cache() {
  static BatchedCache* c = new BatchedCache();  // never destroyed: graphs may outlive static teardown order
  return *c;
}

uint64_t mix(uint64_t h, uint64_t v) {
  h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
  return h;
}

}  // namespace

BatchedLayout batched_layout(const std::vector<Plan*>& plans, const int64_t* n_slices, size_t ws_bytes,
                             int max_branches) {
  const int n = (int)plans.size();
  BatchedLayout best;
  bool repeated = false;
  {
    std::vector<Plan*> s = plans;
    std::sort(s.begin(), s.end());
    repeated = std::adjacent_find(s.begin(), s.end()) != s.end();
  }
  // a plan listed twice shares its slice-id buffer across its calls: one branch
  const int kmax = repeated ? 1 : std::max(1, std::min({max_branches, kMaxBranches, std::max(n, 1)}));
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::vector<double> work(n);
  for (int i = 0; i < n; ++i) work[i] = (plans[i]->useful_flops_per_slice + 1.0) * (double)std::max<int64_t>(n_slices[i], 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
  for (int K = kmax; K >= 1; --K) {
    BatchedLayout L;
    L.branches = K;
    L.branch_of.assign(n, 0);
    std::vector<double> load(K, 0.0);
    std::vector<int64_t> region(K, 0);
    for (int i : order) {
      const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      L.branch_of[i] = k;
      load[k] += work[i];
      if (n_slices[i] > 0) region[k] = std::max<int64_t>(region[k], (plans[i]->mem.ws_bytes + 255) / 256 * 256);
    }
    L.offset.assign(K, 0);
    int64_t off = 0;
    for (int k = 0; k < K; ++k) {
      L.offset[k] = off;
      off += region[k];
    }
    L.bytes = off;
    if (off <= (int64_t)ws_bytes || K == 1) return L;
  }
  return best;
}

void drop_batched_graphs(uint64_t serial) {
  BatchedCache& C = cache();
  std::lock_guard<std::mutex> lock(C.mu);
  for (auto it = C.entries.begin(); it != C.entries.end();) {
    if (std::find(it->serials.begin(), it->serials.end(), serial) != it->serials.end()) {
      cudaDeviceSynchronize();  // a replay may still be running
      cudaGraphExecDestroy(it->exec);
      it = C.entries.erase(it);
    } else {
      ++it;
    }
  }
}

void contract_batched(const std::vector<Plan*>& plans, const int64_t* const* slice_ids, const int64_t* n_slices,
                      void* const* amps, int accumulate, void* workspace, size_t ws_bytes, cudaStream_t stream) {
  const int n = (int)plans.size();
  if (n == 0) return;
  int dev = -1;
  TN_CUDA(cudaGetDevice(&dev));
  for (Plan* P : plans)
    TN_CHECK(P->device == dev, TN_ERR_INVALID_ARG, "every plan must live on the current device");
  const BatchedLayout L = batched_layout(plans, n_slices, ws_bytes, kMaxBranches);
  TN_CHECK(L.bytes <= (int64_t)ws_bytes, TN_ERR_INVALID_ARG, "workspace too small");
  // cache key: plans (serial, launch-form generation), ids, outputs, workspace, layout
  BatchedKey key;
  key.words.push_back((uint64_t)dev);
  key.words.push_back((uint64_t)accumulate);
  key.words.push_back((uint64_t)(uintptr_t)workspace);
  key.words.push_back((uint64_t)L.branches);
  for (int i = 0; i < n; ++i) {
    key.words.push_back(plans[i]->serial);
    key.words.push_back(plans[i]->generation);
    key.words.push_back((uint64_t)(uintptr_t)amps[i]);
    key.words.push_back((uint64_t)n_slices[i]);
    uint64_t h = 0x2406188890ull;
    for (int64_t j = 0; j < n_slices[i]; ++j) h = mix(h, (uint64_t)slice_ids[i][j]);
    key.words.push_back(h);
  }
  BatchedCache& C = cache();
  std::unique_lock<std::mutex> lock(C.mu);
  for (auto it = C.entries.begin(); it != C.entries.end(); ++it) {
    if (it->key == key) {
      C.entries.splice(C.entries.begin(), C.entries, it);
      TN_CUDA(cudaGraphLaunch(C.entries.front().exec, stream));
      return;
    }
  }
  // capture streams and fork/join events of this device
  std::vector<cudaStream_t>& cs = C.streams[dev];
  std::vector<cudaEvent_t>& ev = C.events[dev];
  while ((int)cs.size() < kMaxBranches) {
    cudaStream_t st = nullptr;
    TN_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cs.push_back(st);
  }
  while ((int)ev.size() < kMaxBranches + 1) {
    cudaEvent_t e = nullptr;
    TN_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ev.push_back(e);
  }
  cudaGraph_t g = nullptr;
  TN_CUDA(cudaStreamBeginCapture(cs[0], cudaStreamCaptureModeThreadLocal));
  try {
    TN_CUDA(cudaEventRecord(ev[0], cs[0]));
    for (int k = 1; k < L.branches; ++k) TN_CUDA(cudaStreamWaitEvent(cs[k], ev[0], 0));
    for (int i = 0; i < n; ++i) {
      const int k = L.branch_of[i];
      char* ws = reinterpret_cast<char*>(workspace) + L.offset[k];
      const size_t region = (size_t)(k + 1 < L.branches ? L.offset[k + 1] - L.offset[k] : L.bytes - L.offset[k]);
      contract_checked(*plans[i], slice_ids[i], n_slices[i], amps[i], accumulate, ws, region, cs[k],
                       [](Plan& Q, void* w, void* a, int acc, cudaStream_t st) { run_batch_direct(Q, w, a, acc, st); });
    }
    for (int k = 1; k < L.branches; ++k) {
      TN_CUDA(cudaEventRecord(ev[k], cs[k]));
      TN_CUDA(cudaStreamWaitEvent(cs[0], ev[k], 0));
    }
  } catch (...) {
    cudaStreamEndCapture(cs[0], &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  cudaError_t e = cudaStreamEndCapture(cs[0], &g);
  if (e != cudaSuccess) fail(TN_ERR_CUDA, std::string("batched graph capture: ") + cudaGetErrorString(e));
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) fail(TN_ERR_CUDA, std::string("batched graph instantiate: ") + cudaGetErrorString(e));
  BatchedEntry ent;
  ent.key = std::move(key);
  for (Plan* P : plans) ent.serials.push_back(P->serial);
  ent.device = dev;
  ent.exec = exec;
  C.entries.push_front(std::move(ent));
  while (C.entries.size() > 4) {
    TN_CUDA(cudaDeviceSynchronize());  // a replay of the evicted graph may still be running
    cudaGraphExecDestroy(C.entries.back().exec);
    C.entries.pop_back();
  }
  TN_CUDA(cudaGraphLaunch(exec, stream));
}

}  // namespace tn
