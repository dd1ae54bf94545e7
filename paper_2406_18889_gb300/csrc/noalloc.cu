// tn_contract_slices_noalloc: tn_contract_slices with a library-owned,
// statically sized workspace, for callers that cannot allocate device memory.
//
// The workspace is one file-scope __device__ array.  Host code never uses the
// array's name as a device address: the address is looked up once per device
// with cudaGetSymbolAddress (with that device current) and cached.  Work is
// launched directly (no CUDA graph is instantiated), so the call allocates
// nothing.  Every call on a device shares the same array; calls whose work
// overlaps on the GPU race on it.  Nothing in the array needs to start at
// zero: every intermediate is written before it is read.
#include <functional>
#include <mutex>
#include <string>
#include <vector>

#include "plan.h"

struct tn_plan_s {
  std::unique_ptr<tn::Plan> p;
};

namespace tn {

static __device__ __align__(256) unsigned char g_static_workspace[TN_STATIC_WORKSPACE_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_ws_addr[kMaxDevices] = {};

// Device address of the static workspace on the current device (set-up on
// first use per device).
void* static_workspace() {
  int dev = 0;
  TN_CUDA(cudaGetDevice(&dev));
  TN_CHECK(dev >= 0 && dev < kMaxDevices, TN_ERR_UNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_ws_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_workspace);
    if (e != cudaSuccess || p == nullptr)
      fail(TN_ERR_CUDA, std::string("cudaGetSymbolAddress(static workspace): ") + cudaGetErrorString(e));
    g_ws_addr[dev] = p;
  }
  return g_ws_addr[dev];
}

}  // namespace

void run_batch_direct(Plan& P, void* ws, void* amps, int accumulate, cudaStream_t stream);
tn_status guarded_call(const std::function<void()>& f);

}  // namespace tn

extern "C" tn_status tn_contract_slices_noalloc(tn_plan_t plan, const int64_t* slice_ids, int64_t n_slices,
                                                void* amps, int accumulate, void* stream) {
  using namespace tn;
  return guarded_call([&] {
    TN_CHECK(plan != nullptr, TN_ERR_INVALID_ARG, "plan is null");
    Plan& P = *plan->p;
    TN_CHECK(!(P.flags & TN_FLAG_PLAN_ONLY), TN_ERR_INVALID_ARG, "plan was created with TN_FLAG_PLAN_ONLY");
    TN_CHECK(amps != nullptr, TN_ERR_INVALID_ARG, "amps is null");
    TN_CHECK(n_slices >= 0 && (n_slices == 0 || slice_ids), TN_ERR_INVALID_ARG, "bad slice list");
    TN_CHECK(accumulate == 0 || accumulate == 1, TN_ERR_INVALID_ARG, "accumulate must be 0 or 1");
    TN_CHECK(P.mem.ws_bytes <= (int64_t)TN_STATIC_WORKSPACE_BYTES, TN_ERR_INVALID_ARG,
             "plan needs " + std::to_string(P.mem.ws_bytes) + " bytes of workspace; the static workspace holds " +
                 std::to_string((long long)TN_STATIC_WORKSPACE_BYTES) +
                 " (use tn_contract_slices or a smaller max_slice_batch)");
    const int64_t S = int64_t(1) << P.sliced.size();
    for (int64_t i = 0; i < n_slices; ++i)
      TN_CHECK(slice_ids[i] >= 0 && slice_ids[i] < S, TN_ERR_INVALID_ARG, "slice id out of range");
    cudaStream_t s = (cudaStream_t)stream;
    void* ws = static_workspace();
    if (n_slices == 0) {
      if (!accumulate) TN_CUDA(cudaMemsetAsync(amps, 0, (size_t)(P.G * P.J * 16), s));
      return;
    }
    std::vector<int64_t> chunk(P.B);
    for (int64_t start = 0; start < n_slices; start += P.B) {
      int32_t nv = (int32_t)std::min<int64_t>(P.B, n_slices - start);
      for (int b = 0; b < P.B; ++b) chunk[b] = slice_ids[start + (b < nv ? b : 0)];
      // pageable host -> device: the runtime stages the source before returning
      launch_set_slice_ids(P.d_slice_ids, P.d_n_valid, chunk.data(), P.B, nv, s);
      run_batch_direct(P, ws, amps, start == 0 ? accumulate : 1, s);
    }
    TN_CUDA(cudaGetLastError());
  });
}
