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

tn_status guarded_call(const std::function<void()>& f);

}  // namespace tn

extern "C" tn_status tn_contract_slices_noalloc(tn_plan_t plan, const int64_t* slice_ids, int64_t n_slices,
                                                void* amps, int accumulate, void* stream) {
  using namespace tn;
  return guarded_call([&] {
    TN_CHECK(plan != nullptr, TN_ERR_INVALID_ARG, "plan is null");
    Plan& P = *plan->p;
    TN_CHECK(!(P.flags & TN_FLAG_PLAN_ONLY), TN_ERR_INVALID_ARG, "plan was created with TN_FLAG_PLAN_ONLY");
    // the static array of the plan's device: that device must be current
    int dev = -1;
    TN_CUDA(cudaGetDevice(&dev));
    TN_CHECK(dev == P.device, TN_ERR_INVALID_ARG,
             "the plan lives on device " + std::to_string(P.device) + " but device " + std::to_string(dev) +
                 " is current");
    TN_CHECK(P.mem.ws_bytes <= (int64_t)TN_STATIC_WORKSPACE_BYTES, TN_ERR_INVALID_ARG,
             "plan needs " + std::to_string(P.mem.ws_bytes) + " bytes of workspace; the static workspace holds " +
                 std::to_string((long long)TN_STATIC_WORKSPACE_BYTES) +
                 " (use tn_contract_slices or a smaller max_slice_batch)");
    void* ws = static_workspace();
    // the same argument checks, fault injection and batching as tn_contract_slices;
    // each batch's ids reach the device as kernel arguments (no staging copy),
    // and the batch is launched directly (no graph is instantiated)
    contract_checked(P, slice_ids, n_slices, amps, accumulate, ws, (size_t)TN_STATIC_WORKSPACE_BYTES,
                     (cudaStream_t)stream, [](Plan& Q, void* w, void* a, int acc, cudaStream_t st) {
                       run_batch_direct(Q, w, a, acc, st);
                     });
  });
}
