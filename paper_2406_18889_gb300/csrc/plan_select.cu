// Plan creation choices that need measurements or several candidate plans:
//  * the slice batch from the memory budget (max_slice_batch = 0);
//  * the placement of split-precision (hi + lo) products (TN_FLAG_HILO_AUTO):
//    hi + lo only on the contractions whose 16-bit error measurably moves
//    the result.  Each candidate placement is a plan
//    of its own; the calibration slices are contracted once in complex64 and
//    once per candidate, and the relative L2 of the 16-bit amplitudes against
//    the complex64 ones decides.
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <string>

#include "plan.h"

namespace tn {

namespace {

constexpr int kErrBlocks = 152;
constexpr int kErrThreads = 256;

// Partial sums of |a - r|^2 and |r|^2 over a grid-stride share, reduced in a
// fixed order inside the block; out[2 b], out[2 b + 1] for block b.
__global__ void rel_l2_kernel(const double2* __restrict__ a, const double2* __restrict__ r, int64_t n,
                              double* __restrict__ out) {
  double d = 0.0, q = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 x = a[i], y = r[i];
    const double dx = x.x - y.x, dy = x.y - y.y;
    d += dx * dx + dy * dy;
    q += y.x * y.x + y.y * y.y;
  }
  __shared__ double sd[kErrThreads], sq[kErrThreads];
  sd[threadIdx.x] = d;
  sq[threadIdx.x] = q;
  __syncthreads();
  for (int o = kErrThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sd[threadIdx.x] += sd[threadIdx.x + o];
      sq[threadIdx.x] += sq[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = sd[0];
    out[2 * blockIdx.x + 1] = sq[0];
  }
}

// device buffer owned by the selection (freed on every exit path)
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  void reserve(size_t b) {
    if (b <= bytes) return;
    if (p) TN_CUDA(cudaFree(p));
    p = nullptr;
    bytes = 0;
    TN_CUDA(cudaMalloc(&p, std::max<size_t>(b, 256)));
    bytes = b;
  }
};

int64_t memory_need(const Plan& Q) {
  return std::max<int64_t>(Q.mem.plan_bytes + Q.mem.ws_bytes, Q.calib_bytes);
}

// Largest power-of-two slice batch whose device memory fits the budget.
int choose_slice_batch(const tn_network_desc* net, const tn_tree_desc* tree, const tn_plan_options& opt,
                       cudaStream_t stream) {
  TN_CHECK(tree != nullptr, TN_ERR_INVALID_ARG, "null descriptor");
  int64_t cap = opt.mem_cap_bytes;
  if (cap <= 0) {
    TN_CHECK(!(opt.flags & TN_FLAG_PLAN_ONLY), TN_ERR_INVALID_ARG,
             "max_slice_batch = 0 on a plan-only plan needs mem_cap_bytes > 0");
    size_t fr = 0, tot = 0;
    TN_CUDA(cudaMemGetInfo(&fr, &tot));
    cap = (int64_t)(fr / 2);
  }
  const int top = std::min(std::max(tree->n_sliced, 0), 16);
  tn_plan_options o = opt;
  o.flags |= TN_FLAG_PLAN_ONLY;
  o.mem_cap_bytes = 0;  // probes are measured, not rejected
  // the automatic split placement is an upper bound when every step is split
  if (o.flags & TN_FLAG_HILO_AUTO) o.flags = (o.flags & ~TN_FLAG_HILO_AUTO) | TN_FLAG_HILO;
  for (int lb = top; lb >= 1; --lb) {
    o.max_slice_batch = 1 << lb;
    auto q = build_plan(net, tree, &o, stream);
    if (memory_need(*q) <= cap) return 1 << lb;
  }
  return 1;
}

// Contract a plan's calibration batch into `amps` (direct launches).
void run_calibration(Plan& Q, DevBuf& ws, void* amps, cudaStream_t s) {
  ws.reserve((size_t)std::max<int64_t>(Q.mem.ws_bytes, 256));
  std::vector<int64_t> ids = calibration_ids(Q.B, (int)Q.sliced.size());
  launch_set_slice_ids(Q.d_slice_ids, Q.d_n_valid, ids.data(), Q.B, Q.B, s);
  run_batch_direct(Q, ws.p, amps, 0, s);
}

double relative_l2(const void* a, const void* r, int64_t n, DevBuf& part, cudaStream_t s) {
  part.reserve(sizeof(double) * 2 * kErrBlocks);
  rel_l2_kernel<<<kErrBlocks, kErrThreads, 0, s>>>((const double2*)a, (const double2*)r, n, (double*)part.p);
  TN_CUDA(cudaGetLastError());
  std::vector<double> h(2 * kErrBlocks);
  TN_CUDA(cudaMemcpyAsync(h.data(), part.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
  TN_CUDA(cudaStreamSynchronize(s));
  double d = 0.0, q = 0.0;
  for (int b = 0; b < kErrBlocks; ++b) {
    d += h[2 * b];
    q += h[2 * b + 1];
  }
  TN_CHECK(std::isfinite(d) && std::isfinite(q), TN_ERR_NUMERIC, "calibration amplitudes are not finite");
  return q > 0 ? std::sqrt(d / q) : std::sqrt(d);
}

void check_timeouts(const Plan& Q, cudaStream_t s) {
  TN_CUDA(cudaStreamSynchronize(s));
  int h_err = 0;
  TN_CUDA(cudaMemcpy(&h_err, Q.d_err, sizeof(int), cudaMemcpyDeviceToHost));
  TN_CHECK(h_err == 0, TN_ERR_TIMEOUT, "a bounded device wait timed out during the split-precision selection");
}

}  // namespace

std::unique_ptr<Plan> create_plan(const tn_network_desc* net, const tn_tree_desc* tree, const tn_plan_options* opt_in,
                                  cudaStream_t stream) {
  TN_CHECK(net && tree && opt_in, TN_ERR_INVALID_ARG, "null descriptor");
  tn_plan_options opt = *opt_in;
  const bool autohl = (opt.flags & TN_FLAG_HILO_AUTO) != 0;
  TN_CHECK(!(opt.hilo_steps && (opt.flags & (TN_FLAG_HILO | TN_FLAG_HILO_AUTO))), TN_ERR_INVALID_ARG,
           "hilo_steps is not combined with TN_FLAG_HILO or TN_FLAG_HILO_AUTO");
  TN_CHECK(!(autohl && (opt.flags & TN_FLAG_HILO)), TN_ERR_INVALID_ARG,
           "TN_FLAG_HILO_AUTO is not combined with TN_FLAG_HILO");
  TN_CHECK(opt.hilo_tol == 0.0 || (opt.hilo_tol > 0.0 && opt.hilo_tol < 1.0), TN_ERR_INVALID_ARG,
           "hilo_tol must lie in (0, 1), or be 0");
  TN_CHECK(opt.max_slice_batch >= 0, TN_ERR_INVALID_ARG, "max_slice_batch < 0");
  TN_CHECK(tree->n_steps >= 0, TN_ERR_INVALID_ARG, "n_steps < 0");
  if (opt.max_slice_batch == 0) opt.max_slice_batch = choose_slice_batch(net, tree, opt, stream);
  std::vector<char> mask;
  if (opt.hilo_steps) {
    for (int t = 0; t < tree->n_steps; ++t)
      TN_CHECK(opt.hilo_steps[t] <= 1, TN_ERR_INVALID_ARG, "hilo_steps entries must be 0 or 1");
    mask.assign(opt.hilo_steps, opt.hilo_steps + tree->n_steps);
    return build_plan(net, tree, &opt, stream, &mask);
  }
  if (!autohl || opt.prec == TN_PREC_C64 || (opt.flags & TN_FLAG_PLAN_ONLY)) {
    // a plan-only or complex64 plan makes no split (nothing to measure)
    if (autohl) {
      mask.assign(tree->n_steps, 0);
      return build_plan(net, tree, &opt, stream, &mask);
    }
    return build_plan(net, tree, &opt, stream);
  }

  // ---- TN_FLAG_HILO_AUTO
  const double tol = opt.hilo_tol > 0 ? opt.hilo_tol : 3e-3;
  tn_plan_options o = opt;  // candidates: direct launches, placement by mask
  o.flags = (o.flags & ~TN_FLAG_HILO_AUTO) | TN_FLAG_NO_GRAPH;
  DevBuf ws, ref, amps, part;
  int64_t n_amps = 0;
  {
    tn_plan_options oc = o;
    oc.prec = TN_PREC_C64;
    auto R = build_plan(net, tree, &oc, stream);
    n_amps = R->G * R->J;
    ref.reserve((size_t)n_amps * 16);
    amps.reserve((size_t)n_amps * 16);
    run_calibration(*R, ws, ref.p, stream);
    check_timeouts(*R, stream);
  }
  // tensor-core steps, in split groups (steps linked through a stored 16-bit
  // operand split together; build_plan enforces it)
  std::vector<std::vector<int>> groups;
  auto measure = [&](const std::vector<char>& m) {
    auto Q = build_plan(net, tree, &o, stream, &m);
    if (groups.empty()) {
      std::map<int, std::vector<int>> g;
      for (size_t t = 0; t < Q->steps.size(); ++t)
        if (Q->steps[t].tc) g[Q->steps[t].hilo_group].push_back((int)t);
      for (auto& kv : g) groups.push_back(kv.second);
    }
    run_calibration(*Q, ws, amps.p, stream);
    check_timeouts(*Q, stream);
    return relative_l2(amps.p, ref.p, n_amps, part, stream);
  };
  const int T = tree->n_steps;
  auto set_group = [&](std::vector<char>& m, int gi, char v) {
    for (int t : groups[gi]) m[t] = v;
  };
  std::vector<char> chosen(T, 0);
  const double e_none = measure(chosen);
  double e_chosen = e_none;
  const int NG = (int)groups.size();
  if (e_none > tol && NG > 0) {
    std::vector<char> all(T, 0);
    for (int gi = 0; gi < NG; ++gi) set_group(all, gi, 1);
    const double e_all = measure(all);
    // each group's share of the squared error: the error with that group alone
    // left unsplit, above the all-split floor (errors of independent roundings
    // add in quadrature)
    std::vector<double> share(NG, 0.0);
    for (int gi = 0; gi < NG; ++gi) {
      std::vector<char> m = all;
      set_group(m, gi, 0);
      const double e = measure(m);
      share[gi] = std::max(0.0, e * e - e_all * e_all);
    }
    std::vector<int> order(NG);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return share[a] > share[b]; });
    // smallest prefix whose estimated error is within 0.8 tol
    double est = e_all * e_all;
    for (int gi = 0; gi < NG; ++gi) est += share[gi];
    size_t take = 0;
    const double target = (0.8 * tol) * (0.8 * tol);
    while (take < order.size() && est > target) {
      est -= share[order[take]];
      set_group(chosen, order[take], 1);
      ++take;
    }
    // verify, adding the next-largest shares while the measured error is above tol
    e_chosen = measure(chosen);
    while (e_chosen > tol && take < order.size()) {
      set_group(chosen, order[take], 1);
      ++take;
      e_chosen = measure(chosen);
    }
  }
  tn_plan_options of = opt;  // final plan: the caller's flags (graph replay etc.)
  of.flags &= ~TN_FLAG_HILO_AUTO;
  auto P = build_plan(net, tree, &of, stream, &chosen);
  P->flags |= TN_FLAG_HILO_AUTO;
  P->calib_err_chosen = e_chosen;
  P->calib_err_none = e_none;
  return P;
}

}  // namespace tn
