// The C ABI declared in include/tn.h.  Validation happens before any device
// work; no C++ exception crosses the boundary.
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include "plan.h"

struct tn_plan_s {
  std::unique_ptr<tn::Plan> p;
};

namespace tn {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

struct Failure {
  tn_status code;
  std::string msg;
};

[[noreturn]] void fail(tn_status code, const std::string& msg) { throw Failure{code, msg}; }

template <class F>
static tn_status guarded(F&& f) {
  try {
    f();
    g_last_error.clear();
    return TN_OK;
  } catch (const Failure& e) {
    g_last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return TN_ERR_OOM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return TN_ERR_INVALID_ARG;
  } catch (...) {
    g_last_error = "unknown failure";
    return TN_ERR_INVALID_ARG;
  }
}

// Run f under the same error handling as the C entry points (used by
// entry points defined in other translation units).
tn_status guarded_call(const std::function<void()>& f) { return guarded(f); }

// 256 bytes of device memory per host thread and device for small results the
// host reads back within the same call (a flag, a scalar).  Allocated once,
// outside any stream-ordered pool (whose memory may be handed back to the
// driver at every synchronisation), and kept for the process's lifetime.
static void* thread_scratch() {
  thread_local std::map<int, void*> by_dev;
  int dev = 0;
  TN_CUDA(cudaGetDevice(&dev));
  auto it = by_dev.find(dev);
  if (it != by_dev.end()) return it->second;
  void* p = nullptr;
  TN_CUDA(cudaMalloc(&p, 256));
  by_dev[dev] = p;
  return p;
}

// TN_FAULT=<what>: host-side fault injection, checked before any device work
static bool fault_injected(const char* what) {
  const char* v = getenv("TN_FAULT");
  return v && strcmp(v, what) == 0;
}

void contract_checked(Plan& P, const int64_t* ids, int64_t n, void* amps, int accumulate, void* ws,
                      size_t ws_bytes, cudaStream_t s, const BatchRunner& run) {
  TN_CHECK(!(P.flags & TN_FLAG_PLAN_ONLY), TN_ERR_INVALID_ARG, "plan was created with TN_FLAG_PLAN_ONLY");
  TN_CHECK(!fault_injected("stream"), TN_ERR_CUDA, "injected stream failure (TN_FAULT=stream)");
  {
    int dev = -1;
    TN_CUDA(cudaGetDevice(&dev));
    TN_CHECK(dev == P.device, TN_ERR_INVALID_ARG,
             "the plan lives on device " + std::to_string(P.device) + " but device " + std::to_string(dev) +
                 " is current");
  }
  TN_CHECK(amps != nullptr, TN_ERR_INVALID_ARG, "amps is null");
  TN_CHECK(n >= 0, TN_ERR_INVALID_ARG, "n_slices < 0");
  TN_CHECK(n == 0 || ids != nullptr, TN_ERR_INVALID_ARG, "slice_ids is null");
  TN_CHECK(accumulate == 0 || accumulate == 1, TN_ERR_INVALID_ARG, "accumulate must be 0 or 1");
  const int64_t S = int64_t(1) << P.sliced.size();
  for (int64_t i = 0; i < n; ++i)
    TN_CHECK(ids[i] >= 0 && ids[i] < S, TN_ERR_INVALID_ARG, "slice id out of range");
  if (n > 0) {
    TN_CHECK(ws != nullptr && (reinterpret_cast<uintptr_t>(ws) & 255) == 0, TN_ERR_INVALID_ARG,
             "workspace must be non-null and 256-byte aligned");
    TN_CHECK((int64_t)ws_bytes >= P.mem.ws_bytes, TN_ERR_INVALID_ARG, "workspace too small");
  }
  if (n == 0) {
    if (!accumulate) launch_zero(amps, (size_t)(P.G * P.J * 16), s);
    TN_CUDA(cudaGetLastError());
    return;
  }
  std::vector<int64_t> chunk(P.B);
  for (int64_t start = 0; start < n; start += P.B) {
    int32_t nv = (int32_t)std::min<int64_t>(P.B, n - start);
    for (int b = 0; b < P.B; ++b) chunk[b] = ids[start + (b < nv ? b : 0)];
    launch_set_slice_ids(P.d_slice_ids, P.d_n_valid, chunk.data(), P.B, nv, s);
    run(P, ws, amps, start == 0 ? accumulate : 1, s);
  }
  TN_CUDA(cudaGetLastError());
}

static void contract_one(Plan& P, const int64_t* ids, int64_t n, void* amps, int accumulate, void* ws,
                         size_t ws_bytes, cudaStream_t s, std::vector<LaunchRecord>* rec = nullptr) {
  contract_checked(P, ids, n, amps, accumulate, ws, ws_bytes, s,
                   [rec](Plan& Q, void* w, void* a, int acc, cudaStream_t st) { run_batch(Q, w, a, acc, st, rec); });
}

}  // namespace tn

using namespace tn;

extern "C" {

tn_status tn_plan_create(const tn_network_desc* net, const tn_tree_desc* tree, const tn_plan_options* opt,
                         void* stream, tn_plan_t* out) {
  return guarded([&] {
    TN_CHECK(out != nullptr, TN_ERR_INVALID_ARG, "out is null");
    TN_CHECK(!fault_injected("alloc"), TN_ERR_OOM, "injected allocation failure (TN_FAULT=alloc)");
    TN_CHECK(!fault_injected("invalid_plan"), TN_ERR_INVALID_ARG, "injected invalid plan (TN_FAULT=invalid_plan)");
    auto p = create_plan(net, tree, opt, (cudaStream_t)stream);
    auto* h = new tn_plan_s{std::move(p)};
    *out = h;
  });
}

tn_status tn_plan_destroy(tn_plan_t plan) {
  return guarded([&] {
    TN_CHECK(plan != nullptr, TN_ERR_INVALID_ARG, "plan is null");
    delete plan;
  });
}

tn_status tn_plan_slice_batch(tn_plan_t plan, int32_t* batch) {
  return guarded([&] {
    TN_CHECK(plan != nullptr && batch != nullptr, TN_ERR_INVALID_ARG, "null pointer");
    *batch = plan->p->B;
  });
}

tn_status tn_plan_precision(tn_plan_t plan, double* rel_l2_chosen, double* rel_l2_none, int32_t* n_tc_steps,
                            int32_t* n_hilo_steps) {
  return guarded([&] {
    TN_CHECK(plan != nullptr, TN_ERR_INVALID_ARG, "plan is null");
    const Plan& P = *plan->p;
    int32_t tc = 0, hl = 0;
    for (const Step& S : P.steps) {
      tc += S.tc ? 1 : 0;
      hl += (S.tc && S.hilo) ? 1 : 0;
    }
    if (rel_l2_chosen) *rel_l2_chosen = P.calib_err_chosen;
    if (rel_l2_none) *rel_l2_none = P.calib_err_none;
    if (n_tc_steps) *n_tc_steps = tc;
    if (n_hilo_steps) *n_hilo_steps = hl;
  });
}

tn_status tn_plan_query(tn_plan_t plan, int64_t* flops, int64_t* bytes, int64_t* peak, int64_t* ws) {
  return guarded([&] {
    TN_CHECK(plan != nullptr, TN_ERR_INVALID_ARG, "plan is null");
    const Plan& P = *plan->p;
    if (flops) *flops = (int64_t)P.useful_flops_per_slice;
    if (bytes) *bytes = (int64_t)P.algo_bytes_per_slice;
    if (peak) *peak = (int64_t)P.peak_intermediate_bytes;
    if (ws) *ws = P.mem.ws_bytes;
  });
}

tn_status tn_plan_steps(tn_plan_t plan, int32_t max_steps, int64_t* batch, int64_t* m, int64_t* n,
                        int64_t* k, int32_t* kinds, int32_t* n_steps_out) {
  return guarded([&] {
    TN_CHECK(plan != nullptr, TN_ERR_INVALID_ARG, "plan is null");
    const Plan& P = *plan->p;
    if (n_steps_out) *n_steps_out = (int32_t)P.steps.size();
    TN_CHECK(max_steps >= 0, TN_ERR_INVALID_ARG, "max_steps < 0");
    int cnt = std::min<int>(max_steps, (int)P.steps.size());
    for (int t = 0; t < cnt; ++t) {
      const Step& S = P.steps[t];
      if (batch) batch[t] = S.gp.nbt;
      if (m) m[t] = S.gp.M;
      if (n) n[t] = S.gp.N;
      if (k) k[t] = S.gp.K;
      if (kinds) kinds[t] = (S.variant ? 1 : 0) | (S.post_perm ? 2 : 0) | (S.hoisted ? 4 : 0) | (S.tc ? 8 : 0) |
                               (S.hilo ? 16 : 0) | (S.fuse_expand ? 32 : 0) | (S.b_fused ? 64 : 0) |
                               (S.micro ? 128 : 0) | (S.pair_rows ? 256 : 0);
    }
  });
}

tn_status tn_plan_autotune(tn_plan_t plan, const int64_t* slice_ids, int64_t n_slices, void* amps,
                           void* workspace, size_t ws_bytes, void* stream, int32_t reps, int32_t* forms) {
  std::vector<LaunchRecord> rec;
  auto free_rec = [&] {
    for (auto& r : rec) {
      if (r.start) cudaEventDestroy(r.start);
      if (r.stop) cudaEventDestroy(r.stop);
    }
    rec.clear();
  };
  std::vector<TcForm> saved;
  Plan* Pp = nullptr;
  tn_status st = guarded([&] {
    TN_CHECK(plan != nullptr, TN_ERR_INVALID_ARG, "plan is null");
    Plan& P = *plan->p;
    Pp = &P;
    TN_CHECK(!(P.flags & TN_FLAG_PLAN_ONLY), TN_ERR_INVALID_ARG, "plan was created with TN_FLAG_PLAN_ONLY");
    TN_CHECK(n_slices >= 1 && n_slices <= P.B, TN_ERR_INVALID_ARG, "n_slices must be 1 .. the slice batch");
    TN_CHECK(reps >= 1 && reps <= 64, TN_ERR_INVALID_ARG, "reps must be 1 .. 64");
    const size_t T = P.steps.size();
    for (size_t t = 0; t < T; ++t) saved.push_back({P.steps[t].tc_bn, P.steps[t].tc_mh});
    // the tuned steps in launch order (the order of their profiling records)
    std::vector<size_t> tuned;
    std::vector<std::vector<TcForm>> cand;
    size_t most = 0;
    for (size_t t = 0; t < T; ++t) {
      std::vector<TcForm> f = tc_step_forms(P, t);
      if (f.empty()) continue;
      tuned.push_back(t);
      most = std::max(most, f.size());
      cand.push_back(std::move(f));
    }
    std::vector<float> best(tuned.size(), 3.0e38f);
    std::vector<TcForm> pick(tuned.size());
    cudaStream_t s = (cudaStream_t)stream;
    for (size_t c = 0; c < most; ++c) {
      for (size_t i = 0; i < tuned.size(); ++i) {
        const TcForm& f = cand[i][std::min(c, cand[i].size() - 1)];
        Step& S = P.steps[tuned[i]];
        S.tc_bn = f.bn;
        S.tc_mh = f.mh;
      }
      for (int r = 0; r < reps; ++r) {
        contract_one(P, slice_ids, n_slices, amps, 0, workspace, ws_bytes, s, &rec);
        TN_CUDA(cudaStreamSynchronize(s));
        int h_err = 0;
        TN_CUDA(cudaMemcpy(&h_err, P.d_err, sizeof(int), cudaMemcpyDeviceToHost));
        TN_CHECK(h_err == 0, TN_ERR_TIMEOUT, "a bounded device wait timed out");
        size_t i = 0;
        for (const LaunchRecord& L : rec) {
          if (L.kind != 5) continue;
          TN_CHECK(i < tuned.size(), TN_ERR_INVALID_ARG, "internal: tensor-core launch count");
          float ms = 0.f;
          TN_CUDA(cudaEventElapsedTime(&ms, L.start, L.stop));
          if (ms < best[i]) {
            best[i] = ms;
            pick[i] = cand[i][std::min(c, cand[i].size() - 1)];
          }
          ++i;
        }
        TN_CHECK(i == tuned.size(), TN_ERR_INVALID_ARG, "internal: tensor-core launch count");
        free_rec();
      }
    }
    for (size_t i = 0; i < tuned.size(); ++i) {
      Step& S = P.steps[tuned[i]];
      S.tc_bn = pick[i].bn;
      S.tc_mh = pick[i].mh;
    }
    drop_graph(P);
    if (forms) {
      for (size_t t = 0; t < T; ++t) {
        forms[2 * t] = P.steps[t].tc_bn;
        forms[2 * t + 1] = P.steps[t].tc_mh;
      }
    }
  });
  free_rec();
  if (st != TN_OK && Pp && saved.size() == Pp->steps.size()) {
    // keep the forms the plan had before the call
    for (size_t t = 0; t < saved.size(); ++t) {
      Pp->steps[t].tc_bn = saved[t].bn;
      Pp->steps[t].tc_mh = saved[t].mh;
    }
    drop_graph(*Pp);
  }
  return st;
}

tn_status tn_plan_set_tuning(tn_plan_t plan, const int32_t* forms, int32_t n_steps) {
  return guarded([&] {
    TN_CHECK(plan != nullptr, TN_ERR_INVALID_ARG, "plan is null");
    Plan& P = *plan->p;
    TN_CHECK(forms != nullptr, TN_ERR_INVALID_ARG, "forms is null");
    TN_CHECK(n_steps == (int32_t)P.steps.size(), TN_ERR_INVALID_ARG, "n_steps differs from the plan's step count");
    for (int32_t t = 0; t < n_steps; ++t) {
      const int32_t bn = forms[2 * t], mh = forms[2 * t + 1];
      if (bn == 0 && mh == 0) continue;
      bool ok = false;
      for (const TcForm& f : tc_step_forms(P, (size_t)t)) ok = ok || (f.bn == bn && f.mh == mh);
      TN_CHECK(ok, TN_ERR_INVALID_ARG, "step " + std::to_string(t) + ": not a launch form of this step");
    }
    for (int32_t t = 0; t < n_steps; ++t) {
      Step& S = P.steps[t];
      S.tc_bn = forms[2 * t];
      S.tc_mh = forms[2 * t + 1];
    }
    drop_graph(P);
  });
}

tn_status tn_contract_slices(tn_plan_t plan, const int64_t* slice_ids, int64_t n_slices, void* amps,
                             int accumulate, void* workspace, size_t ws_bytes, void* stream) {
  return guarded([&] {
    TN_CHECK(plan != nullptr, TN_ERR_INVALID_ARG, "plan is null");
    contract_one(*plan->p, slice_ids, n_slices, amps, accumulate, workspace, ws_bytes, (cudaStream_t)stream);
  });
}

tn_status tn_contract_slices_batched(const tn_plan_t* plans, int32_t n_plans, const int64_t* const* slice_ids,
                                     const int64_t* n_slices, void* const* amps, int accumulate,
                                     void* workspace, size_t ws_bytes, void* stream) {
  return guarded([&] {
    TN_CHECK(n_plans >= 0, TN_ERR_INVALID_ARG, "n_plans < 0");
    TN_CHECK(n_plans == 0 || (plans && slice_ids && n_slices && amps), TN_ERR_INVALID_ARG, "null array");
    TN_CHECK(!fault_injected("stream"), TN_ERR_CUDA, "injected stream failure (TN_FAULT=stream)");
    TN_CHECK(accumulate == 0 || accumulate == 1, TN_ERR_INVALID_ARG, "accumulate must be 0 or 1");
    // validate every plan's arguments before queuing any work
    std::vector<Plan*> ps;
    for (int32_t i = 0; i < n_plans; ++i) {
      TN_CHECK(plans[i] != nullptr, TN_ERR_INVALID_ARG, "plan is null");
      Plan& P = *plans[i]->p;
      TN_CHECK(!(P.flags & TN_FLAG_PLAN_ONLY), TN_ERR_INVALID_ARG, "plan was created with TN_FLAG_PLAN_ONLY");
      TN_CHECK(amps[i] != nullptr, TN_ERR_INVALID_ARG, "amps is null");
      TN_CHECK(n_slices[i] >= 0 && (n_slices[i] == 0 || slice_ids[i]), TN_ERR_INVALID_ARG, "bad slice list");
      const int64_t S = int64_t(1) << P.sliced.size();
      for (int64_t j = 0; j < n_slices[i]; ++j)
        TN_CHECK(slice_ids[i][j] >= 0 && slice_ids[i][j] < S, TN_ERR_INVALID_ARG, "slice id out of range");
      ps.push_back(&P);
    }
    if (n_plans == 0) return;
    TN_CHECK(workspace != nullptr && (reinterpret_cast<uintptr_t>(workspace) & 255) == 0, TN_ERR_INVALID_ARG,
             "workspace must be non-null and 256-byte aligned");
    TN_CHECK(batched_layout(ps, n_slices, ws_bytes, 8).bytes <= (int64_t)ws_bytes, TN_ERR_INVALID_ARG,
             "workspace too small");
    contract_batched(ps, slice_ids, n_slices, amps, accumulate, workspace, ws_bytes, (cudaStream_t)stream);
  });
}

tn_status tn_batched_workspace_bytes(const tn_plan_t* plans, int32_t n_plans, const int64_t* n_slices,
                                     int32_t max_branches, int64_t* bytes) {
  return guarded([&] {
    TN_CHECK(n_plans >= 0 && (n_plans == 0 || (plans && n_slices)) && bytes, TN_ERR_INVALID_ARG, "null array");
    TN_CHECK(max_branches >= 1, TN_ERR_INVALID_ARG, "max_branches must be >= 1");
    std::vector<Plan*> ps;
    for (int32_t i = 0; i < n_plans; ++i) {
      TN_CHECK(plans[i] != nullptr && n_slices[i] >= 0, TN_ERR_INVALID_ARG, "bad plan or slice count");
      ps.push_back(plans[i]->p.get());
    }
    *bytes = n_plans == 0 ? 0 : batched_layout(ps, n_slices, (size_t)INT64_MAX, max_branches).bytes;
  });
}

tn_status tn_sum_partials(const void* parts, int64_t n_parts, int64_t n_amps, void* out, int accumulate,
                          void* stream) {
  return guarded([&] {
    TN_CHECK(n_parts >= 0 && n_amps >= 0, TN_ERR_INVALID_ARG, "negative count");
    TN_CHECK(out != nullptr && (n_parts == 0 || parts != nullptr), TN_ERR_INVALID_ARG, "null pointer");
    TN_CHECK(accumulate == 0 || accumulate == 1, TN_ERR_INVALID_ARG, "accumulate must be 0 or 1");
    TN_CHECK(n_parts <= (int64_t(1) << 40) / std::max<int64_t>(n_amps, 1), TN_ERR_INVALID_ARG, "too many elements");
    launch_sum_partials(parts, n_parts, n_amps, out, accumulate, (cudaStream_t)stream);
    TN_CUDA(cudaGetLastError());
  });
}

tn_status tn_topk_postprocess(const void* amps, int64_t G, int64_t B, int32_t k, double inv_f, int global_mode,
                              const int64_t* block_base_idx, const int64_t* open_bit_pos, int32_t l,
                              int64_t* out_idx, double* out_p, void* stream) {
  return guarded([&] {
    TN_CHECK(amps && block_base_idx && out_idx && out_p, TN_ERR_INVALID_ARG, "null pointer");
    TN_CHECK(global_mode == 0 || global_mode == 1, TN_ERR_INVALID_ARG, "global_mode must be 0 or 1");
    // per block: B <= 2^16, k <= 512; global: G * B <= 2^40 candidates, k <= 2^26
    const int max_l = global_mode ? 40 : 16;
    TN_CHECK(G >= 1 && B >= 1 && l >= 0 && l <= max_l && (int64_t(1) << l) == B, TN_ERR_INVALID_ARG,
             "bad G or B (B must equal 2^l)");
    TN_CHECK(l == 0 || open_bit_pos, TN_ERR_INVALID_ARG, "open_bit_pos is null");
    TN_CHECK(!global_mode || G <= (int64_t(1) << 40) / B, TN_ERR_INVALID_ARG, "too many candidates");
    TN_CHECK(k >= 1 && k <= (global_mode ? (1 << 26) : 512) && k <= (global_mode ? G * B : B), TN_ERR_INVALID_ARG,
             "k out of range");
    TN_CHECK(global_mode || G <= 0x7fffffff, TN_ERR_INVALID_ARG, "too many blocks");
    TN_CHECK(inv_f > 0 && inv_f == inv_f, TN_ERR_INVALID_ARG, "inv_f must be positive");
    TopkParams tp{};
    tp.G = G;
    tp.Bsz = B;
    tp.k = k;
    tp.l = l;
    tp.global_mode = global_mode;
    tp.inv_f = inv_f;
    for (int i = 0; i < l; ++i) {
      TN_CHECK(open_bit_pos[i] >= 0 && open_bit_pos[i] < 63, TN_ERR_INVALID_ARG, "open bit position out of range");
      tp.open_pos[i] = (int8_t)open_bit_pos[i];
    }
    cudaStream_t s = (cudaStream_t)stream;
    int* d_flag = reinterpret_cast<int*>(thread_scratch());
    TN_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), s));
    if (global_mode)
      topk_global((const double2*)amps, tp, block_base_idx, out_idx, out_p, d_flag, s);
    else
      launch_topk((const double2*)amps, tp, block_base_idx, out_idx, out_p, d_flag, s);
    int h_flag = 0;
    TN_CUDA(cudaMemcpyAsync(&h_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    TN_CUDA(cudaStreamSynchronize(s));
    TN_CHECK(h_flag == 0, TN_ERR_NUMERIC, "NaN probability in top-k input");
  });
}

tn_status tn_xeb(const double* q, int64_t n_sel, int32_t n_qubits, double* out_xeb, void* stream) {
  return guarded([&] {
    TN_CHECK(q && out_xeb, TN_ERR_INVALID_ARG, "null pointer");
    TN_CHECK(n_sel >= 1, TN_ERR_INVALID_ARG, "empty selection");
    TN_CHECK(n_qubits >= 1 && n_qubits <= 1000, TN_ERR_INVALID_ARG, "n_qubits out of range");
    cudaStream_t s = (cudaStream_t)stream;
    double* d_out = reinterpret_cast<double*>(reinterpret_cast<char*>(thread_scratch()) + 64);
    launch_xeb(q, n_sel, n_qubits, d_out, s);
    TN_CUDA(cudaMemcpyAsync(out_xeb, d_out, sizeof(double), cudaMemcpyDeviceToHost, s));
    TN_CUDA(cudaStreamSynchronize(s));
  });
}

tn_status tn_contract_slices_profile(tn_plan_t plan, const int64_t* slice_ids, int64_t n_slices, void* amps,
                                     int accumulate, void* workspace, size_t ws_bytes, void* stream,
                                     int32_t max_records, int32_t* kind, float* ms, double* flops,
                                     double* bytes, int32_t* n_records) {
  std::vector<LaunchRecord> rec;
  tn_status st = guarded([&] {
    TN_CHECK(plan != nullptr, TN_ERR_INVALID_ARG, "plan is null");
    TN_CHECK(max_records >= 0 && (max_records == 0 || (kind && ms && flops && bytes)), TN_ERR_INVALID_ARG,
             "null record array");
    cudaStream_t s = (cudaStream_t)stream;
    contract_one(*plan->p, slice_ids, n_slices, amps, accumulate, workspace, ws_bytes, s, &rec);
    TN_CUDA(cudaStreamSynchronize(s));
    int h_err = 0;
    TN_CUDA(cudaMemcpy(&h_err, plan->p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    TN_CHECK(h_err == 0, TN_ERR_TIMEOUT, "a bounded device wait timed out");
    if (n_records) *n_records = (int32_t)rec.size();
    for (int32_t i = 0; i < (int32_t)rec.size() && i < max_records; ++i) {
      kind[i] = rec[i].kind;
      flops[i] = rec[i].flops;
      bytes[i] = rec[i].bytes;
      float t = 0.f;
      TN_CUDA(cudaEventElapsedTime(&t, rec[i].start, rec[i].stop));
      ms[i] = t;
    }
  });
  for (auto& r : rec) {
    if (r.start) cudaEventDestroy(r.start);
    if (r.stop) cudaEventDestroy(r.stop);
  }
  return st;
}

tn_status tn_selftest_bounded_wait(uint64_t limit_ns, void* stream) {
  bool timed_out = false;
  tn_status st = guarded([&] {
    TN_CHECK(limit_ns >= 1000 && limit_ns <= 1000000000ull, TN_ERR_INVALID_ARG, "limit_ns out of range");
    timed_out = selftest_bounded_wait(limit_ns, (cudaStream_t)stream);
  });
  if (st != TN_OK) return st;
  if (timed_out) {
    set_error("bounded wait gave up (expected)");
    return TN_ERR_TIMEOUT;
  }
  return TN_OK;
}

tn_status tn_selftest_fp32_peak(double* tflops, void* stream) {
  return guarded([&] {
    TN_CHECK(tflops != nullptr, TN_ERR_INVALID_ARG, "tflops is null");
    *tflops = selftest_fp32_peak((cudaStream_t)stream);
  });
}

tn_status tn_selftest_gemm_tc(int64_t nbt, int64_t M, int64_t N, int64_t K, int32_t prec, uint64_t seed,
                              double* max_rel_err, void* stream) {
  return guarded([&] {
    TN_CHECK(max_rel_err != nullptr, TN_ERR_INVALID_ARG, "max_rel_err is null");
    TN_CHECK(prec == TN_PREC_BF16 || prec == TN_PREC_FP16, TN_ERR_INVALID_ARG, "prec must be bf16 or fp16");
    TN_CHECK(nbt >= 1 && M >= 1 && N >= 1 && K >= 4 && nbt * M * K <= (int64_t(1) << 30) &&
                 nbt * K * N <= (int64_t(1) << 30) && nbt * M * N <= (int64_t(1) << 30),
             TN_ERR_INVALID_ARG, "self-test shape out of range");
    TN_CHECK(K % 4 == 0 && nbt <= 65535, TN_ERR_INVALID_ARG, "K must be a multiple of 4");
    cudaStream_t s = (cudaStream_t)stream;
    int* d_err = nullptr;
    TN_CUDA(cudaMalloc(&d_err, sizeof(int)));
    TN_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), s));
    double r = 0;
    try {
      r = selftest_gemm_tc(nbt, M, N, K, prec == TN_PREC_BF16, seed, s, d_err);
    } catch (...) {
      cudaFree(d_err);
      throw;
    }
    int h_err = 0;
    TN_CUDA(cudaMemcpy(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost));
    cudaFree(d_err);
    TN_CHECK(h_err == 0, TN_ERR_TIMEOUT, "tensor-core GEMM: a bounded wait timed out");
    *max_rel_err = r;
  });
}

tn_status tn_plan_status(tn_plan_t plan, void* stream) {
  return guarded([&] {
    TN_CHECK(plan != nullptr, TN_ERR_INVALID_ARG, "plan is null");
    Plan& P = *plan->p;
    if (P.flags & TN_FLAG_PLAN_ONLY) return;
    TN_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int h_err = 0;
    TN_CUDA(cudaMemcpy(&h_err, P.d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h_err) {
      TN_CUDA(cudaMemset(P.d_err, 0, sizeof(int)));
      fail(TN_ERR_TIMEOUT, "a bounded device wait timed out in an earlier call on this plan");
    }
  });
}

tn_status tn_permute(const void* in, void* out, int32_t nbits, const int32_t* out_bit, int32_t elem_bytes,
                     void* stream) {
  return guarded([&] {
    TN_CHECK(in && out && out_bit, TN_ERR_INVALID_ARG, "null pointer");
    TN_CHECK(nbits >= 1 && nbits <= 40, TN_ERR_INVALID_ARG, "nbits out of range");
    TN_CHECK(elem_bytes == 4 || elem_bytes == 8, TN_ERR_INVALID_ARG, "elem_bytes must be 4 or 8");
    BitPermute bp{};
    bp.nbits = nbits;
    std::vector<char> seen(nbits, 0);
    for (int i = 0; i < nbits; ++i) {
      TN_CHECK(out_bit[i] >= 0 && out_bit[i] < nbits && !seen[out_bit[i]], TN_ERR_INVALID_ARG,
               "out_bit is not a permutation");
      seen[out_bit[i]] = 1;
      bp.out_bit[i] = out_bit[i];
    }
    launch_bit_permute(in, out, bp, elem_bytes, (cudaStream_t)stream);
    TN_CUDA(cudaGetLastError());
  });
}

const char* tn_last_error(void) { return g_last_error.c_str(); }

const char* tn_version(void) { return "tn-gb300 0.1 (sm_103a)"; }

}  // extern "C"
