// Plan construction and execution (host side).
//
// arXiv 2406.18889, Sec. III "Optimizing tensor contraction":
//  * a sliced sub-network fixes the values of the sliced edges; the network is
//    the sum over all assignments.  Here the slices of one batch are
//    contracted together: every tensor that depends on a sliced leaf carries
//    an extra "slice-batch" edge (one entry per slice of the batch), which is
//    a batch index when both operands carry it and a free index when only one
//    does -- slice-independent operands are then reused across the batch.
//  * dimension order: "placing the contracted dimensions of input tensors at
//    the end, the same order of contracted dimensions in both inputs, input
//    dimensions in the order of the output", assigned greedily from the root.
//    Here each step's operands must be stored as three contiguous blocks
//    (batch, free, contracted) so that the step is one strided batched GEMM;
//    the root-down pass picks, per step, the contracted order and block
//    arrangement for which the producing steps can write their results
//    directly, and inserts a transpose only where no choice allows it.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <numeric>
#include <set>

#include "plan.h"

namespace tn {

namespace {

bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }
int ilog2(int64_t x) {
  int r = 0;
  while ((int64_t(1) << r) < x) ++r;
  return r;
}
int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

std::vector<int> set_inter(const std::vector<int>& a, const std::vector<int>& b) {
  std::vector<int> r;
  std::set_intersection(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(r));
  return r;
}
std::vector<int> set_minus(const std::vector<int>& a, const std::vector<int>& b) {
  std::vector<int> r;
  std::set_difference(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(r));
  return r;
}
bool contains(const std::vector<int>& v, int e) { return std::find(v.begin(), v.end(), e) != v.end(); }

// Is operand a of step S the one stored [batch][free][contracted] and read
// as stored by the tensor cores (the other is expanded)?  The larger one; on
// a tie, the expanded one is preferably the result of a step with K <= 4,
// which can write the expanded form directly.
bool small_k_result(const Plan& P, int node) {
  if (P.nodes[node].leaf) return false;
  int64_t K = 1;
  for (int e : P.steps[node - P.n_leaves].k) K *= P.dim[e];
  return K <= 4;
}
bool a_is_big(const Plan& P, const Step& S) {
  const int64_t ea = P.nodes[S.a].elems, eb = P.nodes[S.b].elems;
  if (ea != eb) return ea > eb;
  return !(small_k_result(P, S.a) && !small_k_result(P, S.b));
}

// edges of `group` in the order they appear in `layout`
std::vector<int> order_by(const std::vector<int>& group, const std::vector<int>& layout) {
  std::vector<int> r;
  for (int e : layout)
    if (contains(group, e)) r.push_back(e);
  return r;
}

// Does `layout` consist of one contiguous run per non-empty group?
bool decomposes(const std::vector<int>& layout, const std::vector<const std::vector<int>*>& groups) {
  int prev = -1;
  std::vector<char> seen(groups.size(), 0);
  for (int e : layout) {
    int g = -1;
    for (size_t i = 0; i < groups.size(); ++i)
      if (contains(*groups[i], e)) {
        g = (int)i;
        break;
      }
    if (g < 0) return false;
    if (g != prev) {
      if (seen[g]) return false;
      seen[g] = 1;
      prev = g;
    }
  }
  return true;
}

struct Arena {
  std::vector<std::pair<int64_t, int64_t>> live;  // (off, bytes), sorted by off
  int64_t peak = 0;
  int64_t align = 256;
  int64_t alloc(int64_t bytes) {
    bytes = round_up(std::max<int64_t>(bytes, 1), align);
    int64_t off = 0;
    for (auto& b : live) {
      if (b.first - off >= bytes) break;
      off = std::max(off, b.first + b.second);
    }
    live.push_back({off, bytes});
    std::sort(live.begin(), live.end());
    peak = std::max(peak, off + bytes);
    return off;
  }
  void release(int64_t off) {
    for (size_t i = 0; i < live.size(); ++i)
      if (live[i].first == off) {
        live.erase(live.begin() + i);
        return;
      }
  }
};

}  // namespace

Plan::~Plan() {
  if (device >= 0) drop_batched_graphs(serial);
  if (graph) cudaGraphExecDestroy(graph);
  if (capture_stream) cudaStreamDestroy(capture_stream);
  for (cudaStream_t st : branch_streams) cudaStreamDestroy(st);
  for (cudaEvent_t e : unit_events) cudaEventDestroy(e);
  if (d_plan) cudaFree(d_plan);
  if (d_slice_ids) cudaFree(d_slice_ids);
  if (d_n_valid) cudaFree(d_n_valid);
  if (d_gather) cudaFree(d_gather);
  if (d_err) cudaFree(d_err);
  if (d_micro) cudaFree(d_micro);
  if (d_micro_groups) cudaFree(d_micro_groups);
  if (d_micro_loads) cudaFree(d_micro_loads);
}

// ---------------------------------------------------------------- layouts
namespace {

struct Builder {
  Plan& P;
  explicit Builder(Plan& p) : P(p) {}

  int64_t dims_prod(const std::vector<int>& es) const {
    int64_t r = 1;
    for (int e : es) r *= P.dim[e];
    return r;
  }
  std::map<int, int64_t> strides(const std::vector<int>& layout) const {
    std::map<int, int64_t> s;
    int64_t acc = 1;
    for (int i = (int)layout.size() - 1; i >= 0; --i) {
      s[layout[i]] = acc;
      acc *= P.dim[layout[i]];
    }
    return s;
  }
  int producer(int node) const { return P.nodes[node].leaf ? -1 : node - P.n_leaves; }

  // Root-down (the paper's greedy dimension ordering from the root): both
  // operands are stored [batch][free][contracted] -- contracted dimensions
  // last and in the same order in both inputs, free dimensions in the
  // result's order; the larger operand is the one the tensor cores read as
  // stored, the smaller is read along k when it is expanded.  The contracted
  // order groups the larger operand's producer's index groups so that the
  // producer writes long contiguous runs.
  void assign_layouts() {
    Node& R = P.nodes[P.root];
    std::vector<int> rl;
    if (R.variant) rl.push_back(P.batch_edge);
    if (P.block_edge >= 0) rl.push_back(P.block_edge);
    for (int e : P.open_edges) rl.push_back(e);
    R.layout = rl;
    for (int t = (int)P.steps.size() - 1; t >= 0; --t) {
      Step& S = P.steps[t];
      const std::vector<int>& Lc = P.nodes[S.c].layout;
      S.lc_nat = Lc;
      S.post_perm = false;
      std::vector<int> bt_o = order_by(S.bt, Lc), m_o = order_by(S.m, Lc), n_o = order_by(S.n, Lc);
      const bool a_big = a_is_big(P, S);
      std::vector<int> k_o = S.k;
      const int q = producer(a_big ? S.a : S.b);
      if (q >= 0) {
        const Step& Q = P.steps[q];
        std::vector<int> kk;
        for (auto* g : {&Q.bt, &Q.m, &Q.n})
          for (int e : *g)
            if (contains(S.k, e)) kk.push_back(e);
        if (kk.size() == S.k.size()) k_o = kk;
      }
      std::vector<int> big, small;
      const std::vector<int>& fb = a_big ? m_o : n_o;
      const std::vector<int>& fs = a_big ? n_o : m_o;
      big.insert(big.end(), bt_o.begin(), bt_o.end());
      big.insert(big.end(), fb.begin(), fb.end());
      big.insert(big.end(), k_o.begin(), k_o.end());
      small.insert(small.end(), bt_o.begin(), bt_o.end());
      small.insert(small.end(), fs.begin(), fs.end());
      small.insert(small.end(), k_o.begin(), k_o.end());
      P.nodes[S.a].layout = a_big ? big : small;
      P.nodes[S.b].layout = a_big ? small : big;
    }
  }

  // runs of `group` (canonical order `order`, slowest first) inside `layout`
  Runs runs_of(const std::vector<int>& order, const std::vector<int>& layout) const {
    auto st = strides(layout);
    Runs r{};
    r.n = 0;
    for (int i = (int)order.size() - 1; i >= 0; --i) {
      const int e = order[i];
      const int lg = ilog2(P.dim[e]);
      if (lg == 0) continue;
      const int64_t s = st.at(e);
      if (r.n > 0 && s == r.st[r.n - 1] << r.lg[r.n - 1] && r.lg[r.n - 1] + lg <= 62) {
        r.lg[r.n - 1] = (int8_t)(r.lg[r.n - 1] + lg);
      } else {
        TN_CHECK(r.n < kMaxRuns, TN_ERR_UNSUPPORTED, "an index group is split into too many runs");
        r.lg[r.n] = (int8_t)lg;
        r.st[r.n] = s;
        ++r.n;
      }
    }
    return r;
  }

  void fill_gemm(Step& S) {
    const auto& La = P.nodes[S.a].layout;
    const auto& Lb = P.nodes[S.b].layout;
    const auto& Lc = P.nodes[S.c].layout;
    std::vector<int> bt_o = order_by(S.bt, Lc), m_o = order_by(S.m, Lc), n_o = order_by(S.n, Lc);
    std::vector<int> k_o = order_by(S.k, a_is_big(P, S) ? La : Lb);
    GemmParams& g = S.gp;
    g.nbt = dims_prod(bt_o);
    g.M = dims_prod(m_o);
    g.N = dims_prod(n_o);
    g.K = dims_prod(k_o);
    g.a_bt = runs_of(bt_o, La);
    g.a_m = runs_of(m_o, La);
    g.a_k = runs_of(k_o, La);
    g.b_bt = runs_of(bt_o, Lb);
    g.b_k = runs_of(k_o, Lb);
    g.b_n = runs_of(n_o, Lb);
    g.c_bt = runs_of(bt_o, Lc);
    g.c_m = runs_of(m_o, Lc);
    g.c_n = runs_of(n_o, Lc);
    g.c_dec = decode_of(g.c_bt, g.c_m, g.c_n);
    g.elems_max = std::max({P.nodes[S.a].elems, P.nodes[S.b].elems, P.nodes[S.c].elems});
    S.cost = (double)g.nbt * g.M * g.N * g.K;
  }

  BitPermute bit_perm(const std::vector<int>& from, const std::vector<int>& to) const {
    auto positions = [&](const std::vector<int>& L) {
      std::map<int, int> base;
      int acc = 0;
      for (int i = (int)L.size() - 1; i >= 0; --i) {
        base[L[i]] = acc;
        acc += ilog2(P.dim[L[i]]);
      }
      return std::make_pair(base, acc);
    };
    auto [fb, nb] = positions(from);
    auto [tb, nb2] = positions(to);
    TN_CHECK(nb == nb2 && nb <= kMaxBits, TN_ERR_UNSUPPORTED, "tensor too large to transpose");
    BitPermute bp{};
    bp.nbits = nb;
    for (int e : from)
      for (int s = 0; s < ilog2(P.dim[e]); ++s) bp.out_bit[fb[e] + s] = tb[e] + s;
    return bp;
  }
};

}  // namespace

// ---------------------------------------------------------------- memory plans
namespace {

// bytes of node x: complex64 (8), 16-bit complex (4), or hi + lo 16-bit (8)
int64_t node_bytes(const Plan& P, int x, bool c64) {
  const Node& N = P.nodes[x];
  if (c64 || N.kind == KIND_C64 || N.hilo) return N.elems * 8;
  return N.elems * 4;
}
int node_word(const Plan& P, int x, bool c64) { return (c64 || P.nodes[x].kind == KIND_C64) ? 8 : 4; }

// tensor-core operand roles of a step: A is read as stored ([bt][m][k], k
// contiguous: single runs), B is expanded through its runs
struct TcRoles {
  int a_node, b_node;
  int64_t M, N, K;
  int64_t a_bt, a_m;               // A strides (complex elements)
  Runs b_bt, b_k, b_n;             // B index maps
  Runs c_bt, c_m, c_n;             // output index maps
};
int64_t single_stride(const Runs& r, int64_t extent, bool* ok) {
  if (extent <= 1) return 0;
  if (r.n != 1) *ok = false;
  return r.n > 0 ? r.st[0] : 0;
}
TcRoles tc_roles(const Step& S, bool* ok_out = nullptr) {
  const GemmParams& g = S.gp;
  TcRoles r{};
  bool ok = true;
  if (!S.tc_swap) {
    r.a_node = S.a;
    r.b_node = S.b;
    r.M = g.M;
    r.N = g.N;
    r.K = g.K;
    r.a_bt = single_stride(g.a_bt, g.nbt, &ok);
    r.a_m = single_stride(g.a_m, g.M, &ok);
    ok = ok && (g.K <= 1 || (g.a_k.n == 1 && g.a_k.st[0] == 1));
    r.b_bt = g.b_bt;
    r.b_k = g.b_k;
    r.b_n = g.b_n;
    r.c_bt = g.c_bt;
    r.c_m = g.c_m;
    r.c_n = g.c_n;
  } else {
    r.a_node = S.b;
    r.b_node = S.a;
    r.M = g.N;
    r.N = g.M;
    r.K = g.K;
    r.a_bt = single_stride(g.b_bt, g.nbt, &ok);
    r.a_m = single_stride(g.b_n, g.N, &ok);
    ok = ok && (g.K <= 1 || (g.b_k.n == 1 && g.b_k.st[0] == 1));
    r.b_bt = g.a_bt;
    r.b_k = g.a_k;
    r.b_n = g.a_m;
    r.c_bt = g.c_bt;
    r.c_m = g.c_n;
    r.c_n = g.c_m;
  }
  if (S.pair_rows) {
    // Row pairs: A's rows are K contiguous entries, so rows 2i and 2i + 1 read
    // as one row of 2K entries -- a whole 128-byte k tile instead of a half-
    // filled one -- and the GEMM becomes C'[i][(p, n)] = sum_{(p', k)}
    // A'[i][(p', k)] B'[(p', k)][(p, n)] with B' = [[B, 0], [0, B]]: half the
    // rows, twice N and K (the zero blocks cost tensor flops, not bytes).  The
    // output keeps its layout: row 2i + p of C is row i of C' at column
    // block p, so m loses its lowest bit to a new top digit of n.
    r.M /= 2;
    r.N *= 2;
    r.K *= 2;
    r.a_m *= 2;
    const int64_t pst = r.c_m.st[0];
    if (r.c_m.lg[0] == 1) {
      for (int i = 1; i < r.c_m.n; ++i) {
        r.c_m.lg[i - 1] = r.c_m.lg[i];
        r.c_m.st[i - 1] = r.c_m.st[i];
      }
      --r.c_m.n;
    } else {
      r.c_m.lg[0] = (int8_t)(r.c_m.lg[0] - 1);
      r.c_m.st[0] = 2 * pst;
    }
    r.c_n.lg[r.c_n.n] = 1;
    r.c_n.st[r.c_n.n] = pst;
    ++r.c_n.n;
  }
  if (ok_out) *ok_out = ok;
  return r;
}
// expanded-operand bytes of a tensor-core step (its GEMM as run, hi + lo doubled)
int64_t tc_bx_bytes(const Step& S, const TcRoles& r) {
  return expanded_b_bytes(S.gp.nbt, r.N, r.K) * (S.hilo ? 2 : 1);
}

// split products also accumulate K in chunks (the tensor cores' own
// accumulation error grows with K): 4 k tiles, or 1 with TN_FLAG_FINE_ACC;
// single CTAs then
int tc_acc_split(const Plan& P, const Step& S) { return (P.flags & TN_FLAG_FINE_ACC) ? 1 : S.hilo ? 4 : 0; }
// The default launch form: the widest tile for N; 256-row tiles for K-heavy
// steps (they load each B tile once for two 128-row MMAs, and the expanded B
// dominates the bytes a tile brings into shared memory).
TcForm tc_default_form(const Plan& P, const Step& S, const TcRoles& r) {
  TcForm f{tc_gemm_bn(r.N), 1};
  const bool acc = tc_acc_split(P, S) != 0;
  f.mh = (!acc && f.bn == 256 && r.M >= 256 && r.K >= 256) ? 2 : 1;
  return f;
}
// Every form the tuner may try (the default first): the widest tile for N or
// half of it; at width 256 also 256-row tiles (M >= 256, not with chunked
// accumulation) -- the forms the launcher accepts.
std::vector<TcForm> tc_forms(const Plan& P, const Step& S) {
  const TcRoles r = tc_roles(S);
  std::vector<TcForm> out{tc_default_form(P, S, r)};
  auto add = [&](TcForm f) {
    for (const TcForm& g : out)
      if (g.bn == f.bn && g.mh == f.mh) return;
    out.push_back(f);
  };
  const bool acc = tc_acc_split(P, S) != 0;
  const int bn0 = tc_gemm_bn(r.N);
  for (int bn : {bn0, bn0 / 2}) {
    if (bn < 32) continue;
    add({bn, 1});
    if (bn == 256 && !acc && r.M >= 256) add({bn, 2});
  }
  return out;
}

MemPlan plan_memory(const Plan& P, bool c64, const std::vector<std::vector<int>>& leaf_src_layout,
                    bool micro) {
  MemPlan M;
  M.c64 = c64;
  M.micro = micro && !P.micro_groups.empty();
  const int nn = (int)P.nodes.size();
  M.off.assign(nn, -1);
  M.in_plan.assign(nn, 0);
  M.tmp_off.assign(P.steps.size(), -1);
  M.bx_off.assign(P.steps.size(), -1);
  int64_t poff = 0;
  std::vector<int64_t> src_off(P.n_leaves, -1);
  for (int i = 0; i < P.n_leaves; ++i) {
    int64_t el = 1;
    for (int e : leaf_src_layout[i]) el *= P.dim[e];
    src_off[i] = poff;
    poff += round_up(el * 8, 256);  // leaves are always complex64
    if (!P.nodes[i].variant) {
      M.off[i] = src_off[i];
      M.in_plan[i] = 1;
    }
  }
  // hoisted steps run once at creation; their transposes and expanded operands
  // use a creation-time scratch buffer: [transpose temp | expanded operand]
  int64_t tmax = 0, bmax = 0;
  for (size_t t = 0; t < P.steps.size(); ++t)
    if (P.steps[t].hoisted) {
      const Step& S = P.steps[t];
      M.off[S.c] = poff;
      M.in_plan[S.c] = 1;
      poff += round_up(node_bytes(P, S.c, c64), 256);
      if (S.post_perm) tmax = std::max(tmax, node_bytes(P, S.c, c64));
      if (!c64 && S.tc) {
        TcRoles r = tc_roles(S);
        bmax = std::max(bmax, tc_bx_bytes(S, r));
      }
    }
  for (size_t t = 0; t < P.steps.size(); ++t)
    if (P.steps[t].hoisted) {
      if (P.steps[t].post_perm) M.tmp_off[t] = 0;
      if (!c64 && P.steps[t].tc) M.bx_off[t] = round_up(tmax, 256);
    }
  M.create_scratch = (tmax || bmax) ? round_up(tmax, 256) + bmax : 0;
  M.plan_bytes = poff;
  // Two arenas: the batch's slice-independent steps (and fused small-step
  // groups) allocate in `wi`, everything else in `ws`; the workspace is
  // [wi | ws].  Regions of one arena are reused only within it, so the
  // slice-independent subtrees share no memory with the rest of the batch
  // but the results the slice-dependent steps read from them, and can run
  // concurrently with it (the batch graph's branches).
  Arena ws, wi;
  M.wsz.assign(nn, 0);
  M.tmp_sz.assign(P.steps.size(), 0);
  M.bx_sz.assign(P.steps.size(), 0);
  std::vector<char> in_wi(nn, 0), tmp_wi(P.steps.size(), 0), bx_wi(P.steps.size(), 0);
  auto alloc_node = [&](int x, int64_t bytes, bool inv) {
    M.off[x] = (inv ? wi : ws).alloc(bytes);
    M.wsz[x] = round_up(std::max<int64_t>(bytes, 1), 256);
    in_wi[x] = inv ? 1 : 0;
  };
  auto release_node = [&](int x) {
    if (!M.in_plan[x]) (in_wi[x] ? wi : ws).release(M.off[x]);
  };
  for (int i = 0; i < P.n_leaves; ++i)
    if (P.nodes[i].variant) {
      M.gather_node.push_back(i);
      alloc_node(i, node_bytes(P, i, c64), false);
    }
  if (M.micro) {
    // the fused small steps run together right after the gather: each result
    // gets its own region; their operands and inner results are free afterwards
    for (size_t g = 0; g < P.micro_groups.size(); ++g)
      for (int t : P.micro_groups[g]) {
        const Step& S = P.steps[t];
        alloc_node(S.c, node_bytes(P, S.c, c64), (int)g < P.n_micro_inv);
      }
    for (const Step& S : P.steps)
      if (S.micro)
        for (int x : {S.a, S.b})
          if (!M.in_plan[x] && (P.nodes[x].leaf || P.steps[x - P.n_leaves].micro)) release_node(x);
  }
  for (size_t t = 0; t < P.steps.size(); ++t) {
    const Step& S = P.steps[t];
    if (S.hoisted || (M.micro && S.micro)) continue;
    const bool inv = !S.variant;
    Arena& A = inv ? wi : ws;
    if (!c64 && S.fuse_expand) {
      // the result is stored only as its consumer's expanded operand
      const Step& U = P.steps[P.nodes[S.c].consumer];
      TcRoles r = tc_roles(U);
      alloc_node(S.c, expanded_b_bytes(U.gp.nbt, r.N, r.K) * (U.hilo ? 2 : 1), inv);
    } else {
      alloc_node(S.c, node_bytes(P, S.c, c64), inv);
    }
    int64_t tmp = -1, bx = -1;
    if (S.post_perm) {
      tmp = M.tmp_off[t] = A.alloc(node_bytes(P, S.c, c64));
      M.tmp_sz[t] = round_up(std::max<int64_t>(node_bytes(P, S.c, c64), 1), 256);
      tmp_wi[t] = inv;
    }
    if (!c64 && S.tc) {
      TcRoles r = tc_roles(S);
      if (!S.b_fused) {
        bx = M.bx_off[t] = A.alloc(tc_bx_bytes(S, r));
        M.bx_sz[t] = round_up(std::max<int64_t>(tc_bx_bytes(S, r), 1), 256);
        bx_wi[t] = inv;
      }
    }
    if (tmp >= 0) A.release(tmp);
    if (bx >= 0) A.release(bx);
    for (int x : {S.a, S.b}) release_node(x);
  }
  // place the slice-dependent arena after the slice-independent one
  M.inv_bytes = round_up(wi.peak, 256);
  for (int x = 0; x < nn; ++x)
    if (!M.in_plan[x] && M.off[x] >= 0 && !in_wi[x]) M.off[x] += M.inv_bytes;
  for (size_t t = 0; t < P.steps.size(); ++t) {
    const Step& S = P.steps[t];
    if (S.hoisted) continue;
    if (M.tmp_off[t] >= 0 && !tmp_wi[t]) M.tmp_off[t] += M.inv_bytes;
    if (M.bx_off[t] >= 0 && !bx_wi[t]) M.bx_off[t] += M.inv_bytes;
    if (!c64 && S.tc && S.b_fused && !(M.micro && S.micro)) M.bx_off[t] = M.off[tc_roles(S).b_node];
  }
  ws.peak += M.inv_bytes;
  M.ws_bytes = round_up(std::max<int64_t>(ws.peak, 256), 256);
  // gather table (offsets relative to the plan-memory and workspace bases)
  for (int i : M.gather_node) {
    const Node& N = P.nodes[i];
    GatherLeaf g{};
    g.src_off = src_off[i];
    g.dst_off = M.off[i];
    g.rest = N.elems / P.B;
    int64_t acc = 1, inner = 1;
    for (int d = (int)N.layout.size() - 1; d >= 0; --d) {
      if (N.layout[d] == P.batch_edge) inner = acc;
      acc *= P.dim[N.layout[d]];
    }
    g.inner = inner;
    std::vector<int> sl_here;
    for (int e : leaf_src_layout[i])
      if (std::find(P.sliced.begin(), P.sliced.end(), e) != P.sliced.end()) sl_here.push_back(e);
    TN_CHECK(sl_here.size() <= 8, TN_ERR_UNSUPPORTED, "a leaf holds more than 8 sliced edges");
    g.n_sel = (int)sl_here.size();
    for (int j = 0; j < g.n_sel; ++j) {
      g.slice_bit[j] = (int)(std::find(P.sliced.begin(), P.sliced.end(), sl_here[j]) - P.sliced.begin());
      g.sel_stride[j] = g.rest << (g.n_sel - 1 - j);
    }
    M.gather.push_back(g);
    M.gather_max_rest = std::max(M.gather_max_rest, g.rest);
  }
  return M;
}

// where a leaf's source lives in plan memory (variant leaves: the gather source)
int64_t leaf_src_offset(const MemPlan& M, const Plan& P, int i) {
  if (!P.nodes[i].variant) return M.off[i];
  for (size_t j = 0; j < M.gather_node.size(); ++j)
    if (M.gather_node[j] == i) return M.gather[j].src_off;
  fail(TN_ERR_INVALID_ARG, "internal: sliced leaf without a gather entry");
}

struct Exec {
  const Plan& P;
  const MemPlan& M;
  char* pb;  // plan memory base
  char* wb;  // workspace base
  char* base(int node) const { return (M.in_plan[node] ? pb : wb) + M.off[node]; }
};

struct Recorder {
  std::vector<LaunchRecord>* rec;
  cudaStream_t s;
  void begin(int kind, double flops, double bytes) {
    if (!rec) return;
    LaunchRecord r{kind, flops, bytes, nullptr, nullptr};
    TN_CUDA(cudaEventCreate(&r.start));
    TN_CUDA(cudaEventCreate(&r.stop));
    TN_CUDA(cudaEventRecord(r.start, s));
    rec->push_back(r);
  }
  void end() {
    if (rec) TN_CUDA(cudaEventRecord(rec->back().stop, s));
  }
};

// One contraction step: GEMM (tensor-core or CUDA-core) + transpose if needed.
// `amax` (calibration, complex64 only): per-node maxima of |re|, |im|.
void enqueue_step(const Exec& X, size_t t, cudaStream_t s, Recorder& R, unsigned* amax) {
  const Plan& P = X.P;
  const MemPlan& M = X.M;
  const Step& S = P.steps[t];
  const Node& NC = P.nodes[S.c];
  char* dst = X.base(S.c);
  char* out = S.post_perm ? X.wb + M.tmp_off[t] : dst;
  const int out_kind = M.c64 ? KIND_C64 : NC.kind;
  const bool out_hilo = !M.c64 && NC.hilo;
  const int64_t lo_off = NC.elems * 4;  // hi + lo storage: lo follows hi
  const double flops = 8.0 * S.cost;
  const double bytes = (double)(node_bytes(P, S.a, M.c64) + node_bytes(P, S.b, M.c64) + node_bytes(P, S.c, M.c64));
  // stored = true * 2^-exp2; the tensor-core B operand is scaled by 2^-bexp as it is expanded
  const int e_in = S.tc ? P.nodes[S.tc_swap ? S.b : S.a].exp2 + S.bexp : P.nodes[S.a].exp2 + P.nodes[S.b].exp2;
  const float scale = M.c64 ? 1.0f : ldexpf(1.0f, e_in - P.nodes[S.c].exp2);
  if (M.c64) {
    GemmParams g = S.gp;
    g.A = X.base(S.a);
    g.B = X.base(S.b);
    g.C = out;
    g.C2 = nullptr;
    R.begin(0, flops, bytes);
    launch_gemm_c64(g, 0, s);
    R.end();
  } else if (S.tc) {
    TcRoles r = tc_roles(S);
    const Node& NA = P.nodes[r.a_node];
    char* bx = X.wb + M.bx_off[t];
    const int64_t bx_bytes = expanded_b_bytes(S.gp.nbt, r.N, r.K);
    char* bx_lo = S.hilo ? bx + bx_bytes : nullptr;
    const bool b_c64 = P.nodes[r.b_node].kind == KIND_C64;
    TN_CHECK(NA.kind == P.skind && NA.hilo == S.hilo, TN_ERR_INVALID_ARG, "internal: tensor-core operand storage");
    if (!S.b_fused) {
      R.begin(4, 0, (double)node_bytes(P, r.b_node, false) + (double)bx_bytes * (S.hilo ? 2 : 1));
      // row-paired steps: B's own extents, written block-diagonally
      const int pr = S.pair_rows ? 1 : 0;
      launch_expand_b(X.base(r.b_node), r.b_bt, r.b_k, r.b_n, S.gp.nbt, r.N >> pr, r.K >> pr,
                      P.skind == KIND_BF16, bx, s, b_c64, bx_lo, ldexpf(1.0f, -S.bexp), S.pair_rows);
      R.end();
    }
    TcGemmParams tp{};
    tp.nbt = S.gp.nbt;
    tp.M = r.M;
    tp.N = r.N;
    tp.K = r.K;
    tp.c_bt = r.c_bt;
    tp.c_m = r.c_m;
    tp.c_n = r.c_n;
    tp.C = out;
    tp.C2 = out_hilo ? out + lo_off : nullptr;
    tp.out_kind = out_kind;
    tp.out_hilo = out_hilo ? 1 : 0;
    tp.scale = scale;
    tp.err = P.d_err;
    tp.acc_split = tc_acc_split(P, S);
    const TcForm f = S.tc_bn ? TcForm{S.tc_bn, S.tc_mh} : tc_default_form(P, S, r);
    tp.bn = f.bn;
    tp.m_halves = f.mh;
    const char* a_hi = X.base(r.a_node);
    R.begin(5, flops, bytes);
    launch_gemm_tc(a_hi, S.hilo ? a_hi + NA.elems * 4 : nullptr, r.a_bt, r.a_m, bx, bx_lo, tp,
                   P.skind == KIND_BF16, s);
    R.end();
  } else {
    TN_CHECK(P.nodes[S.a].kind == KIND_C64 && P.nodes[S.b].kind == KIND_C64, TN_ERR_INVALID_ARG,
             "internal: CUDA-core step operands must be complex64");
    GemmParams g = S.gp;
    g.A = X.base(S.a);
    g.B = X.base(S.b);
    g.C = out;
    g.C2 = out_hilo ? out + lo_off : nullptr;
    if (S.fuse_expand) {
      // written as the consumer's expanded operand, scaled by its 2^-bexp
      const Step& U = P.steps[NC.consumer];
      TcRoles r = tc_roles(U);
      ExpandedDst ex{};
      ex.b_bt = r.b_bt;
      ex.b_k = r.b_k;
      ex.b_n = r.b_n;
      ex.nbt = U.gp.nbt;
      ex.N = r.N;
      ex.K = r.K;
      ex.Bx = dst;
      ex.Bx_lo = U.hilo ? dst + expanded_b_bytes(U.gp.nbt, r.N, r.K) : nullptr;
      ex.bf16 = P.skind == KIND_BF16;
      R.begin(0, flops, bytes);
      launch_gemm_simt(g, KIND_C64, out_kind, ldexpf(scale, -U.bexp), s, false, &ex);
      R.end();
    } else {
      R.begin(0, flops, bytes);
      launch_gemm_simt(g, KIND_C64, out_kind, scale, s, out_hilo);
      R.end();
    }
  }
  if (S.post_perm) {
    const int pe = out_kind == KIND_C64 ? 8 : 4;
    R.begin(1, 0, 2.0 * (double)node_bytes(P, S.c, M.c64));
    launch_bit_permute(out, dst, S.perm, pe, s);
    if (out_hilo) launch_bit_permute(out + lo_off, dst + lo_off, S.perm, pe, s);
    R.end();
  }
  if (amax) launch_amax_c64(dst, P.nodes[S.c].elems, amax + S.c, s);
}

void enqueue_gather(const Exec& X, cudaStream_t s, Recorder& R) {
  const Plan& P = X.P;
  if (X.M.gather.empty()) return;
  double bytes = 0;
  for (auto& g : X.M.gather) bytes += 2.0 * g.rest * P.B * 8.0;
  R.begin(2, 0, bytes);
  launch_gather_leaves(P.d_gather, (int)X.M.gather.size(), X.M.gather_max_rest, P.d_slice_ids, P.B, X.pb, X.wb, s,
                       8);
  R.end();
}

// fused small-step groups [g0, g1)
void enqueue_micro(const Exec& X, int g0, int g1, cudaStream_t s, Recorder& R) {
  const Plan& P = X.P;
  if (g0 >= g1) return;
  TN_CHECK(P.d_micro, TN_ERR_INVALID_ARG, "internal: fused small steps unavailable");
  double flops = 0, bytes = 0;
  for (int g = g0; g < g1; ++g)
    for (int t : P.micro_groups[g]) {
      const Step& S = P.steps[t];
      flops += 8.0 * S.cost;
      bytes += (double)(node_bytes(P, S.a, X.M.c64) + node_bytes(P, S.b, X.M.c64) + node_bytes(P, S.c, X.M.c64));
    }
  R.begin(0, flops, bytes);
  launch_micro(P.d_micro, P.d_micro_groups + g0, P.d_micro_loads, g1 - g0, P.micro_smem, X.pb, X.wb, s);
  R.end();
}

void enqueue_accumulate(const Exec& X, void* amps, int accumulate, cudaStream_t s, Recorder& R) {
  const Plan& P = X.P;
  R.begin(3, 0, 8.0 * (double)P.nodes[P.root].elems + 16.0 * P.G * P.J * (accumulate ? 2 : 1));
  launch_accumulate_c64(X.base(P.root), P.root_sb, P.root_sg, P.root_sj, P.G, P.J, P.d_n_valid, P.B, amps,
                        accumulate, s, ldexp(1.0, P.nodes[P.root].exp2));
  R.end();
}

void enqueue_batch_mem(const Plan& P, const MemPlan& M, char* pb, void* ws, void* amps, int accumulate,
                       cudaStream_t s, std::vector<LaunchRecord>* rec, unsigned* amax, bool hoisted_too) {
  Exec X{P, M, pb, (char*)ws};
  Recorder R{rec, s};
  enqueue_gather(X, s, R);
  if (amax)
    for (int i = 0; i < P.n_leaves; ++i) launch_amax_c64(X.base(i), P.nodes[i].elems, amax + i, s);
  if (M.micro) {
    TN_CHECK(!amax, TN_ERR_INVALID_ARG, "internal: fused small steps during calibration");
    // as in the batch graph: the slice-independent groups, then the rest
    enqueue_micro(X, 0, P.n_micro_inv, s, R);
    enqueue_micro(X, P.n_micro_inv, (int)P.micro_groups.size(), s, R);
  }
  for (size_t t = 0; t < P.steps.size(); ++t) {
    if (P.steps[t].hoisted && !hoisted_too) continue;
    if (M.micro && P.steps[t].micro) continue;
    enqueue_step(X, t, s, R, amax);
  }
  if (amps) enqueue_accumulate(X, amps, accumulate, s, R);
}

// ---------------------------------------------------------------- concurrent batch graph
// One batch as launch units -- the gather (kind 0), the slice-independent and
// the other fused small-step groups (1, 2), one step each (3: its expansion,
// GEMM and transpose) -- in the order of the sequential schedule.  Two units
// depend on each other when the workspace ranges they touch (read or write)
// overlap: the true data dependencies, and the reuse of a region freed by an
// earlier unit.  Plan memory is read-only during a batch.
constexpr int kBranches = 4;
using Ranges = std::vector<std::pair<int64_t, int64_t>>;

void plan_batch_graph(Plan& P) {
  const MemPlan& M = P.mem;
  std::vector<Ranges> rg;
  P.unit_kind.clear();
  P.unit_step.clear();
  auto add = [](Ranges& r, int64_t off, int64_t bytes) {
    if (off >= 0 && bytes > 0) r.push_back({off, off + bytes});
  };
  auto node = [&](Ranges& r, int x) {
    if (!M.in_plan[x]) add(r, M.off[x], M.wsz[x]);
  };
  auto unit = [&](int kind, int step) {
    P.unit_kind.push_back(kind);
    P.unit_step.push_back(step);
    rg.emplace_back();
    return &rg.back();
  };
  if (!M.gather.empty()) {
    Ranges* r = unit(0, -1);
    for (int i : M.gather_node) node(*r, i);
  }
  if (M.micro)
    for (int part = 0; part < 2; ++part) {
      const int g0 = part ? P.n_micro_inv : 0, g1 = part ? (int)P.micro_groups.size() : P.n_micro_inv;
      if (g0 >= g1) continue;
      Ranges* r = unit(1 + part, -1);
      for (int g = g0; g < g1; ++g)
        for (int t : P.micro_groups[g])
          for (int x : {P.steps[t].a, P.steps[t].b, P.steps[t].c}) node(*r, x);
    }
  for (size_t t = 0; t < P.steps.size(); ++t) {
    const Step& S = P.steps[t];
    if (S.hoisted || (M.micro && S.micro)) continue;
    Ranges* r = unit(3, (int)t);
    for (int x : {S.a, S.b, S.c}) node(*r, x);
    if (S.post_perm) add(*r, M.tmp_off[t], M.tmp_sz[t]);
    add(*r, M.bx_off[t], M.bx_sz[t]);
  }
  const int n = (int)rg.size();
  auto overlap = [&](int i, int j) {
    for (auto& a : rg[i])
      for (auto& b : rg[j])
        if (a.first < b.second && b.first < a.second) return true;
    return false;
  };
  // branches: a unit continues the branch whose last unit is its latest
  // dependency; else takes an unused branch; else the branch idle longest.
  // It waits, on every other branch, for the latest unit it depends on.
  P.unit_branch.assign(n, 0);
  P.unit_waits.assign(n, {});
  std::vector<int> tail(kBranches, -1);
  for (int j = 0; j < n; ++j) {
    std::vector<char> dep(j, 0);
    for (int i = 0; i < j; ++i) dep[i] = overlap(i, j) ? 1 : 0;
    int b = -1;
    for (int k = 0; k < kBranches; ++k)
      if (tail[k] >= 0 && dep[tail[k]] && (b < 0 || tail[k] > tail[b])) b = k;
    for (int k = 0; k < kBranches && b < 0; ++k)
      if (tail[k] < 0) b = k;
    if (b < 0) {
      b = 0;
      for (int k = 1; k < kBranches; ++k)
        if (tail[k] < tail[b]) b = k;
    }
    std::vector<int> last(kBranches, -1);
    for (int i = 0; i < j; ++i)
      if (dep[i] && P.unit_branch[i] != b) last[P.unit_branch[i]] = std::max(last[P.unit_branch[i]], i);
    for (int k = 0; k < kBranches; ++k)
      if (last[k] >= 0) P.unit_waits[j].push_back(last[k]);
    P.unit_branch[j] = b;
    tail[b] = j;
  }
  // Self-check: every two units whose ranges overlap are ordered by the
  // graph (the earlier one happens before the later: same branch, or a chain
  // of branch order and waits), so no two launches that share workspace run
  // concurrently.
  const int words = (n + 63) / 64;
  std::vector<std::vector<uint64_t>> hb(n, std::vector<uint64_t>(words, 0));  // hb[j]: units before j
  std::vector<int> prev(kBranches, -1);
  auto join = [&](int j, int i) {
    for (int w = 0; w < words; ++w) hb[j][w] |= hb[i][w];
    hb[j][i / 64] |= uint64_t(1) << (i % 64);
  };
  for (int j = 0; j < n; ++j) {
    const int b = P.unit_branch[j];
    if (prev[b] >= 0) join(j, prev[b]);
    for (int i : P.unit_waits[j]) join(j, i);
    prev[b] = j;
    for (int i = 0; i < j; ++i)
      TN_CHECK(!overlap(i, j) || ((hb[j][i / 64] >> (i % 64)) & 1), TN_ERR_INVALID_ARG,
               "internal: batch graph leaves two launches that share workspace unordered");
  }
}

// The branch streams and events of the batch graph (created before a capture:
// creating them is not a stream operation a capture may record).
void make_graph_resources(Plan& P) {
  while ((int)P.branch_streams.size() < kBranches - 1) {
    cudaStream_t st = nullptr;
    TN_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    P.branch_streams.push_back(st);
  }
  while (P.unit_events.size() < P.unit_kind.size() + kBranches) {
    cudaEvent_t e = nullptr;
    TN_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    P.unit_events.push_back(e);
  }
}

// Queue one batch on `s` (being captured) with the units spread over the
// plan's branch streams; every branch joins `s` before the slice sum.
void enqueue_batch_graph(Plan& P, void* ws, void* amps, int accumulate, cudaStream_t s) {
  const MemPlan& M = P.mem;
  Exec X{P, M, (char*)P.d_plan, (char*)ws};
  Recorder R{nullptr, s};
  const int n = (int)P.unit_kind.size();
  TN_CHECK((int)P.branch_streams.size() == kBranches - 1 && (int)P.unit_events.size() >= n + kBranches,
           TN_ERR_INVALID_ARG, "internal: batch graph streams not created");
  cudaEvent_t fork = P.unit_events[n];
  TN_CUDA(cudaEventRecord(fork, s));
  std::vector<char> used(kBranches, 0);
  used[0] = 1;
  for (int j = 0; j < n; ++j) {
    const int b = P.unit_branch[j];
    cudaStream_t st = b ? P.branch_streams[b - 1] : s;
    if (!used[b]) {
      TN_CUDA(cudaStreamWaitEvent(st, fork, 0));
      used[b] = 1;
    }
    for (int i : P.unit_waits[j]) TN_CUDA(cudaStreamWaitEvent(st, P.unit_events[i], 0));
    switch (P.unit_kind[j]) {
      case 0: enqueue_gather(X, st, R); break;
      case 1: enqueue_micro(X, 0, P.n_micro_inv, st, R); break;
      case 2: enqueue_micro(X, P.n_micro_inv, (int)P.micro_groups.size(), st, R); break;
      default: enqueue_step(X, (size_t)P.unit_step[j], st, R, nullptr); break;
    }
    TN_CUDA(cudaEventRecord(P.unit_events[j], st));
  }
  for (int b = 1; b < kBranches; ++b)
    if (used[b]) {
      TN_CUDA(cudaEventRecord(P.unit_events[n + b], P.branch_streams[b - 1]));
      TN_CUDA(cudaStreamWaitEvent(s, P.unit_events[n + b], 0));
    }
  if (amps) enqueue_accumulate(X, amps, accumulate, s, R);
}

}  // namespace

// ---------------------------------------------------------------- build
std::vector<int64_t> calibration_ids(int B, int n_sliced) {
  // seeded pseudo-random ids (splitmix64) spread over all sliced edges, so no
  // sliced edge is pinned to one value across the sample
  std::vector<int64_t> ids(B);
  const uint64_t mask = n_sliced >= 63 ? ~0ull : (uint64_t(1) << n_sliced) - 1;
  uint64_t z = 0x2406188890ull;
  for (int b = 0; b < B; ++b) {
    z += 0x9E3779B97F4A7C15ull;
    uint64_t x = z;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    ids[b] = (int64_t)(x & mask);
  }
  return ids;
}

std::unique_ptr<Plan> build_plan(const tn_network_desc* net, const tn_tree_desc* tree,
                                 const tn_plan_options* opt, cudaStream_t stream,
                                 const std::vector<char>* hilo_mask) {
  auto Pp = std::make_unique<Plan>();
  Plan& P = *Pp;
  TN_CHECK(net && tree && opt, TN_ERR_INVALID_ARG, "null descriptor");
  TN_CHECK(net->n_leaves >= 1 && net->n_edges >= 1, TN_ERR_INVALID_ARG, "empty network");
  TN_CHECK(net->leaf_rank && net->leaf_edges && net->edge_dim && net->leaf_data, TN_ERR_INVALID_ARG,
           "null network array");
  TN_CHECK(opt->prec == TN_PREC_C64 || opt->prec == TN_PREC_BF16 || opt->prec == TN_PREC_FP16,
           TN_ERR_INVALID_ARG, "unknown precision");
  TN_CHECK(opt->max_slice_batch >= 1 && opt->max_slice_batch <= 65536 && is_pow2(opt->max_slice_batch),
           TN_ERR_INVALID_ARG, "max_slice_batch must be a power of two in [1, 65536]");
  P.prec = opt->prec;
  P.skind = opt->prec == TN_PREC_C64 ? KIND_C64 : opt->prec == TN_PREC_BF16 ? KIND_BF16 : KIND_F16;
  P.flags = opt->flags;
  P.n_leaves = net->n_leaves;
  P.n_edges = net->n_edges;
  P.dim.assign(net->edge_dim, net->edge_dim + net->n_edges);
  for (int64_t d : P.dim) TN_CHECK(is_pow2(d), TN_ERR_UNSUPPORTED, "edge dimensions must be powers of two");
  // leaves
  std::vector<int> count(P.n_edges, 0);
  int64_t pos = 0, eoff = 0;
  P.leaf_edges.resize(P.n_leaves);
  P.leaf_off.resize(P.n_leaves);
  for (int i = 0; i < P.n_leaves; ++i) {
    int r = net->leaf_rank[i];
    TN_CHECK(r >= 0 && r <= 32, TN_ERR_INVALID_ARG, "leaf rank out of range");
    int64_t el = 1;
    for (int j = 0; j < r; ++j) {
      int e = net->leaf_edges[pos + j];
      TN_CHECK(e >= 0 && e < P.n_edges, TN_ERR_INVALID_ARG, "leaf edge id out of range");
      TN_CHECK(!contains(P.leaf_edges[i], e), TN_ERR_INVALID_ARG, "edge repeated within a leaf");
      P.leaf_edges[i].push_back(e);
      count[e]++;
      el *= P.dim[e];
      TN_CHECK(el <= (int64_t(1) << 40), TN_ERR_UNSUPPORTED, "leaf too large");
    }
    pos += r;
    P.leaf_off[i] = eoff;
    eoff += el;
  }
  const int64_t total_leaf_elems = eoff;
  TN_CHECK(net->n_open >= 0 && (net->n_open == 0 || net->open_edges), TN_ERR_INVALID_ARG, "bad open edges");
  P.open_edges.assign(net->open_edges, net->open_edges + net->n_open);
  P.block_edge = net->block_edge;
  TN_CHECK(P.block_edge >= -1 && P.block_edge < P.n_edges, TN_ERR_INVALID_ARG, "bad block edge");
  std::vector<int> outputs = P.open_edges;
  if (P.block_edge >= 0) outputs.push_back(P.block_edge);
  {
    std::vector<int> so = outputs;
    std::sort(so.begin(), so.end());
    TN_CHECK(std::adjacent_find(so.begin(), so.end()) == so.end(), TN_ERR_INVALID_ARG, "output edge repeated");
    for (int e : so) TN_CHECK(e >= 0 && e < P.n_edges, TN_ERR_INVALID_ARG, "output edge id out of range");
  }
  for (int e = 0; e < P.n_edges; ++e) {
    if (e == P.block_edge) {
      TN_CHECK(count[e] >= 1, TN_ERR_INVALID_ARG, "block edge unused");
    } else if (contains(P.open_edges, e)) {
      TN_CHECK(count[e] == 1, TN_ERR_INVALID_ARG, "open edge must appear in exactly one leaf");
    } else {
      TN_CHECK(count[e] == 2 || count[e] == 0, TN_ERR_INVALID_ARG, "bond must appear in exactly two leaves");
    }
  }
  P.G = P.block_edge >= 0 ? P.dim[P.block_edge] : 1;
  P.J = 1;
  for (int e : P.open_edges) P.J *= P.dim[e];
  TN_CHECK(P.G * P.J <= (int64_t(1) << 34), TN_ERR_UNSUPPORTED, "output too large");
  // slicing
  TN_CHECK(tree->n_sliced >= 0 && tree->n_sliced <= 62, TN_ERR_INVALID_ARG, "n_sliced out of range");
  TN_CHECK(tree->n_sliced == 0 || tree->sliced_edges, TN_ERR_INVALID_ARG, "null sliced_edges");
  for (int i = 0; i < tree->n_sliced; ++i) {
    int e = tree->sliced_edges[i];
    TN_CHECK(e >= 0 && e < P.n_edges && !contains(outputs, e) && count[e] == 2 && P.dim[e] == 2 &&
                 !contains(P.sliced, e),
             TN_ERR_INVALID_ARG, "sliced edge must be a distinct dimension-2 bond");
    P.sliced.push_back(e);
  }
  P.batch_edge = P.n_edges;
  P.B = P.sliced.empty() ? 1 : opt->max_slice_batch;
  P.dim.push_back(P.B);
  // tree replay
  TN_CHECK(tree->n_steps == P.n_leaves - 1 && (tree->n_steps == 0 || tree->pairs), TN_ERR_INVALID_ARG,
           "a tree over n leaves has n - 1 steps");
  int n_nodes = P.n_leaves + tree->n_steps;
  P.nodes.resize(n_nodes);
  std::vector<char> sliced_mark(P.n_edges + 1, 0);
  for (int e : P.sliced) sliced_mark[e] = 1;
  std::vector<std::set<int>> occ(P.n_edges + 1);
  for (int i = 0; i < P.n_leaves; ++i) {
    Node& N = P.nodes[i];
    N.leaf = true;
    N.leaf_id = i;
    for (int e : P.leaf_edges[i]) {
      if (sliced_mark[e])
        N.variant = true;
      else
        N.edges.push_back(e);
    }
    if (N.variant) N.edges.push_back(P.batch_edge);
    std::sort(N.edges.begin(), N.edges.end());
    for (int e : N.edges) occ[e].insert(i);
    N.elems = 1;
    for (int e : N.edges) N.elems *= P.dim[e];
  }
  std::vector<char> consumed(n_nodes, 0);
  std::set<int> keep(outputs.begin(), outputs.end());
  keep.insert(P.batch_edge);
  for (int t = 0; t < tree->n_steps; ++t) {
    int a = tree->pairs[2 * t], b = tree->pairs[2 * t + 1];
    int c = P.n_leaves + t;
    TN_CHECK(a >= 0 && b >= 0 && a < c && b < c && a != b, TN_ERR_INVALID_ARG, "tree pair refers to a later id");
    TN_CHECK(!consumed[a] && !consumed[b], TN_ERR_INVALID_ARG, "tree consumes an id twice");
    consumed[a] = consumed[b] = 1;
    Step S;
    S.a = a;
    S.b = b;
    S.c = c;
    const auto& Xe = P.nodes[a].edges;
    const auto& Ye = P.nodes[b].edges;
    std::vector<int> shared = set_inter(Xe, Ye);
    std::vector<int> C;
    std::vector<int> uni;
    std::set_union(Xe.begin(), Xe.end(), Ye.begin(), Ye.end(), std::back_inserter(uni));
    for (int e : uni) {
      bool drop = false;
      if (contains(shared, e) && !keep.count(e)) {
        drop = true;
        for (int o : occ[e])
          if (o != a && o != b) drop = false;
      }
      if (!drop) C.push_back(e);
    }
    for (int e : Xe) occ[e].erase(a);
    for (int e : Ye) occ[e].erase(b);
    for (int e : C) occ[e].insert(c);
    Node& N = P.nodes[c];
    N.edges = C;
    N.variant = P.nodes[a].variant || P.nodes[b].variant;
    N.elems = 1;
    for (int e : C) N.elems *= P.dim[e];
    TN_CHECK(N.elems <= (int64_t(1) << 40), TN_ERR_UNSUPPORTED, "intermediate too large");
    P.nodes[a].consumer = t;
    P.nodes[b].consumer = t;
    S.bt = set_inter(shared, C);
    S.k = set_minus(shared, C);
    S.m = set_minus(Xe, Ye);
    S.n = set_minus(Ye, Xe);
    S.variant = N.variant;
    P.steps.push_back(S);
  }
  P.root = n_nodes - 1;
  {
    std::vector<int> want = outputs;
    if (P.nodes[P.root].variant) want.push_back(P.batch_edge);
    std::sort(want.begin(), want.end());
    TN_CHECK(P.nodes[P.root].edges == want, TN_ERR_INVALID_ARG,
             "the tree does not contract the network to its open and block edges");
  }
  const bool hoist = (P.flags & TN_FLAG_HOIST_INVARIANT) && !P.sliced.empty();
  for (auto& S : P.steps) S.hoisted = hoist && !S.variant;

  Builder bld(P);
  bld.assign_layouts();
  for (auto& S : P.steps) {
    bld.fill_gemm(S);
    double bscale = P.nodes[S.c].variant ? (double)P.B : 1.0;
    S.cost_one = S.cost / bscale;
    P.useful_flops_per_slice += 8.0 * S.cost_one;
    if (S.post_perm) S.perm = bld.bit_perm(S.lc_nat, P.nodes[S.c].layout);
    // tensor cores: the larger K-contiguous operand is A (used as stored), the
    // other is expanded to its real 2x2 form
    if (P.skind != KIND_C64) {
      const GemmParams& g = S.gp;
      const bool big = g.K >= 8 && (double)g.nbt * g.M * g.N * g.K >= double(1 << 18);
      // Both operands are stored [bt][free][contracted], so either can be the
      // one read as stored (A); the other is expanded.  Preferred: A owns the
      // result's unit-stride index (the epilogue then stores along TMEM lanes),
      // if the other operand is small enough to expand; else the larger one.
      auto valid = [&](bool swap) {
        S.tc_swap = swap;
        bool ok = false;
        TcRoles r = tc_roles(S, &ok);
        return ok && !P.nodes[r.a_node].leaf && r.M >= 64 &&
               tc_gemm_supported(g.nbt, r.M, r.N, r.K, r.a_bt, r.a_m, 1);
      };
      const bool larger = !a_is_big(P, S);
      bool want = larger;
      if (g.c_n.n > 0 && g.c_n.st[0] == 1)
        want = true;
      else if (g.c_m.n > 0 && g.c_m.st[0] == 1)
        want = false;
      const int64_t expanded = P.nodes[want ? S.a : S.b].elems;
      if (want != larger && expanded > (int64_t(1) << 22)) want = larger;
      bool ok = big && valid(want);
      if (big && !ok && want != larger) ok = valid(larger);
      if (ok) {
        S.tc = true;
        const size_t t = &S - P.steps.data();
        S.hilo = hilo_mask ? (t < hilo_mask->size() && (*hilo_mask)[t] != 0) : (P.flags & TN_FLAG_HILO) != 0;
      } else {
        S.tc_swap = larger;
      }
    }
  }
  // each tensor-core step splits on its own: a producer writes its result hi +
  // lo whenever the step consuming it splits (the output's storage), whatever
  // its own product
  for (size_t t = 0; t < P.steps.size(); ++t) P.steps[t].hilo_group = P.steps[t].tc ? (int)t : -1;
  // storage: tensor-core A operands in 16 bits (hi + lo when split), all else complex64
  for (auto& S : P.steps)
    if (S.tc) {
      Node& A = P.nodes[S.tc_swap ? S.b : S.a];
      A.kind = P.skind;
      A.hilo = S.hilo;
    }
  // a small-K step whose result is the expanded operand of a tensor-core step
  // writes that expanded form itself (per-batch steps, k a multiple of the k tile)
  if (P.skind != KIND_C64)
    for (auto& S : P.steps) {
      if (!S.tc || S.hoisted) continue;
      TcRoles r = tc_roles(S);
      const Node& NB = P.nodes[r.b_node];
      if (NB.leaf || NB.kind != KIND_C64) continue;
      Step& Q = P.steps[r.b_node - P.n_leaves];
      if (Q.hoisted || Q.tc || Q.post_perm || Q.gp.K > 4 || expanded_half_pitch(r.K) != r.K) continue;
      Q.fuse_expand = true;
      S.b_fused = true;
    }
  // row pairs (tc_roles): tensor-core steps whose A rows are K contiguous
  // entries filling at most half a k tile, N small, B expanded by its own
  // launch, no split product
  if (P.skind != KIND_C64)
    for (auto& S : P.steps) {
      if (!S.tc || S.hilo || S.b_fused) continue;
      const TcRoles r = tc_roles(S);
      if (r.a_m != r.K || r.K % 2 != 0 || 4 * r.K > kTcKTile || r.N > 32 || r.M < 256 || r.c_m.n < 1 ||
          r.c_n.n >= kMaxRuns)
        continue;
      if (!tc_gemm_supported(S.gp.nbt, r.M / 2, 2 * r.N, 2 * r.K, r.a_bt, 2 * r.a_m, 1)) continue;
      S.pair_rows = true;
    }
  // micro steps: per-batch CUDA-core steps with at most 2^14 outputs and K <= 4
  // whose operands are leaves, plan-resident results or other micro steps;
  // grouped into subtrees (a step joins its consumer's group)
  for (auto& S : P.steps) {
    if (S.hoisted || S.tc || S.fuse_expand || S.post_perm || S.gp.K > 4) continue;
    if (S.gp.nbt * S.gp.M * S.gp.N > (int64_t(1) << kMicroMaxBits)) continue;
    bool ok = P.nodes[S.a].elems < (int64_t(1) << 31) && P.nodes[S.b].elems < (int64_t(1) << 31);
    for (int x : {S.a, S.b})
      if (!P.nodes[x].leaf) {
        const Step& Q = P.steps[x - P.n_leaves];
        ok = ok && (Q.hoisted || Q.micro);
      }
    S.micro = ok;
  }
  {
    std::vector<int> group(P.steps.size(), -1);
    for (int t = (int)P.steps.size() - 1; t >= 0; --t) {
      if (!P.steps[t].micro) continue;
      const int u = P.nodes[P.steps[t].c].consumer;
      if (u >= 0 && P.steps[u].micro) {
        group[t] = group[u];
      } else {
        group[t] = (int)P.micro_groups.size();
        P.micro_groups.emplace_back();
      }
    }
    for (size_t t = 0; t < P.steps.size(); ++t)
      if (group[t] >= 0) P.micro_groups[group[t]].push_back((int)t);
    // slice-independent groups (their last step, the group's root, depends on
    // no sliced bond) first: they run in a launch of their own
    std::stable_partition(P.micro_groups.begin(), P.micro_groups.end(),
                          [&](const std::vector<int>& g) { return !P.steps[g.back()].variant; });
    P.n_micro_inv = 0;
    for (const auto& g : P.micro_groups) P.n_micro_inv += P.steps[g.back()].variant ? 0 : 1;
  }
  // leaf storage layouts (variant leaves: sliced edges outermost, then the batch copy's order)
  std::vector<std::vector<int>> leaf_src_layout(P.n_leaves);
  for (int i = 0; i < P.n_leaves; ++i) {
    const Node& N = P.nodes[i];
    if (N.variant) {
      for (int e : P.sliced)
        if (contains(P.leaf_edges[i], e)) leaf_src_layout[i].push_back(e);
      for (int e : N.layout)
        if (e != P.batch_edge) leaf_src_layout[i].push_back(e);
    } else {
      leaf_src_layout[i] = N.layout;
    }
  }
  // algorithmic bytes of one sub-network: operands and result once each, at their storage size
  for (auto& S : P.steps) {
    const bool c64 = P.skind == KIND_C64;
    auto per = [&](int x) { return (double)node_bytes(P, x, c64) / (P.nodes[x].variant ? P.B : 1); };
    P.algo_bytes_per_slice += per(S.a) + per(S.b) + per(S.c);
    P.peak_intermediate_bytes = std::max(P.peak_intermediate_bytes, per(S.c));
  }
  P.mem = plan_memory(P, P.skind == KIND_C64, leaf_src_layout, true);
  plan_batch_graph(P);
  if (P.skind != KIND_C64) {
    const MemPlan Mc = plan_memory(P, true, leaf_src_layout, false);
    P.calib_bytes = Mc.plan_bytes + Mc.ws_bytes + total_leaf_elems * 16;
  }
  if (opt->mem_cap_bytes > 0)
    TN_CHECK(P.mem.ws_bytes <= opt->mem_cap_bytes, TN_ERR_OOM, "workspace exceeds mem_cap_bytes");
  {
    const Node& R = P.nodes[P.root];
    auto st = bld.strides(R.layout);
    P.root_sb = R.variant ? st.at(P.batch_edge) : 0;
    P.root_sg = P.block_edge >= 0 ? st.at(P.block_edge) : 0;
    P.root_sj = P.open_edges.empty() ? 0 : st.at(P.open_edges.back());
  }
  if (P.flags & TN_FLAG_PLAN_ONLY) return Pp;

  // ------------------------------------------------------------ device setup
  TN_CUDA(cudaGetDevice(&P.device));
  {
    static std::atomic<uint64_t> next_serial{1};
    P.serial = next_serial.fetch_add(1);
  }
  TN_CUDA(cudaMalloc(&P.d_slice_ids, sizeof(int64_t) * P.B));
  TN_CUDA(cudaMalloc(&P.d_n_valid, sizeof(int32_t)));
  TN_CUDA(cudaMalloc(&P.d_err, sizeof(int)));
  TN_CUDA(cudaMemsetAsync(P.d_err, 0, sizeof(int), stream));
  {
    // calibration slices
    std::vector<int64_t> ids = calibration_ids(P.B, (int)P.sliced.size());
    int32_t nv = P.B;
    TN_CUDA(cudaMemcpyAsync(P.d_slice_ids, ids.data(), sizeof(int64_t) * P.B, cudaMemcpyHostToDevice, stream));
    TN_CUDA(cudaMemcpyAsync(P.d_n_valid, &nv, sizeof(int32_t), cudaMemcpyHostToDevice, stream));
    TN_CUDA(cudaStreamSynchronize(stream));
  }
  void* d_stage = nullptr;
  TN_CUDA(cudaMalloc(&d_stage, std::max<int64_t>(total_leaf_elems * 16, 256)));
  TN_CUDA(cudaMemcpyAsync(d_stage, net->leaf_data, total_leaf_elems * 16, cudaMemcpyHostToDevice, stream));
  // upload every leaf into plan memory `pbase` laid out by `M` in storage kind `kind`
  auto upload_leaves = [&](const MemPlan& M, char* pbase, int kind) {
    for (int i = 0; i < P.n_leaves; ++i) {
      std::map<int, int64_t> hs;
      int64_t acc = 1;
      for (int j = (int)P.leaf_edges[i].size() - 1; j >= 0; --j) {
        hs[P.leaf_edges[i][j]] = acc;
        acc *= P.dim[P.leaf_edges[i][j]];
      }
      StridedCopy sc{};
      sc.nd = (int)leaf_src_layout[i].size();
      int64_t el = 1;
      for (int d = 0; d < sc.nd; ++d) {
        int e = leaf_src_layout[i][d];
        sc.dims[d] = P.dim[e];
        sc.in_stride[d] = hs.at(e);
        el *= P.dim[e];
      }
      const char* src = (const char*)d_stage + P.leaf_off[i] * 16;
      launch_strided_copy_c128(src, pbase + leaf_src_offset(M, P, i), sc, el, kind,
                               ldexp(1.0, -P.nodes[i].exp2), stream);
    }
  };
  auto upload_gather = [&](const MemPlan& M, GatherLeaf** dtab) {
    if (M.gather.empty()) return;
    TN_CUDA(cudaMalloc(dtab, sizeof(GatherLeaf) * M.gather.size()));
    TN_CUDA(cudaMemcpyAsync(*dtab, M.gather.data(), sizeof(GatherLeaf) * M.gather.size(), cudaMemcpyHostToDevice,
                            stream));
  };
  auto run_hoisted = [&](const MemPlan& M, char* pbase, unsigned* amax) {
    void* scratch = nullptr;
    if (M.create_scratch) TN_CUDA(cudaMalloc(&scratch, M.create_scratch));
    Exec X{P, M, pbase, (char*)scratch};
    Recorder R{nullptr, stream};
    for (size_t t = 0; t < P.steps.size(); ++t)
      if (P.steps[t].hoisted) enqueue_step(X, t, stream, R, amax);
    TN_CUDA(cudaStreamSynchronize(stream));
    if (scratch) cudaFree(scratch);
  };

  if (P.skind != KIND_C64) {
    // calibration: one complex64 batch (the seeded slice ids above) records every tensor's
    // largest component; exponents make the stored maxima lie in [1/2, 1)
    MemPlan Mc = plan_memory(P, true, leaf_src_layout, false);
    char *cplan = nullptr, *cws = nullptr;
    unsigned* d_amax = nullptr;
    GatherLeaf* cgather = nullptr;
    auto cleanup = [&] {
      if (cplan) cudaFree(cplan);
      if (cws) cudaFree(cws);
      if (d_amax) cudaFree(d_amax);
      if (cgather) cudaFree(cgather);
    };
    try {
      TN_CUDA(cudaMalloc(&cplan, std::max<int64_t>(Mc.plan_bytes, 256)));
      TN_CUDA(cudaMalloc(&cws, std::max<int64_t>(Mc.ws_bytes, 256)));
      TN_CUDA(cudaMalloc(&d_amax, sizeof(unsigned) * P.nodes.size()));
      TN_CUDA(cudaMemsetAsync(d_amax, 0, sizeof(unsigned) * P.nodes.size(), stream));
      upload_leaves(Mc, cplan, KIND_C64);
      upload_gather(Mc, &cgather);
      std::swap(P.d_gather, cgather);
      run_hoisted(Mc, cplan, d_amax);
      enqueue_batch_mem(P, Mc, cplan, cws, nullptr, 0, stream, nullptr, d_amax, false);
      std::swap(P.d_gather, cgather);
      std::vector<unsigned> h(P.nodes.size());
      TN_CUDA(cudaMemcpyAsync(h.data(), d_amax, sizeof(unsigned) * h.size(), cudaMemcpyDeviceToHost, stream));
      TN_CUDA(cudaStreamSynchronize(stream));
      TN_CUDA(cudaGetLastError());
      // magnitude exponent of every tensor; one that was exactly zero in the sample
      // takes the bound of its product, e_a + e_b + log2(K) (steps are topological)
      std::vector<int> mag(P.nodes.size(), 0);
      for (size_t x = 0; x < P.nodes.size(); ++x) {
        float a;
        std::memcpy(&a, &h[x], 4);
        TN_CHECK(std::isfinite(a), TN_ERR_NUMERIC, "calibration found a non-finite value");
        int e = 0;
        if (a > 0) {
          std::frexp(a, &e);
        } else if (!P.nodes[x].leaf) {
          const Step& S = P.steps[x - P.n_leaves];
          e = mag[S.a] + mag[S.b] + ilog2(std::max<int64_t>(S.gp.K, 1));
        }
        mag[x] = e;
        P.nodes[x].exp2 = P.nodes[x].kind == KIND_C64 ? 0 : e;
      }
      for (auto& S : P.steps)
        if (S.tc) S.bexp = mag[S.tc_swap ? S.a : S.b];
    } catch (...) {
      cudaStreamSynchronize(stream);
      cleanup();
      cudaFree(d_stage);
      throw;
    }
    cleanup();
  }
  if (P.mem.micro) {
    // fused small-step descriptors (scales need the calibrated exponents).
    // Each group (one CTA) keeps, where they fit, its descriptors, the
    // operands it reads from outside (copied in before its first step) and its
    // inner results (consumed by the group's next steps) in shared memory:
    // [descriptors | first-fit arena over the group's step order].
    const MemPlan& M = P.mem;
    const bool c64 = M.c64;
    std::vector<MicroStep> desc;
    std::vector<MicroGroup> groups;
    std::vector<MicroLoad> loads;
    constexpr int64_t kDescMax = 48 * 1024;
    P.micro_smem = 0;
    for (const auto& grp : P.micro_groups) {
      MicroGroup G{};
      G.first_step = (int32_t)desc.size();
      G.n_steps = (int32_t)grp.size();
      G.first_load = (int32_t)loads.size();
      const int64_t desc_bytes = (int64_t)grp.size() * (int64_t)sizeof(MicroStep);
      G.desc_in_smem = desc_bytes <= kDescMax ? 1 : 0;
      const int64_t base = G.desc_in_smem ? round_up(desc_bytes, 16) : 0;
      std::set<int> produced;
      for (int t : grp) produced.insert(P.steps[t].c);
      const int root = P.steps[grp.back()].c;
      auto is_c64 = [&](int x) { return c64 || P.nodes[x].kind == KIND_C64; };
      std::map<int, int64_t> soff;  // node -> arena offset
      Arena A;
      A.align = 16;
      bool fits = true;
      for (int t : grp)
        for (int x : {P.steps[t].a, P.steps[t].b})
          if (!produced.count(x) && !soff.count(x)) {
            fits = fits && is_c64(x);
            soff[x] = A.alloc(node_bytes(P, x, c64));
          }
      for (int t : grp) {
        const Step& S = P.steps[t];
        if (S.c != root) {
          fits = fits && is_c64(S.c) && !(!c64 && P.nodes[S.c].hilo);
          soff[S.c] = A.alloc(node_bytes(P, S.c, c64));
        }
        for (int x : {S.a, S.b})
          if (soff.count(x)) A.release(soff[x]);
      }
      fits = fits && base + A.peak <= kMicroSmemBytes;
      if (!fits) soff.clear();
      for (const auto& kv : soff) {
        const int x = kv.first;
        if (produced.count(x)) continue;
        MicroLoad L{};
        L.src_off = M.off[x];
        L.smem_off = (int32_t)(base + kv.second);
        L.elems = (int32_t)(node_bytes(P, x, c64) / 8);
        L.src_loc = M.in_plan[x] ? 0 : 1;
        loads.push_back(L);
      }
      G.n_loads = (int32_t)(loads.size() - (size_t)G.first_load);
      P.micro_smem = std::max<int>(P.micro_smem, (int)(base + (fits ? A.peak : 0)));
      for (int t : grp) {
        const Step& S = P.steps[t];
        const Node& NC = P.nodes[S.c];
        MicroStep d{};
        fill_micro_weights(S.gp, d);
        auto where = [&](int x, int8_t& loc, int64_t& off) {
          if (soff.count(x)) {
            loc = 2;
            off = base + soff[x];
          } else {
            loc = M.in_plan[x] ? 0 : 1;
            off = M.off[x];
          }
        };
        where(S.a, d.a_loc, d.a_off);
        where(S.b, d.b_loc, d.b_off);
        TN_CHECK(!M.in_plan[S.c], TN_ERR_INVALID_ARG, "internal: micro result in plan memory");
        where(S.c, d.c_loc, d.c_off);
        d.out_kind = (int8_t)(c64 ? KIND_C64 : NC.kind);
        d.out_hilo = (int8_t)(!c64 && NC.hilo ? 1 : 0);
        TN_CHECK(d.c_loc == 1 || (d.out_kind == KIND_C64 && !d.out_hilo), TN_ERR_INVALID_ARG,
                 "internal: a shared-memory micro result must be complex64");
        d.c2_off = d.c_off + (d.out_hilo ? NC.elems * 4 : 0);
        d.scale = c64 ? 1.0f : ldexpf(1.0f, P.nodes[S.a].exp2 + P.nodes[S.b].exp2 - NC.exp2);
        desc.push_back(d);
        P.micro_flops += 8.0 * S.cost;
        P.micro_bytes += (double)(node_bytes(P, S.a, c64) + node_bytes(P, S.b, c64) + node_bytes(P, S.c, c64));
      }
      groups.push_back(G);
    }
    TN_CUDA(cudaMalloc(&P.d_micro, sizeof(MicroStep) * desc.size()));
    TN_CUDA(cudaMalloc(&P.d_micro_groups, sizeof(MicroGroup) * groups.size()));
    TN_CUDA(cudaMalloc(&P.d_micro_loads, sizeof(MicroLoad) * std::max<size_t>(loads.size(), 1)));
    TN_CUDA(cudaMemcpyAsync(P.d_micro, desc.data(), sizeof(MicroStep) * desc.size(), cudaMemcpyHostToDevice,
                            stream));
    TN_CUDA(cudaMemcpyAsync(P.d_micro_groups, groups.data(), sizeof(MicroGroup) * groups.size(),
                            cudaMemcpyHostToDevice, stream));
    if (!loads.empty())
      TN_CUDA(cudaMemcpyAsync(P.d_micro_loads, loads.data(), sizeof(MicroLoad) * loads.size(),
                              cudaMemcpyHostToDevice, stream));
  }
  TN_CUDA(cudaMalloc(&P.d_plan, std::max<int64_t>(P.mem.plan_bytes, 256)));
  upload_leaves(P.mem, (char*)P.d_plan, KIND_C64);
  upload_gather(P.mem, &P.d_gather);
  run_hoisted(P.mem, (char*)P.d_plan, nullptr);
  TN_CUDA(cudaStreamSynchronize(stream));
  TN_CUDA(cudaGetLastError());
  cudaFree(d_stage);
  int h_err = 0;
  TN_CUDA(cudaMemcpy(&h_err, P.d_err, sizeof(int), cudaMemcpyDeviceToHost));
  TN_CHECK(h_err == 0, TN_ERR_TIMEOUT, "a bounded device wait timed out during plan creation");
  TN_CUDA(cudaStreamCreateWithFlags(&P.capture_stream, cudaStreamNonBlocking));
  return Pp;
}

// ---------------------------------------------------------------- tuning
std::vector<TcForm> tc_step_forms(const Plan& P, size_t t) {
  const Step& S = P.steps[t];
  if (!S.tc || S.hoisted || P.mem.c64) return {};
  return tc_forms(P, S);
}

void drop_graph(Plan& P) {
  ++P.generation;  // batched graphs holding the old launch forms no longer match
  if (P.graph) cudaGraphExecDestroy(P.graph);
  P.graph = nullptr;
  P.graph_ws = P.graph_amps = nullptr;
  P.graph_acc = -1;
}

// ---------------------------------------------------------------- execute
// Direct launches only (no graph is built or replayed).
void run_batch_direct(Plan& P, void* ws, void* amps, int accumulate, cudaStream_t stream) {
  enqueue_batch_mem(P, P.mem, (char*)P.d_plan, ws, amps, accumulate, stream, nullptr, nullptr, false);
  TN_CUDA(cudaGetLastError());
}

void run_batch(Plan& P, void* ws, void* amps, int accumulate, cudaStream_t stream,
               std::vector<LaunchRecord>* rec) {
  if ((P.flags & TN_FLAG_NO_GRAPH) || rec) {
    enqueue_batch_mem(P, P.mem, (char*)P.d_plan, ws, amps, accumulate, stream, rec, nullptr, false);
    TN_CUDA(cudaGetLastError());
    return;
  }
  if (!P.graph || P.graph_ws != ws || P.graph_amps != amps || P.graph_acc != accumulate) {
    if (P.graph) {
      cudaGraphExecDestroy(P.graph);
      P.graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    if (!(P.flags & TN_FLAG_SERIAL_GRAPH)) make_graph_resources(P);
    TN_CUDA(cudaStreamBeginCapture(P.capture_stream, cudaStreamCaptureModeThreadLocal));
    try {
      if (P.flags & TN_FLAG_SERIAL_GRAPH)
        enqueue_batch_mem(P, P.mem, (char*)P.d_plan, ws, amps, accumulate, P.capture_stream, nullptr, nullptr,
                          false);
      else
        enqueue_batch_graph(P, ws, amps, accumulate, P.capture_stream);
    } catch (...) {
      cudaStreamEndCapture(P.capture_stream, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    cudaError_t e = cudaStreamEndCapture(P.capture_stream, &g);
    if (e != cudaSuccess) fail(TN_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&P.graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) fail(TN_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    P.graph_ws = ws;
    P.graph_amps = amps;
    P.graph_acc = accumulate;
  }
  TN_CUDA(cudaGraphLaunch(P.graph, stream));
}

}  // namespace tn
