"""Contraction path and slicing search (host side, once per circuit).

The paper searches contraction paths under a memory cap and slices edges
until the largest intermediate fits (arXiv 2406.18889, Sec. III "Optimizing
tensor contraction": slicing fixes edge values and sums the sub-networks,
trading time for space).  Its own path optimiser is not described; this
module uses a greedy rule with seeded random restarts:

* greedy: repeatedly contract the pair of tensors sharing an edge with the
  lowest score size(C) - alpha (size(A) + size(B)); restarts add seeded Gumbel
  noise to the score in the log domain (temperature T) and sweep alpha; the
  tree with the lowest cost wins.  Ties break on ids, so results are
  deterministic for a given seed.
* slicing: with a path fixed, repeatedly pick the bond whose removal most
  reduces the largest intermediate (then the total cost), up to the requested
  count or until the largest intermediate fits the cap.

* recursive bisection (``partition_path``): for deep circuits greedy stems
  grow wide; splitting the tensor graph into balanced halves with a small cut
  (spectral bisection on the graph whose edge weights are the bonds' log2
  dimensions, then Fiduccia-Mattheyses moves), recursively, and contracting
  small parts greedily gives trees whose intermediates follow the cuts.
  ``plan_tree(method="both")`` keeps the cheaper of the two searches.
* subtree reconfiguration (``reconfigure``): a tensor's edges after contraction
  depend only on which leaves it holds, so the subtree between any node and a
  frontier of up to 8 of its descendants can be re-contracted in the cheapest
  order, found exactly by dynamic programming over frontier subsets; and
  slicing interleaved with it (``slice_and_reconfigure``: a few bonds sliced at
  a time, the rest of the network reconfigured in between, sliced bonds given
  back while the cap allows).  ``plan_tree(refine=True)`` and
  ``memory_cap_sweep(refine=True)`` add these trees to the candidates.

All sizes are log2 element counts (every edge dimension is a power of two).
Costs are complex multiply-adds: a step costs the product of the dimensions of
every edge of its two operands (batch x M x N x K).
"""
from __future__ import annotations

import heapq
import math
from dataclasses import dataclass
from typing import Dict, FrozenSet, List, Optional, Sequence, Tuple

import numpy as np

from .network import TensorNetwork


@dataclass
class Tree:
    pairs: List[Tuple[int, int]]            # SSA: leaf i = i, step t makes n_leaves + t
    sliced_edges: List[int]                  # slice id bit i <-> value of sliced_edges[i]
    log2_max_intermediate: float             # of one sub-network
    cost_per_slice: float                    # complex MACs of one sub-network
    cost_variant_per_slice: float            # complex MACs of the steps that depend on a slice
    n_leaves: int


def log2dims(tn: TensorNetwork) -> List[float]:
    out = []
    for d in tn.edge_dim:
        if d <= 0 or d & (d - 1):
            raise ValueError("edge dimensions must be powers of two")
        out.append(float(int(d).bit_length() - 1))
    return out


def _result(a: FrozenSet[int], b: FrozenSet[int], occ, keep, i, j) -> FrozenSet[int]:
    out = set(a ^ b)
    for e in a & b:
        if e in keep or (occ[e] - {i, j}):
            out.add(e)
    return frozenset(out)


def greedy(leaves: Sequence[FrozenSet[int]], lg: Sequence[float], keep: FrozenSet[int],
           alpha: float = 1.0, temperature: float = 0.0, seed: int = 0) -> List[Tuple[int, int]]:
    """Greedy pairwise order over ``leaves`` (edge sets); ``keep`` = output edges."""
    rng = np.random.default_rng(seed)
    live: Dict[int, FrozenSet[int]] = {i: frozenset(s) for i, s in enumerate(leaves)}
    occ: Dict[int, set] = {}
    for i, s in live.items():
        for e in s:
            occ.setdefault(e, set()).add(i)
    size = lambda s: sum(lg[e] for e in s)  # noqa: E731
    heap: list = []

    def push(i, j):
        if i > j:
            i, j = j, i
        c = _result(live[i], live[j], occ, keep, i, j)
        sc = size(c)
        score = 2.0 ** sc - alpha * (2.0 ** size(live[i]) + 2.0 ** size(live[j]))
        if temperature > 0:
            gumbel = -math.log(-math.log(rng.random() + 1e-300))
            score = math.copysign(math.log2(abs(score) + 1.0), score) - temperature * gumbel
        heapq.heappush(heap, (score, sc, i, j))

    seen = set()
    for e, ids in occ.items():
        ids = sorted(ids)
        for x in range(len(ids)):
            for y in range(x + 1, len(ids)):
                if (ids[x], ids[y]) not in seen:
                    seen.add((ids[x], ids[y]))
                    push(ids[x], ids[y])
    pairs = []
    nxt = len(leaves)
    while len(live) > 1:
        if heap:
            _, _, i, j = heapq.heappop(heap)
            if i not in live or j not in live:
                continue
        else:  # disconnected parts: outer product of the two smallest
            ids = sorted(live, key=lambda t: (size(live[t]), t))
            i, j = sorted(ids[:2])
        c = _result(live[i], live[j], occ, keep, i, j)
        pairs.append((i, j))
        for e in live[i] | live[j]:
            occ[e].discard(i)
            occ[e].discard(j)
        del live[i], live[j]
        k = nxt
        nxt += 1
        live[k] = c
        nbrs = set()
        for e in c:
            nbrs |= occ[e]
            occ[e].add(k)
        for m in sorted(nbrs):
            push(m, k)
    return pairs


def invariant_first(leaves: Sequence[FrozenSet[int]], pairs, sliced) -> List[Tuple[int, int]]:
    """The same tree with every step that depends on no sliced bond listed
    before the others, each group in its original order (still children
    before parents: a slice-independent step only consumes slice-independent
    tensors).  The library then gives the slice-independent subtrees their
    own workspace region, so they can run concurrently with the rest of a
    batch.  Returns new SSA pairs."""
    sl = set(sliced)
    L = len(leaves)
    variant = [bool(set(x) & sl) for x in leaves]
    for (i, j) in pairs:
        variant.append(variant[i] or variant[j])
    order = [t for t in range(len(pairs)) if not variant[L + t]] + \
            [t for t in range(len(pairs)) if variant[L + t]]
    new_id = {i: i for i in range(L)}
    out: List[Tuple[int, int]] = []
    for t in order:
        i, j = pairs[t]
        out.append((new_id[i], new_id[j]))
        new_id[L + t] = L + len(out) - 1
    return out


def replay(leaves: Sequence[FrozenSet[int]], pairs, keep: FrozenSet[int]):
    """Edge sets of every node (leaves then steps) along ``pairs``."""
    nodes = [frozenset(s) for s in leaves]
    occ: Dict[int, set] = {}
    for i, s in enumerate(nodes):
        for e in s:
            occ.setdefault(e, set()).add(i)
    for (i, j) in pairs:
        k = len(nodes)
        c = _result(nodes[i], nodes[j], occ, keep, i, j)
        for e in nodes[i] | nodes[j]:
            occ[e].discard(i)
            occ[e].discard(j)
        for e in c:
            occ[e].add(k)
        nodes.append(c)
    return nodes


def _incidence(nodes, pairs, n_leaves, n_edges, lg):
    """Per-node and per-step log2 sizes and edge-incidence matrices."""
    node_sz = np.array([sum(lg[e] for e in s) for s in nodes])
    node_inc = np.zeros((n_edges, len(nodes)), dtype=np.float64)
    for k, s in enumerate(nodes):
        for e in s:
            node_inc[e, k] = lg[e]
    step_sets = [nodes[i] | nodes[j] for (i, j) in pairs]
    step_sz = np.array([sum(lg[e] for e in s) for s in step_sets])
    step_inc = np.zeros((n_edges, len(pairs)), dtype=np.float64)
    for t, s in enumerate(step_sets):
        for e in s:
            step_inc[e, t] = lg[e]
    return node_sz, node_inc, step_sz, step_inc


def tree_stats(leaves, pairs, lg, keep, sliced=()):
    """(log2 max intermediate, cost per slice, variant cost per slice) of a path
    whose sliced edges are removed from the leaves."""
    sl = set(sliced)
    stripped = [frozenset(x - sl) for x in leaves]
    nodes = replay(stripped, pairs, keep)
    L = len(leaves)
    variant = [bool(set(x) & sl) for x in leaves]
    mx = max(sum(lg[e] for e in s) for s in nodes)
    cost = vcost = 0.0
    for (i, j) in pairs:
        c = 2.0 ** sum(lg[e] for e in (nodes[i] | nodes[j]))
        v = variant[i] or variant[j]
        variant.append(v)
        cost += c
        vcost += c if v else 0.0
    del L
    return mx, cost, vcost


def choose_slices(leaves, pairs, lg, keep, n_edges: int, n_sliced: int = 0,
                  cap_log2: Optional[float] = None) -> List[int]:
    """Greedy slicing of bonds along a fixed path (vectorised over candidates)."""
    nodes = replay(leaves, pairs, keep)
    count: Dict[int, int] = {}
    for s in leaves:
        for e in s:
            count[e] = count.get(e, 0) + 1
    bonds = np.array(sorted(e for e, c in count.items() if c == 2 and e not in keep), dtype=np.int64)
    node_sz, node_inc, step_sz, step_inc = _incidence(nodes, pairs, len(leaves), n_edges, lg)
    chosen: List[int] = []
    cur_node = node_sz.copy()
    cur_step = step_sz.copy()
    lg_arr = np.asarray(lg)
    while True:
        mx = cur_node.max()
        if len(chosen) >= n_sliced and (cap_log2 is None or mx <= cap_log2):
            break
        mask = np.ones(len(bonds), dtype=bool)
        for e in chosen:
            mask &= bonds != e
        cand = bonds[mask]
        if cand.size == 0:
            raise ValueError("no bond left to slice")
        new_max = (cur_node[None, :] - node_inc[cand]).max(axis=1)
        s_log = sum(lg[e] for e in chosen)
        new_cost = np.exp2(cur_step[None, :] - step_inc[cand]).sum(axis=1) * np.exp2(s_log + lg_arr[cand])
        order = np.lexsort((cand, new_cost, new_max))
        e = int(cand[order[0]])
        chosen.append(e)
        cur_node = cur_node - node_inc[e]
        cur_step = cur_step - step_inc[e]
    return chosen


# Multiply-adds per element moved at which a 16-bit tensor-core step is as long
# bound by HBM as by the tensor pipe: 8 real flops per complex MAC at ~1.94
# PFLOP/s against 4 bytes per complex element at ~6.7 TB/s.
ALPHA_TC = 145.0


SWEEP = [(1.0, 0.0), (2.0, 0.0), (1.0, 0.25), (1.5, 0.25), (2.0, 0.25), (2.0, 0.5), (1.5, 0.5),
         (3.0, 0.5), (2.0, 0.75)]


# ------------------------------------------------------------ recursive bisection
def _weighted_graph(leaves, lg, keep):
    """Adjacency of the tensors: a bond shared by tensors i and j adds its log2
    dimension to w(i, j) (a hyper-edge over m tensors adds lg / (m - 1) to each
    pair); output edges do not join tensors."""
    occ: Dict[int, List[int]] = {}
    for i, s in enumerate(leaves):
        for e in s:
            occ.setdefault(e, []).append(i)
    adj: List[Dict[int, float]] = [dict() for _ in leaves]
    for e, ids in occ.items():
        if len(ids) < 2 or e in keep:
            continue
        w = lg[e] / (len(ids) - 1)
        for x in range(len(ids)):
            for y in range(x + 1, len(ids)):
                a, b = ids[x], ids[y]
                adj[a][b] = adj[a].get(b, 0.0) + w
                adj[b][a] = adj[b].get(a, 0.0) + w
    return adj, occ


def _bisect(V: List[int], adj, imbalance: float) -> np.ndarray:
    """Side (False / True) of every vertex of V: connected components are dealt
    out whole; a connected V is cut at the smallest-weight split, along its
    Fiedler vector, whose larger side holds at most (1 + imbalance) / 2 of V."""
    n = len(V)
    pos = {v: i for i, v in enumerate(V)}
    W = np.zeros((n, n))
    for v in V:
        i = pos[v]
        for u, w in adj[v].items():
            j = pos.get(u)
            if j is not None:
                W[i, j] = w
    # components
    comp = -np.ones(n, dtype=np.int64)
    n_comp = 0
    for s0 in range(n):
        if comp[s0] >= 0:
            continue
        stack = [s0]
        comp[s0] = n_comp
        while stack:
            x = stack.pop()
            for j in np.nonzero(W[x])[0]:
                if comp[j] < 0:
                    comp[j] = n_comp
                    stack.append(int(j))
        n_comp += 1
    side = np.zeros(n, dtype=bool)
    if n_comp > 1:
        sizes = np.bincount(comp, minlength=n_comp)
        a = b = 0
        for c in np.argsort(-sizes, kind="stable"):
            if a <= b:
                a += sizes[c]
            else:
                side[comp == c] = True
                b += sizes[c]
        return side
    L = np.diag(W.sum(axis=1)) - W
    _, vec = np.linalg.eigh(L)
    order = np.argsort(vec[:, 1], kind="stable")
    lo = max(1, int(math.floor(n * (1 - imbalance) / 2)))
    hi = min(n - 1, int(math.ceil(n * (1 + imbalance) / 2)))
    cut, best, best_k = 0.0, None, lo
    to_b = np.zeros(n)
    total = W.sum(axis=1)
    for t in range(n - 1):
        x = order[t]
        cut += (total[x] - to_b[x]) - to_b[x]
        to_b += W[:, x]
        if lo <= t + 1 <= hi and (best is None or cut < best - 1e-9):
            best, best_k = cut, t + 1
    side[order[:best_k]] = True
    return side


def _refine(V: List[int], side: np.ndarray, adj, imbalance: float, passes: int = 3) -> np.ndarray:
    """Fiduccia-Mattheyses passes: move the unlocked vertex of largest gain (cut
    weight removed) within the balance window, keep the best prefix."""
    n = len(V)
    pos = {v: i for i, v in enumerate(V)}
    nb = [[(pos[u], w) for u, w in adj[v].items() if u in pos] for v in V]
    lo, hi = n * (1 - imbalance) / 2, n * (1 + imbalance) / 2
    cur = sum(w for i in range(n) for j, w in nb[i] if j > i and side[i] != side[j])
    for _ in range(passes):
        gain = np.array([sum(w if side[i] != side[j] else -w for j, w in nb[i]) for i in range(n)])
        locked = np.zeros(n, dtype=bool)
        s = side.copy()
        n_true = int(s.sum())
        c, best_c, best_s = cur, cur, side.copy()
        for _m in range(n):
            cand = np.nonzero(~locked)[0]
            ok = np.where(s[cand], n_true - 1 >= lo, n_true + 1 <= hi)
            cand = cand[ok]
            if cand.size == 0:
                break
            i = int(cand[np.argmax(gain[cand])])
            c -= gain[i]
            n_true += -1 if s[i] else 1
            s[i] = not s[i]
            locked[i] = True
            for j, w in nb[i]:
                gain[j] += -2.0 * w if s[i] == s[j] else 2.0 * w
            gain[i] = -gain[i]
            if c < best_c - 1e-9:
                best_c, best_s = c, s.copy()
        if best_c < cur - 1e-9:
            cur, side = best_c, best_s
        else:
            break
    return side


def partition_path(leaves: Sequence[FrozenSet[int]], lg: Sequence[float], keep: FrozenSet[int],
                   imbalance: float = 0.4, leaf_size: int = 12) -> List[Tuple[int, int]]:
    """Contraction path by recursive bisection of the tensor graph; parts of at
    most ``leaf_size`` tensors are contracted greedily (their edges leaving the
    part are kept open)."""
    adj, occ = _weighted_graph(leaves, lg, keep)

    def inside(V):
        Vs = sorted(V)
        members = set(Vs)
        sub_keep = set(keep)
        for v in Vs:
            for e in leaves[v]:
                if any(u not in members for u in occ[e]):
                    sub_keep.add(e)
        nodes: List = list(Vs)
        for (i, j) in greedy([leaves[v] for v in Vs], lg, frozenset(sub_keep)):
            nodes.append((nodes[i], nodes[j]))
        return nodes[-1]

    def rec(V):
        if len(V) <= leaf_size:
            return inside(V)
        side = _refine(V, _bisect(V, adj, imbalance), adj, imbalance)
        A = [v for v, t in zip(V, side) if not t]
        B = [v for v, t in zip(V, side) if t]
        if not A or not B:
            return inside(V)
        return (rec(A), rec(B))

    pairs: List[Tuple[int, int]] = []
    nxt = [len(leaves)]

    def emit(x):
        if isinstance(x, int):
            return x
        a, b = emit(x[0]), emit(x[1])
        pairs.append((a, b))
        nxt[0] += 1
        return nxt[0] - 1

    emit(rec(list(range(len(leaves)))))
    return pairs


PARTITION_IMBALANCES = (0.2, 0.3, 0.4, 0.5)


def _candidate_trees(job):
    """Slicing (and with ``refine`` the refined trees) of one candidate path:
    a list of (pairs, sliced).  Top level, so that a process pool can run it."""
    leaves, pairs, lg, keep, n_edges, n_sliced, cap_log2, sliced, refine, groups, timing = job
    out = _candidate_trees_flops(leaves, pairs, lg, keep, n_edges, n_sliced, cap_log2, sliced, refine, groups)
    if timing is None:
        return out
    batch_log2, alpha = timing
    return out + [(retime(leaves, p, lg, keep, sl, batch_log2, alpha), sl) for p, sl in out]


def _candidate_trees_flops(leaves, pairs, lg, keep, n_edges, n_sliced, cap_log2, sliced, refine, groups):
    if sliced is None:
        sl = choose_slices(leaves, pairs, lg, keep, n_edges, n_sliced, cap_log2) \
            if (n_sliced or cap_log2 is not None) else []
    else:
        sl = list(sliced)
    out = [(pairs, sl)]
    if not refine:
        return out
    if sliced is None and cap_log2 is not None and not n_sliced:
        for g in groups:
            try:
                out.append(slice_and_reconfigure(leaves, pairs, lg, keep, n_edges, cap_log2, group=g))
            except ValueError:
                pass
        return out
    # a fixed slice set: reconfigure within the cap, or within the tree's own
    # largest intermediate when there is no cap
    mx0, _, _ = tree_stats(leaves, pairs, lg, keep, sl)
    stripped = [frozenset(x - set(sl)) for x in leaves]
    lim = cap_log2 if cap_log2 is not None else mx0
    out.append((reconfigure(stripped, pairs, lg, keep, cap_log2=lim), list(sl)))
    if sliced is None and n_sliced:
        # or the given number of bonds chosen a few at a time, with
        # reconfiguration in between
        out.append(slice_count_and_reconfigure(leaves, pairs, lg, keep, n_edges, n_sliced))
    return out


def plan_tree(tn: TensorNetwork, n_sliced: int = 0, cap_log2: Optional[float] = None,
              restarts: int = 4, seed: int = 0, sliced: Optional[Sequence[int]] = None,
              method: str = "greedy", refine: bool = False, groups: Sequence[int] = (2, 4),
              workers: int = 0, objective: str = "flops", batch_log2: Optional[int] = None,
              alpha: float = ALPHA_TC) -> Tree:
    """Search paths -- the greedy alpha/temperature sweep (``restarts`` seeds per
    noisy setting), recursive bisection at several balance windows, or both
    (``method``) -- slice each (unless ``sliced`` is given), keep the cheapest
    total.  ``refine``: every candidate is also re-optimised by subtree
    reconfiguration -- with a cap, slicing interleaved with reconfiguration
    (``slice_and_reconfigure``, each group size in ``groups``); otherwise the
    network without its sliced bonds is reconfigured, its intermediates kept
    within the cap or, without one, within the unrefined tree's largest.
    ``workers`` > 1 slices and refines the candidates in that many processes
    (started with spawn); the result does not depend on it.

    ``objective``: "flops" keeps the tree with the fewest multiply-adds over
    all slices; "time" also re-optimises every candidate for ``time_cost``
    (multiply-adds plus ``alpha`` per element moved, slices run
    2^``batch_log2`` at a time, default all of them) and keeps the tree with
    the lowest estimated time over all batches."""
    if method not in ("greedy", "partition", "both"):
        raise ValueError("method must be greedy, partition or both")
    if objective not in ("flops", "time"):
        raise ValueError("objective must be flops or time")
    lg = log2dims(tn)
    keep = frozenset(tn.output_edges())
    leaves = [frozenset(e) for e in tn.leaf_edges]
    candidates = []
    if method in ("greedy", "both"):
        for (alpha, T) in SWEEP:
            for r in range(restarts if T > 0 else 1):
                candidates.append(greedy(leaves, lg, keep, alpha, T, seed + 1000 * r + 7))
    if method in ("partition", "both"):
        for imb in PARTITION_IMBALANCES:
            candidates.append(partition_path(leaves, lg, keep, imbalance=imb))
    timing = None
    if objective == "time":
        nb = len(sliced) if sliced is not None else n_sliced
        timing = (int(batch_log2) if batch_log2 is not None else int(nb), float(alpha))
    jobs = [(leaves, pairs, lg, keep, len(tn.edge_dim), n_sliced, cap_log2,
             None if sliced is None else list(sliced), refine, tuple(groups), timing) for pairs in candidates]
    if workers > 1 and len(jobs) > 1:
        import multiprocessing
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(max_workers=min(workers, len(jobs)),
                                 mp_context=multiprocessing.get_context("spawn")) as ex:
            results = list(ex.map(_candidate_trees, jobs))
    else:
        results = [_candidate_trees(j) for j in jobs]
    best = None
    for trees in results:
        for pairs, sl in trees:
            mx, cost, vcost = tree_stats(leaves, pairs, lg, keep, sl)
            if cap_log2 is not None and mx > cap_log2:
                continue
            if timing is None:
                key = (cost * 2.0 ** len(sl), mx)
            else:
                bl = min(timing[0], len(sl))
                key = (time_cost(leaves, pairs, lg, keep, sl, bl, timing[1]) * 2.0 ** (len(sl) - bl), mx)
            if best is None or key < best[0]:
                best = (key, pairs, sl, mx, cost, vcost)
    if best is None:
        raise ValueError("no path fits the memory cap")
    _, pairs, sl, mx, cost, vcost = best
    pairs = invariant_first(leaves, pairs, sl)
    return Tree(pairs=pairs, sliced_edges=list(sl), log2_max_intermediate=mx,
                cost_per_slice=cost, cost_variant_per_slice=vcost, n_leaves=len(leaves))


# ------------------------------------------------------------ memory vs complexity
def memory_cap_sweep(tn: TensorNetwork, caps_log2: Sequence[float], method: str = "partition",
                     max_sliced: int = 62, restarts: int = 1, seed: int = 0, refine: bool = False,
                     groups: Sequence[int] = (2, 4)) -> List[dict]:
    """Time complexity against the memory cap (paper Sec. III: a larger cap on
    the largest intermediate means fewer sliced bonds and less total work).

    Each candidate path (recursive bisection at every balance window, the greedy
    sweep, or both) is found once -- it does not depend on the cap -- and then
    sliced greedily down to every cap.  Returns one entry per cap, ascending:
    ``cap_log2``, ``n_sliced``, ``cost_per_slice`` and ``total`` (complex
    multiply-adds over all slices) of the cheapest total found, or only
    ``cap_log2`` when no candidate fits within ``max_sliced`` sliced bonds.  A
    tree found for a smaller cap also fits a larger one and is carried forward,
    so totals never rise with the cap.  ``refine``: each candidate is also sliced with interleaved subtree
    reconfiguration (``slice_and_reconfigure``, every group size in ``groups``)."""
    if method not in ("greedy", "partition", "both"):
        raise ValueError("method must be greedy, partition or both")
    lg = log2dims(tn)
    keep = frozenset(tn.output_edges())
    leaves = [frozenset(e) for e in tn.leaf_edges]
    candidates = []
    if method in ("partition", "both"):
        for imb in PARTITION_IMBALANCES:
            candidates.append(("bisection %.1f" % imb, partition_path(leaves, lg, keep, imbalance=imb)))
    if method in ("greedy", "both"):
        for (alpha, T) in SWEEP:
            for r in range(restarts if T > 0 else 1):
                candidates.append(("greedy %.2g/%.2g" % (alpha, T),
                                   greedy(leaves, lg, keep, alpha, T, seed + 1000 * r + 7)))
    out = []
    for cap in sorted(caps_log2):
        best = None
        for name, pairs in candidates:
            trees = []
            try:
                trees.append((name, pairs, choose_slices(leaves, pairs, lg, keep, len(tn.edge_dim), 0, cap)))
            except ValueError:
                pass
            if refine:
                for g in groups:
                    try:
                        p2, sl2 = slice_and_reconfigure(leaves, pairs, lg, keep, len(tn.edge_dim), cap, group=g)
                    except ValueError:
                        continue
                    trees.append((f"{name} + reconfiguration (groups of {g})", p2, sl2))
            for label, p2, sl in trees:
                if len(sl) > max_sliced:
                    continue
                mx, cost, _ = tree_stats(leaves, p2, lg, keep, sl)
                total = cost * 2.0 ** len(sl)
                if best is None or total < best["total"]:
                    best = dict(cap_log2=cap, n_sliced=len(sl), cost_per_slice=cost, total=total,
                                log2_max_intermediate=mx, path=label, pairs=p2, sliced=list(sl))
        # a tree within a smaller cap fits this one too
        prev = next((r for r in reversed(out) if "total" in r), None)
        if prev is not None and (best is None or prev["total"] < best["total"]):
            best = dict(prev, cap_log2=cap, path=prev["path"] + f" (found for cap 2^{prev['cap_log2']:g})"
                        if "found for cap" not in prev["path"] else prev["path"])
        out.append(best if best is not None else dict(cap_log2=cap))
    return out


# ------------------------------------------------------------ subtree reconfiguration
def reconfigure(leaves: Sequence[FrozenSet[int]], pairs, lg: Sequence[float], keep: FrozenSet[int],
                cap_log2: Optional[float] = None, size: int = 8, sweeps: int = 3, alpha: float = 0.0):
    """Local re-optimisation of a contraction tree (the path stays a tree over the
    same leaves with the same output).

    A tensor's edges after contraction depend only on which leaves it holds, so
    any subtree can be re-contracted freely between its root and a frontier of
    its descendants.  For every node, a frontier of up to ``size`` tensors is
    grown by expanding the most expensive step inside it; the cheapest order
    of contracting the frontier back into the node is found exactly by dynamic
    programming over frontier subsets (a subset's result keeps the edges that
    also occur outside it), and replaces the subtree when cheaper with every
    new intermediate within ``cap_log2``.  Sweeps repeat while the cost falls.
    Costs as in ``tree_stats``: per step, the product of the dimensions of all
    edges of both operands.  Returns the new SSA pairs."""
    L = len(leaves)
    nodes = replay(leaves, pairs, keep)
    ordinary = 0
    special = []
    for s in nodes:
        for e in s:
            if lg[e] == 1.0:
                ordinary |= 1 << e
    for e in {e for s in nodes for e in s}:
        if lg[e] != 1.0:
            special.append((1 << e, lg[e]))

    def weight(m: int) -> float:
        w = float((m & ordinary).bit_count())
        for bit, v in special:
            if m & bit:
                w += v
        return w

    mask = [0] * len(nodes)
    for i, s in enumerate(nodes):
        m = 0
        for e in s:
            m |= 1 << e
        mask[i] = m
    child: Dict[int, Tuple[int, int]] = {L + t: (a, b) for t, (a, b) in enumerate(pairs)}
    root = L + len(pairs) - 1 if pairs else 0
    nxt = len(nodes)

    def step_cost(v: int) -> float:
        a, b = child[v]
        c = 2.0 ** weight(mask[a] | mask[b])
        if alpha:
            c += alpha * (2.0 ** weight(mask[a]) + 2.0 ** weight(mask[b]) + 2.0 ** weight(mask[v]))
        return c

    def try_node(v: int) -> bool:
        nonlocal nxt
        frontier = list(child[v])
        inner = [v]
        while len(frontier) < size:
            cand = [f for f in frontier if f in child]
            if not cand:
                break
            f = max(cand, key=step_cost)
            frontier.remove(f)
            frontier.extend(child[f])
            inner.append(f)
        k = len(frontier)
        if k < 3:
            return False
        current = sum(step_cost(u) for u in inner)
        fm = [mask[f] for f in frontier]
        full = (1 << k) - 1
        union = [0] * (full + 1)
        for S in range(1, full + 1):
            low = S & -S
            union[S] = union[S ^ low] | fm[low.bit_length() - 1]
        out = [0] * (full + 1)
        for S in range(1, full + 1):
            out[S] = union[S] & (union[full ^ S] | mask[v])
        wout = [weight(out[S]) for S in range(full + 1)]
        # a merge's memory term: both operands read, the result written
        mem = [alpha * 2.0 ** x for x in wout] if alpha else None
        best = [0.0] * (full + 1)
        split = [0] * (full + 1)
        for S in range(1, full + 1):
            if S & (S - 1) == 0:
                continue
            if S != full and cap_log2 is not None and wout[S] > cap_log2 + 1e-9:
                best[S] = math.inf
                continue
            low = S & -S
            bc, bs = math.inf, 0
            sub = (S - 1) & S
            while sub:
                if sub & low:
                    rest = S ^ sub
                    c = best[sub] + best[rest]
                    if mem is not None:
                        c += mem[sub] + mem[rest] + mem[S]
                    if c < bc:
                        c += 2.0 ** weight(out[sub] | out[rest])
                        if c < bc:
                            bc, bs = c, sub
                sub = (sub - 1) & S
            best[S], split[S] = bc, bs
        if not best[full] < current * (1 - 1e-9):
            return False
        for u in inner[1:]:
            del child[u]

        def build(S: int) -> int:
            nonlocal nxt
            if S & (S - 1) == 0:
                return frontier[S.bit_length() - 1]
            a, b = build(split[S]), build(S ^ split[S])
            if S == full:
                child[v] = (a, b)
                return v
            u = nxt
            nxt += 1
            mask.append(out[S])
            child[u] = (a, b)
            return u

        build(full)
        return True

    for _ in range(sweeps):
        changed = False
        for v in sorted(child.keys()):
            if v in child and try_node(v):
                changed = True
        if not changed:
            break
    # back to SSA pairs, children before parents
    ssa: Dict[int, int] = {i: i for i in range(L)}
    out_pairs: List[Tuple[int, int]] = []
    stack = [(root, False)]
    while stack:
        v, done = stack.pop()
        if v < L:
            continue
        if done:
            a, b = child[v]
            ssa[v] = L + len(out_pairs)
            out_pairs.append((ssa[a], ssa[b]))
        else:
            stack.append((v, True))
            a, b = child[v]
            stack.append((b, False))
            stack.append((a, False))
    return out_pairs


def slice_count_and_reconfigure(leaves, pairs, lg, keep, n_edges: int, n_sliced: int, group: int = 2,
                                size: int = 8):
    """A fixed number of sliced bonds, chosen ``group`` at a time with the
    network reconfigured in between; no intermediate ever grows past the
    largest one of the tree so far.  Returns (pairs, sliced)."""
    mx, _, _ = tree_stats(leaves, pairs, lg, keep)
    pairs = reconfigure(leaves, pairs, lg, keep, cap_log2=mx, size=size)
    sl: List[int] = []
    while len(sl) < n_sliced:
        stripped = [frozenset(x - set(sl)) for x in leaves]
        sl += choose_slices(stripped, pairs, lg, keep, n_edges, n_sliced=min(group, n_sliced - len(sl)))
        stripped = [frozenset(x - set(sl)) for x in leaves]
        mx, _, _ = tree_stats(leaves, pairs, lg, keep, sl)
        pairs = reconfigure(stripped, pairs, lg, keep, cap_log2=mx, size=size)
    return pairs, sl


def refine_sliced(leaves, pairs, lg, keep, sliced, cap_log2: Optional[float] = None, rounds: int = 2,
                  size: int = 8):
    """Reconfigure a sliced tree on the network with its sliced bonds removed,
    then restore sliced bonds (last chosen first) while the largest
    intermediate still fits the cap -- restoring one never raises the total
    (per-slice cost at most doubles while the slice count halves).  Returns
    (pairs, sliced)."""
    sl = list(sliced)
    for _ in range(rounds):
        stripped = [frozenset(x - set(sl)) for x in leaves]
        pairs = reconfigure(stripped, pairs, lg, keep, cap_log2=cap_log2, size=size)
        for e in list(reversed(sl)):
            trial = [x for x in sl if x != e]
            mx, _, _ = tree_stats(leaves, pairs, lg, keep, trial)
            if cap_log2 is None or mx <= cap_log2 + 1e-9:
                sl = trial
    return pairs, sl


def slice_and_reconfigure(leaves, pairs, lg, keep, n_edges: int, cap_log2: float, group: int = 4,
                          size: int = 8, max_sliced: int = 62):
    """Slicing interleaved with reconfiguration: bonds are sliced ``group`` at a
    time (greedy, as ``choose_slices``) and the network without them is
    reconfigured after each group, until the largest intermediate fits the cap;
    then ``refine_sliced``.  Returns (pairs, sliced); ValueError once more than
    ``max_sliced`` bonds would be needed."""
    sl: List[int] = []
    pairs = reconfigure(leaves, pairs, lg, keep, size=size)
    while True:
        mx, _, _ = tree_stats(leaves, pairs, lg, keep, sl)
        if mx <= cap_log2 + 1e-9:
            break
        if len(sl) >= max_sliced:
            raise ValueError("no tree within the cap with at most max_sliced sliced bonds")
        stripped = [frozenset(x - set(sl)) for x in leaves]
        sl += choose_slices(stripped, pairs, lg, keep, n_edges, n_sliced=group)
        stripped = [frozenset(x - set(sl)) for x in leaves]
        # uncapped in between: a tree may grow before slicing takes it back
        # under the cap (capping it here was measured to give worse trees)
        pairs = reconfigure(stripped, pairs, lg, keep, size=size)
    return refine_sliced(leaves, pairs, lg, keep, sl, cap_log2=cap_log2, size=size)


# ------------------------------------------------------------ time objective


def batched_leaves(leaves, sliced, lg, keep, batch_log2: int):
    """The network as one batch of 2^batch_log2 slices runs it: sliced bonds
    removed, and a batch edge (id len(lg), an output edge) on every leaf that
    held a sliced bond, so that every slice-dependent tensor carries it and
    the rest do not.  Returns (leaves, lg, keep)."""
    sl = set(sliced)
    eb = len(lg)
    out = [frozenset(x - sl) | (frozenset((eb,)) if x & sl else frozenset()) for x in leaves]
    return out, list(lg) + [float(batch_log2)], frozenset(keep) | {eb}


def time_cost(leaves, pairs, lg, keep, sliced, batch_log2: int, alpha: float) -> float:
    """Estimated time of one batch of 2^batch_log2 slices, in multiply-adds:
    over every step, its multiply-adds plus alpha x the elements it reads and
    writes (both operands and the result), each at its batched size -- a step
    that depends on no sliced bond runs once per batch, unbatched."""
    bl, blg, bkeep = batched_leaves(leaves, sliced, lg, keep, batch_log2)
    nodes = replay(bl, pairs, bkeep)
    size = lambda s: 2.0 ** sum(blg[e] for e in s)  # noqa: E731
    total = 0.0
    for t, (i, j) in enumerate(pairs):
        c = nodes[len(leaves) + t]
        total += size(nodes[i] | nodes[j]) + alpha * (size(nodes[i]) + size(nodes[j]) + size(c))
    return total


def retime(leaves, pairs, lg, keep, sliced, batch_log2: int, alpha: float = ALPHA_TC, size: int = 10):
    """Subtree reconfiguration of a sliced tree for ``time_cost``: the batched
    network (``batched_leaves``) re-contracted with every step costing its
    multiply-adds plus alpha x the elements of its operands and result, no
    batched intermediate larger than the tree's largest.  On the GB300 the
    flop-minimal trees of shallow circuits are bound by HBM (their steps move
    many elements per multiply-add), so fewer bytes for more flops is faster.
    Returns the new SSA pairs."""
    bl, blg, bkeep = batched_leaves(leaves, sliced, lg, keep, batch_log2)
    nodes = replay(bl, pairs, bkeep)
    cap = max(sum(blg[e] for e in s) for s in nodes)
    return reconfigure(bl, pairs, blg, bkeep, cap_log2=cap, size=size, alpha=alpha)
