"""Subtree reconfiguration of contraction trees (host planner).  Pins: on tiny
networks the reconfigured tree reaches the optimum found by enumerating every
pairwise contraction order; on the 24-qubit circuit it never raises the cost,
keeps the output and the memory cap; slicing interleaved with reconfiguration
fits the cap with no more total work than plain greedy slicing."""
import itertools

import numpy as np
import pytest

import workloads as W
from paper_2406_18889_gb300 import network as N
from paper_2406_18889_gb300 import pathfind as P


def _random_network(n, n_bonds, n_open, seed):
    rng = np.random.default_rng(seed)
    tensors = [set() for _ in range(n)]
    e = 0
    for i in range(1, n):  # connected: a random spanning tree first
        j = int(rng.integers(0, i))
        tensors[i].add(e)
        tensors[j].add(e)
        e += 1
    for _ in range(n_bonds):
        i, j = rng.choice(n, size=2, replace=False)
        tensors[i].add(e)
        tensors[j].add(e)
        e += 1
    keep = set()
    for _ in range(n_open):
        i = int(rng.integers(0, n))
        tensors[i].add(e)
        keep.add(e)
        e += 1
    lg = [1.0] * e
    return [frozenset(t) for t in tensors], lg, frozenset(keep)


def _optimum(leaves, lg, keep):
    """Cheapest tree by trying every sequence of pairwise contractions."""
    best = [np.inf]

    def rec(alive, pairs):
        if len(alive) == 1:
            _, cost, _ = P.tree_stats(leaves, pairs, lg, keep)
            best[0] = min(best[0], cost)
            return
        k = len(leaves) + len(pairs)
        for a, b in itertools.combinations(alive, 2):
            rec([x for x in alive if x not in (a, b)] + [k], pairs + [(a, b)])

    rec(list(range(len(leaves))), [])
    return best[0]


@pytest.mark.parametrize("seed", range(6))
def test_reconfiguration_reaches_the_optimum_on_tiny_networks(seed):
    n = 5 + seed % 2
    leaves, lg, keep = _random_network(n, n_bonds=3, n_open=2, seed=seed)
    # a deliberately poor start: contract in index order
    pairs, cur = [], 0
    for i in range(1, n):
        pairs.append((cur, i))
        cur = n + len(pairs) - 1
    _, start, _ = P.tree_stats(leaves, pairs, lg, keep)
    new = P.reconfigure(leaves, pairs, lg, keep, size=8)
    _, cost, _ = P.tree_stats(leaves, new, lg, keep)
    opt = _optimum(leaves, lg, keep)
    assert cost == pytest.approx(opt, rel=1e-12) and cost <= start
    assert P.replay(leaves, new, keep)[-1] == P.replay(leaves, pairs, keep)[-1]


@pytest.fixture(scope="module")
def grid24():
    w = W.workload("grid4x6_d14")
    tn = N.circuit_network(w.circuit, w.open_qubits, w.closed_qubits, w.closed_bits)
    lg = P.log2dims(tn)
    return tn, lg, frozenset(tn.output_edges()), [frozenset(e) for e in tn.leaf_edges]


def test_reconfiguration_never_worse_and_keeps_cap(grid24):
    tn, lg, keep, leaves = grid24
    for pairs in (P.greedy(leaves, lg, keep, 1.0, 0.0, 7), P.partition_path(leaves, lg, keep, imbalance=0.4)):
        mx, cost, _ = P.tree_stats(leaves, pairs, lg, keep)
        new = P.reconfigure(leaves, pairs, lg, keep, cap_log2=mx)
        mx2, cost2, _ = P.tree_stats(leaves, new, lg, keep)
        assert cost2 <= cost and mx2 <= mx
        assert len(new) == len(pairs) and P.replay(leaves, new, keep)[-1] == P.replay(leaves, pairs, keep)[-1]


def test_slicing_with_reconfiguration_fits_the_cap(grid24):
    tn, lg, keep, leaves = grid24
    pairs = P.partition_path(leaves, lg, keep, imbalance=0.3)
    cap = 16.0
    sl = P.choose_slices(leaves, pairs, lg, keep, len(tn.edge_dim), 0, cap)
    _, cost, _ = P.tree_stats(leaves, pairs, lg, keep, sl)
    p2, sl2 = P.slice_and_reconfigure(leaves, pairs, lg, keep, len(tn.edge_dim), cap, group=2)
    mx2, cost2, _ = P.tree_stats(leaves, p2, lg, keep, sl2)
    assert mx2 <= cap
    assert cost2 * 2.0 ** len(sl2) <= cost * 2.0 ** len(sl)
    # plan_tree with refinement returns a tree at least as cheap as without
    t0 = P.plan_tree(tn, cap_log2=cap, method="partition")
    t1 = P.plan_tree(tn, cap_log2=cap, method="partition", refine=True)
    assert t1.log2_max_intermediate <= cap
    assert t1.cost_per_slice * 2.0 ** len(t1.sliced_edges) <= t0.cost_per_slice * 2.0 ** len(t0.sliced_edges)


def test_refined_plan_for_the_24_qubit_workload():
    # the same workload (6 sliced bonds, 64 slices): the refined search needs
    # less work per slice than the plain greedy tree, with no larger intermediate
    from paper_2406_18889_gb300 import engine as E
    w = W.workload("grid4x6_d14")
    plain = E.prepare(w, restarts=1).tree
    prep = E.prepare(w, restarts=1, refine=True)
    refined = prep.tree
    assert len(refined.sliced_edges) == len(plain.sliced_edges) == 6
    assert refined.cost_per_slice < plain.cost_per_slice
    assert refined.log2_max_intermediate <= plain.log2_max_intermediate
    # the library plans the refined tree (host-only planning: layouts,
    # tensor-core roles, memory map), with the planner's cost model
    from paper_2406_18889_gb300 import build as Bd
    Bd.build()
    from paper_2406_18889_gb300 import binding as B
    rank, edges, data = E.flatten_network(prep.tn)
    for prec in (0, 2):
        h = B.tn_plan_create(rank, edges, prep.tn.edge_dim, data, prep.tn.open_edges, prep.tn.block_edge,
                             np.asarray(prep.tree.pairs, dtype=np.int32).reshape(-1), prep.tree.sliced_edges,
                             prec, B.TN_FLAG_PLAN_ONLY | B.TN_FLAG_HOIST_INVARIANT, 64, 0, 0)
        q = B.tn_plan_query(h)
        B.tn_plan_destroy(h)
        assert q["useful_flops_per_slice"] == pytest.approx(8 * prep.tree.cost_per_slice, rel=1e-9)
