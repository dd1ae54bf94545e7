"""The planner's time objective (host side): multiply-adds plus alpha x the
elements every step reads and writes, with the slice batch as an edge of the
slice-dependent tensors.

Pins: the cost of two hand-worked three-tensor chains (with and without a
sliced bond); on tiny networks, reconfiguration under this cost reaches the
optimum found by enumerating every pairwise order; on the 24-qubit circuit,
re-optimising a sliced tree never raises its time cost, keeps the output and
keeps every batched intermediate within the tree's largest; the time
objective's choice never costs more time than the flop objective's; the
slice-independent-first order keeps the tree."""
import itertools
import os

import numpy as np
import pytest

import workloads as W
from paper_2406_18889_gb300 import network as N
from paper_2406_18889_gb300 import pathfind as P

from test_planner_reconfigure import _random_network


def test_time_cost_of_a_chain_by_hand():
    # A{a,b} B{b,c} C{c,d}, log2 dims a=1 b=2 c=1 d=1, output {a,d}; tree ((A,B),C)
    a, b, c, d = 0, 1, 2, 3
    lg = [1.0, 2.0, 1.0, 1.0]
    leaves = [frozenset({a, b}), frozenset({b, c}), frozenset({c, d})]
    keep = frozenset({a, d})
    pairs = [(0, 1), (3, 2)]
    # step 1: {a,b,c} = 16 MACs, reads 8 + 8, writes {a,c} = 4
    # step 2: {a,c,d} = 8 MACs, reads 4 + 4, writes {a,d} = 4
    assert P.time_cost(leaves, pairs, lg, keep, [], 0, 10.0) == 16 + 10 * 20 + 8 + 10 * 12
    # slicing c (batch of both its values): B{b,e} and C{d,e} carry the batch edge e
    # step 1: {a,b,e} = 16 MACs, reads A 8 + B 8, writes {a,e} = 4
    # step 2: {a,d,e} = 8 MACs, reads 4 + 4, writes {a,d,e} = 8
    assert P.time_cost(leaves, pairs, lg, keep, [c], 1, 10.0) == 16 + 10 * 20 + 8 + 10 * 16
    # alpha = 0: the multiply-adds of one batch
    assert P.time_cost(leaves, pairs, lg, keep, [], 0, 0.0) == 24


def test_batched_leaves_mark_the_slice_dependent_tensors():
    leaves = [frozenset({0, 1}), frozenset({1, 2}), frozenset({2, 3})]
    bl, blg, bkeep = P.batched_leaves(leaves, [2], [1.0] * 4, frozenset({0, 3}), 5)
    assert bl == [frozenset({0, 1}), frozenset({1, 4}), frozenset({3, 4})]
    assert blg[4] == 5.0 and 4 in bkeep and {0, 3} <= bkeep


def _optimum_time(leaves, lg, keep, alpha):
    best = [np.inf]

    def rec(alive, pairs):
        if len(alive) == 1:
            best[0] = min(best[0], P.time_cost(leaves, pairs, lg, keep, [], 0, alpha))
            return
        k = len(leaves) + len(pairs)
        for x, y in itertools.combinations(alive, 2):
            rec([z for z in alive if z not in (x, y)] + [k], pairs + [(x, y)])

    rec(list(range(len(leaves))), [])
    return best[0]


@pytest.mark.parametrize("seed,alpha", [(0, 1.0), (1, 4.0), (2, 16.0), (3, 145.0), (4, 4.0), (5, 64.0)])
def test_time_reconfiguration_reaches_the_optimum_on_tiny_networks(seed, alpha):
    n = 5 + seed % 2
    leaves, lg, keep = _random_network(n, n_bonds=3, n_open=2, seed=100 + seed)
    pairs, cur = [], 0
    for i in range(1, n):
        pairs.append((cur, i))
        cur = n + len(pairs) - 1
    start = P.time_cost(leaves, pairs, lg, keep, [], 0, alpha)
    new = P.reconfigure(leaves, pairs, lg, keep, size=8, alpha=alpha)
    got = P.time_cost(leaves, new, lg, keep, [], 0, alpha)
    assert got == pytest.approx(_optimum_time(leaves, lg, keep, alpha), rel=1e-12) and got <= start
    assert P.replay(leaves, new, keep)[-1] == P.replay(leaves, pairs, keep)[-1]


def test_retime_on_the_24_qubit_tree_never_worse():
    w = W.workload("grid4x6_d14")
    tn = N.circuit_network(w.circuit, w.open_qubits, w.closed_qubits, w.closed_bits)
    lg = P.log2dims(tn)
    keep = frozenset(tn.output_edges())
    leaves = [frozenset(e) for e in tn.leaf_edges]
    pairs = P.greedy(leaves, lg, keep, 1.0, 0.0, 7)
    sl = P.choose_slices(leaves, pairs, lg, keep, len(tn.edge_dim), n_sliced=6)
    before = P.time_cost(leaves, pairs, lg, keep, sl, 6, P.ALPHA_TC)
    new = P.retime(leaves, pairs, lg, keep, sl, 6, size=8)
    after = P.time_cost(leaves, new, lg, keep, sl, 6, P.ALPHA_TC)
    assert after <= before
    assert len(new) == len(pairs)
    # the same output; no batched intermediate above the tree's largest
    bl, blg, bkeep = P.batched_leaves(leaves, sl, lg, keep, 6)
    old_nodes, new_nodes = P.replay(bl, pairs, bkeep), P.replay(bl, new, bkeep)
    assert new_nodes[-1] == old_nodes[-1]
    size = lambda s: sum(blg[e] for e in s)  # noqa: E731
    assert max(map(size, new_nodes)) <= max(map(size, old_nodes)) + 1e-9
    # a full binary tree over the leaves: every node consumed exactly once
    used = [x for p in new for x in p]
    assert sorted(used) == list(range(len(leaves) + len(new) - 1))


def test_invariant_first_keeps_the_tree():
    # A{0,1} B{1,2} C{2,3} D{3,4}, output {0,4}, bond 3 sliced: C and D depend
    # on the slice.  Pairs ((C,D),(A,B)) list the slice-dependent step first.
    leaves = [frozenset({0, 1}), frozenset({1, 2}), frozenset({2, 3}), frozenset({3, 4})]
    keep = frozenset({0, 4})
    pairs = [(2, 3), (0, 1), (4, 5)]
    out = P.invariant_first(leaves, pairs, [3])
    assert out == [(0, 1), (2, 3), (5, 4)]
    stripped = [x - {3} for x in leaves]
    assert P.replay(stripped, out, keep)[-1] == P.replay(stripped, pairs, keep)[-1] == keep
    # already in that order: unchanged
    assert P.invariant_first(leaves, out, [3]) == out


def test_plan_tree_lists_slice_independent_steps_first():
    w = W.workload("grid4x6_d14")
    tn = N.circuit_network(w.circuit, w.open_qubits, w.closed_qubits, w.closed_bits)
    tree = P.plan_tree(tn, n_sliced=6, restarts=1)
    sl = set(tree.sliced_edges)
    variant = [bool(set(e) & sl) for e in tn.leaf_edges]
    for (i, j) in tree.pairs:
        variant.append(variant[i] or variant[j])
    v = variant[len(tn.leaf_edges):]
    assert v == sorted(v) and not v[0] and v[-1]


def test_time_objective_never_worse_than_the_flop_tree():
    # the time objective keeps the candidate with the lowest time_cost, and the
    # flop-refined trees are among its candidates: its choice costs no more
    # time (and, hoisting nothing, the flop choice no fewer multiply-adds)
    # (the 24-qubit grid at 10 cycles, 4 sliced bonds: a few seconds of planning)
    w = W.workload("grid4x6_d14", cycles=10, n_sliced=4)
    tn = N.circuit_network(w.circuit, w.open_qubits, w.closed_qubits, w.closed_bits)
    lg = P.log2dims(tn)
    keep = frozenset(tn.output_edges())
    leaves = [frozenset(e) for e in tn.leaf_edges]
    kw = dict(n_sliced=4, restarts=1, method="greedy", refine=True, workers=os.cpu_count() or 1)
    flop = P.plan_tree(tn, **kw)
    fast = P.plan_tree(tn, objective="time", batch_log2=4, **kw)
    t_flop = P.time_cost(leaves, flop.pairs, lg, keep, flop.sliced_edges, 4, P.ALPHA_TC)
    t_fast = P.time_cost(leaves, fast.pairs, lg, keep, fast.sliced_edges, 4, P.ALPHA_TC)
    assert t_fast <= t_flop
    assert len(fast.sliced_edges) == 4
    # both trees contract the whole network to the same output
    for t in (flop, fast):
        stripped = [x - set(t.sliced_edges) for x in leaves]
        assert P.replay(stripped, t.pairs, keep)[-1] == keep
