"""Host-only checks of the C ABI: the library builds, loads and exports every
declared symbol; plan validation and host-side planning (no device work)."""
import re
from pathlib import Path

import numpy as np
import pytest

import workloads as W

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lib():
    from paper_2406_18889_gb300 import build as Bd
    Bd.build()
    from paper_2406_18889_gb300 import binding
    return binding


def test_exports_every_declared_symbol(lib):
    header = (ROOT / "include" / "tn.h").read_text()
    declared = set(re.findall(r"^(?:tn_status|const char\*)\s+(tn_\w+)\(", header, re.M))
    assert declared >= {"tn_plan_create", "tn_contract_slices", "tn_contract_slices_batched",
                        "tn_topk_postprocess", "tn_xeb"}
    L = lib.load()
    for name in declared:
        assert hasattr(L, name), name
    assert set(lib.EXPORTS) == declared
    # every entry point with arguments has its C types declared (64-bit sizes and
    # pointers would otherwise be passed as C ints)
    for name in declared - {"tn_last_error", "tn_version"}:
        assert getattr(L, name).argtypes is not None, name
    assert "sm_103a" in lib.tn_version()


def _flat(prep):
    from paper_2406_18889_gb300 import engine as E
    return E.flatten_network(prep.tn)


def _create(lib, prep, flags=None, **kw):
    rank, edges, data = _flat(prep)
    tn, tree = prep.tn, prep.tree
    args = dict(leaf_rank=rank, leaf_edges=edges, edge_dim=tn.edge_dim, leaf_data=data,
                open_edges=tn.open_edges, block_edge=tn.block_edge,
                pairs=np.asarray(tree.pairs).reshape(-1), sliced_edges=tree.sliced_edges,
                prec=0, flags=lib.TN_FLAG_PLAN_ONLY if flags is None else flags, max_slice_batch=8)
    args.update(kw)
    return lib.tn_plan_create(**args)


@pytest.fixture(scope="module")
def prep():
    from paper_2406_18889_gb300 import engine as E
    w = W.workload("grid3x4_d8", cycles=10, l=6, G=8)
    return E.prepare(w, n_sliced=3, restarts=1)


def test_plan_only_cost_model_matches_planner(lib, prep):
    h = _create(lib, prep)
    q = lib.tn_plan_query(h)
    # useful flops per slice = 8 x complex MACs of one sub-network (Table I convention)
    assert q["useful_flops_per_slice"] == pytest.approx(8 * prep.tree.cost_per_slice, rel=1e-12)
    assert q["workspace_bytes"] > 0 and q["workspace_bytes"] % 256 == 0
    st = lib.tn_plan_steps(h)
    assert len(st["m"]) == len(prep.tree.pairs)
    # every GEMM extent is a power of two and the variant steps are those above sliced leaves
    for key in ("batch", "m", "n", "k"):
        v = st[key]
        assert np.all(v >= 1) and np.all((v & (v - 1)) == 0)
    assert (st["kinds"] & 1).sum() >= 1
    lib.tn_plan_destroy(h)


def test_hoist_flag_marks_invariant_steps(lib, prep):
    h = _create(lib, prep, flags=lib.TN_FLAG_PLAN_ONLY | lib.TN_FLAG_HOIST_INVARIANT)
    k = lib.tn_plan_steps(h)["kinds"]
    assert np.all(((k & 4) > 0) == ((k & 1) == 0))
    lib.tn_plan_destroy(h)


@pytest.mark.parametrize("mutate,status", [
    ("bad_pair", 1), ("repeat_pair", 1), ("sliced_open", 1), ("sliced_twice", 1),
    ("batch_not_pow2", 1), ("short_tree", 1), ("unknown_precision", 1)])
def test_plan_validation(lib, prep, mutate, status):
    rank, edges, data = _flat(prep)
    tn, tree = prep.tn, prep.tree
    pairs = np.asarray(tree.pairs).reshape(-1).copy()
    kw = {}
    if mutate == "bad_pair":
        pairs[0] = len(rank) + 5
        kw["pairs"] = pairs
    elif mutate == "repeat_pair":
        pairs[2] = pairs[0]
        pairs[3] = pairs[1]
        kw["pairs"] = pairs
    elif mutate == "sliced_open":
        kw["sliced_edges"] = [tn.open_edges[0]]
    elif mutate == "sliced_twice":
        kw["sliced_edges"] = [tree.sliced_edges[0], tree.sliced_edges[0]]
    elif mutate == "batch_not_pow2":
        kw["max_slice_batch"] = 6
    elif mutate == "short_tree":
        kw["pairs"] = pairs[:-2]
    elif mutate == "unknown_precision":
        kw["prec"] = 7
    with pytest.raises(lib.TNError) as ei:
        _create(lib, prep, **kw)
    assert ei.value.status == status
    assert lib.tn_last_error()


def test_plan_only_rejects_contraction(lib, prep):
    h = _create(lib, prep)
    with pytest.raises(lib.TNError):
        lib.tn_contract_slices(h, [0], 1 << 20, 0, 1 << 20, 1 << 30, 0)
    lib.tn_plan_destroy(h)


def test_topk_argument_validation(lib):
    # rejected before any device work (so this runs without a GPU)
    with pytest.raises(lib.TNError):
        lib.tn_topk_postprocess(0, 4, 1024, 8, 1.0, 0, 0, np.arange(10), 0, 0)
    with pytest.raises(lib.TNError):
        lib.tn_topk_postprocess(16, 4, 1000, 8, 1.0, 0, 16, np.arange(10), 16, 16)  # B != 2^l
    with pytest.raises(lib.TNError):
        lib.tn_topk_postprocess(16, 4, 1024, 0, 1.0, 0, 16, np.arange(10), 16, 16)  # k = 0
    with pytest.raises(lib.TNError):
        lib.tn_topk_postprocess(16, 4, 1024, 513, 1.0, 0, 16, np.arange(10), 16, 16)  # per block: k <= 512
    with pytest.raises(lib.TNError):
        lib.tn_topk_postprocess(16, 1, 1 << 17, 8, 1.0, 0, 16, np.arange(17), 16, 16)  # per block: B <= 2^16
    with pytest.raises(lib.TNError):
        lib.tn_topk_postprocess(16, 4, 1024, 4097, 1.0, 1, 16, np.arange(10), 16, 16)  # global: k <= G*B
    with pytest.raises(lib.TNError):
        lib.tn_topk_postprocess(16, 1 << 20, 1 << 21, (1 << 26) + 1, 1.0, 1, 16, np.arange(21), 16, 16)  # k <= 2^26
    with pytest.raises(lib.TNError):
        lib.tn_topk_postprocess(16, 1 << 20, 1 << 21, 8, 1.0, 1, 16, np.arange(21), 16, 16)  # G*B <= 2^40
    with pytest.raises(lib.TNError):
        lib.tn_xeb(16, 0, 10)


@pytest.fixture(scope="module")
def bench_plan_steps(lib):
    # the 24-qubit workload's reduced-precision plan with invariant subtrees hoisted
    from paper_2406_18889_gb300 import engine as E
    w = W.workload("grid4x6_d14")
    prep = E.prepare(w)
    h = _create(lib, prep, flags=lib.TN_FLAG_PLAN_ONLY | lib.TN_FLAG_HOIST_INVARIANT, prec=2, max_slice_batch=64)
    st = lib.tn_plan_steps(h)
    lib.tn_plan_destroy(h)
    return prep, st


def test_fused_expansion_pairs(lib, bench_plan_steps):
    # every producer that writes an expanded operand (bit 5) is a per-batch CUDA-core
    # step with K <= 4 whose consumer is a tensor-core step marked as fed (bit 6)
    prep, st = bench_plan_steps
    k = st["kinds"]
    n_leaves = len(prep.tn.leaf_edges)
    pairs = np.asarray(prep.tree.pairs)
    consumer = {}
    for t, (a, b) in enumerate(pairs):
        consumer[a] = t
        consumer[b] = t
    producers = np.where(k & 32)[0]
    assert len(producers) >= 1
    for t in producers:
        assert not k[t] & 8 and not k[t] & 4 and st["k"][t] <= 4
        u = consumer[n_leaves + t]
        assert k[u] & 8 and k[u] & 64
    assert (k & 64 > 0).sum() == len(producers)


def test_fused_small_steps(lib, bench_plan_steps):
    # small steps (bit 7): per-batch, CUDA cores, K <= 4, <= 2^14 outputs, operands
    # from leaves, hoisted results or other small steps
    prep, st = bench_plan_steps
    k = st["kinds"]
    n_leaves = len(prep.tn.leaf_edges)
    pairs = np.asarray(prep.tree.pairs)
    micro = np.where(k & 128)[0]
    assert len(micro) >= 1
    for t in micro:
        assert not k[t] & 4 and not k[t] & 8 and not k[t] & 32
        assert st["k"][t] <= 4 and st["batch"][t] * st["m"][t] * st["n"][t] <= 1 << 14
        for x in pairs[t]:
            if x >= n_leaves:
                q = x - n_leaves
                assert k[q] & 4 or k[q] & 128


def test_tensor_core_steps_carry_the_flops(lib, bench_plan_steps):
    prep, st = bench_plan_steps
    k = st["kinds"]
    cost = st["batch"] * st["m"] * st["n"] * st["k"]
    per_batch = (k & 4) == 0
    tc = (k & 8) > 0
    assert cost[per_batch & tc].sum() >= 0.99 * cost[per_batch].sum()


@pytest.mark.parametrize("what,status", [("alloc", 2), ("invalid_plan", 1)])
def test_injected_plan_faults(lib, prep, monkeypatch, what, status):
    # host-side fault injection fails the call before any device work
    monkeypatch.setenv("TN_FAULT", what)
    with pytest.raises(lib.TNError) as ei:
        _create(lib, prep)
    assert ei.value.status == status
    assert "TN_FAULT" in lib.tn_last_error()
    monkeypatch.delenv("TN_FAULT")
    lib.tn_plan_destroy(_create(lib, prep))


def test_tuning_forms_validated_before_any_change(lib):
    # per-step launch forms of the tensor-core steps (no device work: plan-only)
    from paper_2406_18889_gb300 import engine as E
    w = W.workload("grid4x6_d14")
    prep = E.prepare(w)
    h = _create(lib, prep, flags=lib.TN_FLAG_PLAN_ONLY | lib.TN_FLAG_HOIST_INVARIANT, prec=2, max_slice_batch=64)
    try:
        k = lib.tn_plan_steps(h)["kinds"]
        tuned = np.where(((k & 8) > 0) & ((k & 4) == 0))[0]
        other = np.where((k & 8) == 0)[0]
        assert len(tuned) >= 1 and len(other) >= 1
        zeros = np.zeros((len(k), 2), np.int32)
        lib.tn_plan_set_tuning(h, zeros)  # every step at its default form
        candidates = [(256, 1), (256, 2), (128, 1), (64, 1), (32, 1)]
        for t in tuned:
            accepted = []
            for f in candidates:
                forms = zeros.copy()
                forms[t] = f
                try:
                    lib.tn_plan_set_tuning(h, forms)
                    accepted.append(f)
                except lib.TNError as e:
                    assert e.status == 1
            # the widest tile for N and half of it at least; 256-row tiles only at width 256
            assert len(accepted) >= 2
            if (256, 2) in accepted:
                assert (256, 1) in accepted
        for bad_step, bad in ((tuned[0], (999, 1)), (tuned[0], (256, 3)), (other[0], (256, 1))):
            forms = zeros.copy()
            forms[bad_step] = bad
            with pytest.raises(lib.TNError) as ei:
                lib.tn_plan_set_tuning(h, forms)
            assert ei.value.status == 1
        with pytest.raises(lib.TNError):
            lib.tn_plan_set_tuning(h, zeros[:-1])  # step count differs
        with pytest.raises(lib.TNError):  # timing needs a device plan
            lib.tn_plan_autotune(h, [0], 1 << 20, 1 << 20, 1 << 30, 0, 1)
    finally:
        lib.tn_plan_destroy(h)


def test_slice_batch_chosen_from_memory_cap(lib):
    # max_slice_batch = 0: the largest power of two whose memory fits the cap
    from paper_2406_18889_gb300 import engine as E
    w = W.workload("grid4x6_d14")
    prep = E.prepare(w)
    need = {}
    for b in (1, 2, 4, 8, 16, 32, 64):
        h = _create(lib, prep, prec=2, flags=lib.TN_FLAG_PLAN_ONLY | lib.TN_FLAG_HOIST_INVARIANT, max_slice_batch=b)
        need[b] = lib.tn_plan_query(h)["workspace_bytes"]
        lib.tn_plan_destroy(h)
    assert all(need[b] <= need[2 * b] for b in (1, 2, 4, 8, 16, 32))
    for cap, lo, hi in ((need[64] * 4, 64, 64), (need[16] * 1.02 + (1 << 30), 4, 16)):
        h = _create(lib, prep, prec=2, flags=lib.TN_FLAG_PLAN_ONLY | lib.TN_FLAG_HOIST_INVARIANT,
                    max_slice_batch=0, mem_cap_bytes=int(cap))
        b = lib.tn_plan_slice_batch(h)
        assert lo <= b <= hi and (b & (b - 1)) == 0, (cap, b)
        assert lib.tn_plan_query(h)["workspace_bytes"] <= cap
        lib.tn_plan_destroy(h)
    # nothing fits: batch 1, rejected by the cap
    with pytest.raises(lib.TNError) as ei:
        _create(lib, prep, prec=2, flags=lib.TN_FLAG_PLAN_ONLY, max_slice_batch=0, mem_cap_bytes=1)
    assert ei.value.status == 2
    # never more than the number of slices (2^6)
    h = _create(lib, prep, prec=0, flags=lib.TN_FLAG_PLAN_ONLY, max_slice_batch=0, mem_cap_bytes=1 << 50)
    assert lib.tn_plan_slice_batch(h) == 64
    lib.tn_plan_destroy(h)
    # a plan-only plan has no device to ask for free memory
    with pytest.raises(lib.TNError) as ei:
        _create(lib, prep, prec=0, flags=lib.TN_FLAG_PLAN_ONLY, max_slice_batch=0)
    assert ei.value.status == 1


def test_hilo_steps_mask_places_split_products(lib):
    from paper_2406_18889_gb300 import engine as E
    w = W.workload("grid4x6_d14")
    prep = E.prepare(w)
    flags = lib.TN_FLAG_PLAN_ONLY | lib.TN_FLAG_HOIST_INVARIANT
    h = _create(lib, prep, prec=1, flags=flags, max_slice_batch=64)
    k0 = lib.tn_plan_steps(h)["kinds"]
    ws0 = lib.tn_plan_query(h)["workspace_bytes"]
    lib.tn_plan_destroy(h)
    tc = np.where((k0 & 8) > 0)[0]
    assert len(tc) >= 2 and not ((k0 & 16) > 0).any()
    mask = np.zeros(len(k0), np.uint8)
    mask[tc[::2]] = 1
    mask[np.where((k0 & 8) == 0)[0][:3]] = 1  # ignored on CUDA-core steps
    h = _create(lib, prep, prec=1, flags=flags, max_slice_batch=64, hilo_steps=mask)
    k = lib.tn_plan_steps(h)["kinds"]
    assert np.array_equal((k & 8) > 0, (k0 & 8) > 0)
    # the requested steps split, with the tensor-core steps linked to them
    # through a stored 16-bit operand; only tensor-core steps split
    split = np.where((k & 16) > 0)[0]
    assert set(tc[::2]) <= set(split) <= set(tc)
    assert lib.tn_plan_query(h)["workspace_bytes"] >= ws0
    p = lib.tn_plan_precision(h)
    assert p["n_tc_steps"] == len(tc) and p["n_hilo_steps"] == len(split) and p["rel_l2_chosen"] == -1
    lib.tn_plan_destroy(h)
    # the placement is closed: asking for it again gives the same steps
    again = np.zeros(len(k0), np.uint8)
    again[split] = 1
    h = _create(lib, prep, prec=1, flags=flags, max_slice_batch=64, hilo_steps=again)
    assert np.array_equal(np.where((lib.tn_plan_steps(h)["kinds"] & 16) > 0)[0], split)
    lib.tn_plan_destroy(h)
    # the mask does not combine with the global flags; entries are 0 or 1
    for bad in (dict(flags=flags | lib.TN_FLAG_HILO, hilo_steps=mask),
                dict(flags=flags | lib.TN_FLAG_HILO_AUTO, hilo_steps=mask),
                dict(flags=flags | lib.TN_FLAG_HILO_AUTO | lib.TN_FLAG_HILO),
                dict(flags=flags, hilo_steps=mask * 2),
                dict(flags=flags | lib.TN_FLAG_HILO_AUTO, hilo_tol=1.5)):
        with pytest.raises(lib.TNError) as ei:
            _create(lib, prep, prec=1, max_slice_batch=64, **bad)
        assert ei.value.status == 1
    # automatic placement on a plan-only plan: nothing is measured, nothing split
    h = _create(lib, prep, prec=1, flags=flags | lib.TN_FLAG_HILO_AUTO, max_slice_batch=64)
    assert not ((lib.tn_plan_steps(h)["kinds"] & 16) > 0).any()
    lib.tn_plan_destroy(h)


@pytest.mark.parametrize("seed", range(6))
def test_plan_only_graphs_over_random_trees(lib, seed):
    # plans over random (noisy greedy) trees and slicings of small circuits, in
    # every precision, hoisted or not, at several batches: the workspace map in
    # its two arenas and the concurrent batch graph are built, and the graph's
    # self-check (launches that share workspace are ordered) holds for each
    from paper_2406_18889_gb300 import engine as E
    from paper_2406_18889_gb300 import network as N
    from paper_2406_18889_gb300 import pathfind as P
    rng = np.random.default_rng(seed)
    w = W.workload("grid3x4_d8", cycles=int(rng.integers(6, 11)), l=int(rng.integers(3, 8)),
                   G=int(2 ** rng.integers(0, 4)))
    tn = N.circuit_network(w.circuit, w.open_qubits, w.closed_qubits, w.closed_bits)
    lg = P.log2dims(tn)
    keep = frozenset(tn.output_edges())
    leaves = [frozenset(e) for e in tn.leaf_edges]
    pairs = P.greedy(leaves, lg, keep, float(rng.uniform(0.5, 2.5)), float(rng.uniform(0, 0.6)), seed)
    n_sl = int(rng.integers(0, 5))
    sl = P.choose_slices(leaves, pairs, lg, keep, len(tn.edge_dim), n_sliced=n_sl) if n_sl else []
    pairs = P.invariant_first(leaves, pairs, sl)
    mx, cost, vcost = P.tree_stats(leaves, pairs, lg, keep, sl)
    tree = P.Tree(pairs=pairs, sliced_edges=list(sl), log2_max_intermediate=mx, cost_per_slice=cost,
                  cost_variant_per_slice=vcost, n_leaves=len(leaves))
    prep = E.Prepared(tn, tree)
    for prec in (0, 1, 2):
        for hoist in (0, lib.TN_FLAG_HOIST_INVARIANT):
            for batch in (1, 4, 64):
                h = _create(lib, prep, prec=prec, flags=lib.TN_FLAG_PLAN_ONLY | hoist, max_slice_batch=batch)
                assert lib.tn_plan_query(h)["workspace_bytes"] > 0
                lib.tn_plan_destroy(h)
