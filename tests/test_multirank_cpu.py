"""Multi-rank host logic on CPU (gloo): bench.py's rank bookkeeping (each rank
samples its own blocks of the same circuit, the job's slices are summed over
ranks and its time is the max over ranks), and the slices of one problem split
over ranks with their FP64 partials gathered on rank 0 and summed in rank
order (multirank.py), against the single-rank sum."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    w_env = bench.dist_env()
    d = bench.init_dist(world, "gloo")
    w = bench.rank_workload(rank)
    t = bench.max_over_ranks(1.0 + rank, d)
    n = bench.sum_over_ranks(64.0, d)
    q.put((rank, w_env, w.closed_bits.tobytes(), w.circuit.ops[0].name, t, n))
    dist.destroy_process_group()


def test_two_gloo_ranks_partition_blocks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, e0, b0, g0, t0, n0), (r1, e1, b1, g1, t1, n1) = res
    assert e0 == (2, 0, 0) and e1 == (2, 1, 1)
    assert b0 != b1          # different closed bitstrings: independent problems
    assert g0 == g1          # same circuit
    assert t0 == t1 == 2.0   # max over ranks
    assert n0 == n1 == 128.0  # slices summed over ranks


def _slice_worker(rank, world, port, q):
    # the slices split over ranks (each rank contracts its share with the FP64
    # oracle in place of the GPU), partials gathered on rank 0 in rank order
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import numpy as np
    import workloads as W
    from oracle import einsum_tn as et
    from paper_2406_18889_gb300 import multirank as MR
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = W.workload("grid3x4_d8", cycles=10, l=6, G=8)
    wires = [(q, 1) for q in range(5)]
    ids = W.draw_slice_subset(32, 13, seed=3)
    net = et.build_network(w.circuit, w.open_qubits, w.closed_qubits, w.closed_bits)
    mine = MR.partition(ids, rank, world)
    local = et.contract(net, wires, mine) if len(mine) else np.zeros((w.G, 1 << w.l), complex)
    parts = MR.gather_partials(torch.as_tensor(local), dist, world, rank)
    q.put((rank, mine.tolist(), None if parts is None else parts.numpy()))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slices_split_over_gloo_ranks_sum_to_the_single_rank_result(world):
    import numpy as np
    import workloads as W
    from oracle import einsum_tn as et
    from oracle import postprocess as pp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slice_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ids = W.draw_slice_subset(32, 13, seed=3)
    # the shares partition the ids, in order
    assert sum((r[1] for r in res), []) == ids.tolist()
    assert max(len(r[1]) for r in res) - min(len(r[1]) for r in res) <= 1
    parts = res[0][2]
    assert parts.shape[0] == world and all(r[2] is None for r in res[1:])
    total = parts[0].copy()
    for p in parts[1:]:
        total = total + p  # rank order: what tn_sum_partials computes on the device
    w = W.workload("grid3x4_d8", cycles=10, l=6, G=8)
    net = et.build_network(w.circuit, w.open_qubits, w.closed_qubits, w.closed_bits)
    single = et.contract(net, [(q, 1) for q in range(5)], ids)
    assert pp.relative_l2(total, single) <= 1e-13
    a = pp.topk_blocks(total, 8, 32 / 13, w.block_base(), w.open_bit_pos())
    b = pp.topk_blocks(single, 8, 32 / 13, w.block_base(), w.open_bit_pos())
    assert np.array_equal(a[0], b[0])


def test_partition_shares():
    import numpy as np
    from paper_2406_18889_gb300 import multirank as MR
    ids = np.arange(10, 74)
    for world in (1, 2, 3, 8, 100):
        shares = [MR.partition(ids, r, world) for r in range(world)]
        assert np.array_equal(np.concatenate(shares), ids)
        assert max(map(len, shares)) - min(map(len, shares)) <= 1
    with pytest.raises(ValueError):
        MR.partition(ids, 2, 2)


def test_clock_samples_filtered_to_timed_regions():
    """bench.py's clock record keeps only nvidia-smi samples whose timestamps fall
    inside the marked timed regions; reasons are collected from those alone."""
    import datetime
    import bench
    c = bench.ClockSampler(0)
    base = datetime.datetime(2026, 1, 2, 3, 4, 5)

    def line(dt_ms, mhz, thermal):
        stamp = (base + datetime.timedelta(milliseconds=dt_ms)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return (f"{stamp}, {mhz}, 2070, 900.0, 0x0, Not Active, Not Active, "
                f"{'Active' if thermal else 'Not Active'}, Not Active")

    c.out = "\n".join([line(0, 1000, True), line(100, 2070, False), line(150, 2055, False),
                       line(400, 900, True)])
    t0 = base.timestamp()
    c.timed(t0 + 0.05, t0 + 0.2)
    s = c.summary()
    assert s["samples"] == 2 and s["sm_mhz"] == (2070 + 2055) / 2 and s["reasons"] == []
    c.timed(t0 + 0.39, t0 + 0.41)
    s = c.summary()
    assert s["samples"] == 3 and s["reasons"] == ["sw_thermal_slowdown"]
    # no sample inside: the first ones after the region's start, and it says so
    c.windows = [(t0 + 0.16, t0 + 0.17)]
    s = c.summary()
    assert s["samples"] == 1 and s["sm_mhz"] == 900 and "no sample" in s["note"]


def test_bench_slice_batch_per_rank_share():
    # with the slices split over N ranks each rank runs its share as one batch
    # (the power of two that holds it); with blocks split, the full batch
    import argparse
    import bench
    args = argparse.Namespace(batch=64, partition="slices", prec="fp16", hilo=False, hoist=False,
                              autotune=False, serial_graph=False, path="time")
    got = {n: bench.bench_config(args, n)["slice_batch"] for n in (1, 2, 3, 4, 8)}
    assert got == {1: 64, 2: 32, 3: 32, 4: 16, 8: 8}
    args.partition = "blocks"
    assert bench.bench_config(args, 8)["slice_batch"] == 64
    assert bench.bench_config(args, 8)["parallelism"].startswith("8 independent block sets")
