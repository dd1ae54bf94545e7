"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): each rank
samples its own blocks of the same circuit (independent problems), the job's
slices are summed over ranks and its time is the max over ranks."""
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
