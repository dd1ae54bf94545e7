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
