#!/usr/bin/env python
"""Benchmark: sliced tensor-network contraction of a random circuit on GB300.

Workload (one "step" = one pass of the whole hot path over one batch):
  24-qubit 4x6 grid random circuit, 14 cycles (sqrt X/Y/W + fSim, ABCDCDAB),
  6 sliced bonds (64 sub-networks), 10 open qubits (1024 amplitudes per block),
  64 blocks of closed bitstrings; a step contracts all 64 slices with an FP64
  cross-slice sum, keeps the top 64 strings per block and scores them by XEB.
  Subtrees that depend on no sliced bond are contracted once per step and
  shared by its 64 slices (--hoist: once per plan instead).

Metric: slices/s (whole job, all ranks) and the executed complex TFLOP/s
(8 real flops per complex multiply-add the step's kernels perform).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec c64] [--impl reference]

N > 1 runs one process per GPU (torchrun).  --partition slices (default):
the 64 slices of the one problem are split over the ranks and their FP64
partial sums added on rank 0 (strong scaling).  --partition blocks: each rank
samples its own 64 blocks of the same circuit (independent problems, no
collective on the data path), the job's value the sum over ranks (weak
scaling).  Time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

if "--impl" in sys.argv and "reference" in sys.argv:
    # the CPU reference arm runs on rank 0 alone, on every host core: under
    # torchrun, whose default OMP_NUM_THREADS=1 would leave NumPy's BLAS one
    # thread, give the threads back before NumPy loads its BLAS
    _cores = str(len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1))
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = _cores

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "grid4x6_d14"
WORKLOAD_DESC = ("24-qubit 4x6 grid random circuit, 14 cycles, 6 sliced bonds (64 slices), "
                 "l=10 open qubits (1024 amplitudes/block), G=64 blocks, top-64 per block")
METRIC = "sliced-contraction slices/s (24-qubit 4x6 grid, 14 cycles, 64 slices) on 1 GB300"
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


def fp32_alu_peak_tflops(mhz: float = SM_MAX_MHZ) -> float:
    """FP32 FMA peak: 152 SMs x 128 lanes x 2 flop x clock."""
    return SM_COUNT * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


# ------------------------------------------------------------------ distributed
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_dist(world: int, backend: str):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend)
    return dist if world > 1 else None


def max_over_ranks(x: float, dist, device="cpu") -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, dist, device="cpu") -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def rank_workload(rank: int):
    """The circuit is shared; rank r draws its own blocks of closed bitstrings."""
    import workloads as W
    w = W.workload(WORKLOAD)
    if rank:
        w.closed_bits = W.draw_closed_bitstrings(len(w.closed_qubits), w.G,
                                                 seed=W.configs.SEED0 + 7919 * rank)
    return w


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons, every 50 ms, kept only
    where their timestamp falls inside a window marked with `timed()`."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        self.windows = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.5)  # let the sampler start before the first timed window
        except OSError:
            self.proc = None
        return self

    def timed(self, t0: float, t1: float):
        """Marks [t0, t1] (time.time() seconds) as a timed region."""
        self.windows.append((t0, t1))

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    @staticmethod
    def _epoch(stamp: str):
        import datetime
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.datetime.strptime(stamp, fmt).timestamp()
            except ValueError:
                continue
        return None

    def summary(self) -> dict:
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((self._epoch(parts[0]), float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        inside = [r for r in rows if r[0] is not None and any(a <= r[0] <= b for a, b in self.windows)]
        note = "samples inside the timed regions"
        if not inside:  # timed regions shorter than the sampling interval: nearest samples after the start
            t0 = min((a for a, _ in self.windows), default=None)
            after = [r for r in rows if r[0] is not None and t0 is not None and r[0] >= t0]
            inside = after[:2] or rows[-2:]
            note = "no sample inside the timed regions; the first samples after their start"
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, _, r in inside for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": float(np.median([r[1] for r in inside])), "sm_max_mhz": inside[0][2],
                "reasons": reasons, "samples": len(inside), "note": note}


# ------------------------------------------------------------------ oracle arm
def oracle_slices_per_s(w, wires, slice_ids) -> float:
    from oracle import einsum_tn as et
    net = et.build_network(w.circuit, w.open_qubits, w.closed_qubits, w.closed_bits)
    t0 = time.perf_counter()
    et.contract_each_slice(net, wires, slice_ids)
    return len(slice_ids) / (time.perf_counter() - t0)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def prepare_path(w, path: str, batch: int = 64):
    """The contraction tree of workload w for --path: "time" (greedy and
    bisection trees refined for the flop count, then re-optimised for the
    estimated time of one batch of ``batch`` slices: multiply-adds plus the
    elements each step moves), "refined" (the flop-refined trees alone) or
    "greedy"."""
    from paper_2406_18889_gb300 import engine as E
    if path == "greedy":
        return E.prepare(w)
    kw = {}
    if path == "time":
        kw = dict(objective="time", batch_log2=max(int(batch).bit_length() - 1, 0))
    return E.prepare(w, refine=True, method="both", workers=host_cores(), **kw)


PATH_DESC = {"time": "greedy and bisection + subtree reconfiguration, re-optimised for time per batch "
                     "(multiply-adds + 145 x elements moved)",
             "refined": "greedy and bisection + subtree reconfiguration (fewest multiply-adds)",
             "greedy": "greedy"}


def rank_batch(args, world: int, n_slices: int = 64) -> int:
    """A rank's slice batch: --batch, or, with the slices split over the
    ranks, the power of two that holds a rank's share (at most --batch)."""
    if not (world > 1 and args.partition == "slices"):
        return args.batch
    share, batch = -(-n_slices // world), 1
    while batch < share:
        batch *= 2
    return min(args.batch, batch)


def bench_config(args, world: int) -> dict:
    """The workload's config as both arms report it."""
    split_slices = world > 1 and args.partition == "slices"
    return {"workload": WORKLOAD_DESC, "slice_batch": rank_batch(args, world), "prec": args.prec, "hilo": args.hilo,
            "hoist_invariant": bool(args.hoist), "autotune": bool(args.autotune),
            "graph": "one chain" if args.serial_graph else "concurrent branches",
            "path": PATH_DESC[args.path],
            "l2": "flushed between steps (256 MiB write outside the timed events)",
            "parallelism": (f"the 64 slices split over {world} GPUs, FP64 partials gathered and summed "
                            "on rank 0" if split_slices else f"{world} independent block sets (one per GPU)")}


def oracle_wires(w):
    """Sliced bonds for the CPU oracle's samples: the greedy tree's six.  The
    oracle contracts every sub-network along its own greedy path; on the time
    tree's slicing that path is ~4x slower (47 s against 11 s per slice on 8
    host cores), which would make a bounded sample of 25 slices run for many
    minutes.  Each is one of 64 sub-networks of the same circuit."""
    from paper_2406_18889_gb300 import engine as E
    prep = E.prepare(w)
    return [prep.tn.wire_of_edge[e] for e in prep.tree.sliced_edges]


ORACLE_SAMPLE = ("1 slice of 64 per step (the greedy tree's six sliced bonds), oracle O2 (naive FP64 einsum "
                 "contractor along its own greedy path, numpy matmul)")


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    w = rank_workload(0)
    wires = oracle_wires(w)
    sample = ORACLE_SAMPLE
    for s in range(args.warmup):
        oracle_slices_per_s(w, wires, [s % 64])
    t0 = time.perf_counter()
    for s in range(args.steps):
        oracle_slices_per_s(w, wires, [(args.warmup + s) % 64])
    dt = time.perf_counter() - t0
    v = args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "slices/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "strong" if world > 1 and args.partition == "slices" else "weak",
            "vs_baseline": None, "dtype": "complex128",
            "data": "synthetic", "config": bench_config(args, world),
            "cpu_baseline": {"value": v, "unit": "slices/s", "cores": host_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "slices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ roofline
KIND_NAMES = {0: "gemm_cuda_core", 1: "bit_permute", 2: "gather", 3: "accumulate_fp64",
              4: "expand_operand", 5: "gemm_tensor_core"}


# DRAM bytes (read + write) of the tensor-core launches that can be a step's
# longest, per configuration (path, precision, slice batch, split products,
# hoisting) and the launch's algorithmic bytes, as one ncu capture of a step
# measured them (dram__bytes_read.sum + dram__bytes_write.sum; the tree as
# planned on the GB300 host).  The time tree's two longest launches take
# ~0.21 ms each, so either can be the longest in a run.  A configuration or
# launch without an entry, or whose kernels changed since, reports null.
DOMINANT_TRAFFIC = {
    ("time", "fp16", 64, False, False): {
        1141374976: 70072320 + 1009223936,    # tile width 256: reads 70 MB, writes 1009 MB
        1224736768: 1090625024 + 122336512,   # tile width 32: reads 1091 MB, writes 122 MB
    },
}


def fp32_peak_measured(B) -> tuple:
    """(TFLOP/s, source): the library's FP32 FMA microbenchmark on this GPU, else
    the derived 152 SMs x 128 lanes x 2 flop x clock."""
    try:
        return float(B.tn_selftest_fp32_peak()), "measured: FP32 FMA microbenchmark (tn_selftest_fp32_peak)"
    except Exception:
        return fp32_alu_peak_tflops(), "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"


def roofline_from_profile(prof, cfg_key=None, alu=None) -> tuple:
    """Per-launch rooflines of one profiled step (CUDA events around every launch).

    Each launch i has algorithmic FLOPs F_i and bytes B_i (operands and result
    once, at their storage size) and time t_i; its roofline time is
    max(F_i / P, B_i / BW), with P the tensor (or FP32 ALU) peak and BW the HBM
    peak.  Reported: the dominant launch (largest t_i) with its binding
    resource, the path's sum of roofline times over its summed time, and the
    per-class totals."""
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    tc_peak = float(peaks.get("bf16_tflops", 1900.0))
    alu_peak, alu_src = alu if alu is not None else (fp32_alu_peak_tflops(), "derived")
    src = "of measured" if peaks else "of fallback"
    kinds, ms, flops, nbytes = prof["kind"], prof["ms"], prof["flops"], prof["bytes"]
    per_kind = {}
    for k in np.unique(kinds):
        sel = kinds == k
        t = float(ms[sel].sum())
        entry = {"launches": int(sel.sum()), "ms": t}
        if k in (0, 5):
            entry["tflops"] = float(flops[sel].sum() / (t / 1e3) / 1e12) if t > 0 else None
        entry["gbs"] = float(nbytes[sel].sum() / (t / 1e3) / 1e9) if t > 0 else None
        per_kind[KIND_NAMES[int(k)]] = entry
    t_roof, t_all, launches = 0.0, 0.0, []
    for k, t, f, b in zip(kinds, ms, flops, nbytes):
        pk = tc_peak if k == 5 else alu_peak if k == 0 else None
        tf = f / (pk * 1e12) * 1e3 if pk else 0.0
        tb = b / (hbm * 1e9) * 1e3
        t_roof += max(tf, tb)
        t_all += float(t)
        if k == 5:
            launches.append({"ms": float(t), "tflops": float(f / (t / 1e3) / 1e12), "gbs": float(b / (t / 1e3) / 1e9),
                             "bound": "tensor" if tf >= tb else "hbm", "frac": float(max(tf, tb) / t)})
    i = int(np.argmax(ms))
    k, t, f, b = int(kinds[i]), float(ms[i]), float(flops[i]), float(nbytes[i])
    tf = f / (tc_peak * 1e12) * 1e3 if k == 5 else f / (alu_peak * 1e12) * 1e3 if k == 0 else 0.0
    tb = b / (hbm * 1e9) * 1e3
    if k == 5 and tf >= tb:
        r = {"bound": "tensor", "achieved": f / (t / 1e3) / 1e12, "peak": tc_peak, "unit": "TFLOP/s",
             "peak_source": f"bf16_tflops burst {src} (fp16 dense rate is the same)"}
    elif k == 0 and tf >= tb:
        r = {"bound": "alu", "achieved": f / (t / 1e3) / 1e12, "peak": alu_peak, "unit": "TFLOP/s",
             "peak_source": alu_src}
    else:
        r = {"bound": "hbm", "achieved": b / (t / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
             "peak_source": f"hbm_gbs {src}"}
    r["frac"] = r["achieved"] / r["peak"]
    r["traffic"] = DOMINANT_TRAFFIC.get(cfg_key, {}).get(int(round(b))) if k == 5 else None
    if r["traffic"] is None:
        r["traffic_note"] = "no ncu DRAM capture of this configuration's longest launch with the current kernels"
    r["kernel"] = f"{KIND_NAMES[k]}: the step's longest launch ({t:.3f} ms)"
    r["algorithmic"] = {"flops": f, "bytes": b}
    r["path"] = {"roofline_ms": t_roof, "ms": t_all, "frac": t_roof / t_all if t_all > 0 else None,
                 "note": "sum over launches of max(F/P, B/BW) over their summed event time"}
    r["tensor_core_launches"] = launches
    r["per_kind"] = per_kind
    return r, per_kind


def permute_bandwidth(B, torch, stream, bits: int = 28) -> dict:
    """HBM bandwidth of tn_permute on a 2^28-element complex64 tensor whose two
    14-bit halves swap places (a full transpose), events over 5 launches."""
    peaks = measured_peaks()
    x = torch.empty(1 << bits, dtype=torch.int64, device="cuda")
    y = torch.empty_like(x)
    half = bits // 2
    out_bit = [(i + half) % bits for i in range(bits)]
    B.tn_permute(x.data_ptr(), y.data_ptr(), out_bit, 8, stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(5):
        B.tn_permute(x.data_ptr(), y.data_ptr(), out_bit, 8, stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 5
    gbs = 2.0 * 8 * (1 << bits) / (ms / 1e3) / 1e9
    peak = float(peaks.get("hbm_gbs", 6800.0))
    del x, y
    return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "case": "2^28 complex64 elements, 14-bit halves swapped (read + write bytes)", "ms": ms}


# ------------------------------------------------------------------ GPU arm
def run_ours(args):
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_18889_gb300 import binding as B
    from paper_2406_18889_gb300 import engine as E

    # N > 1: the 64 slices of one problem split over the ranks, partials summed on
    # rank 0 (--partition slices), or every rank its own blocks (--partition blocks)
    split_slices = world > 1 and args.partition == "slices"
    w = rank_workload(0 if split_slices else rank)
    # slices split over the ranks: each rank's share runs as one batch (the
    # power of two that holds it), and the tree is searched for that batch
    batch = rank_batch(args, world, w.n_slices)
    prep = prepare_path(w, args.path, batch)
    hoist = (B.TN_FLAG_HOIST_INVARIANT if args.hoist else 0) | (B.TN_FLAG_SERIAL_GRAPH if args.serial_graph else 0)
    flags = (B.TN_FLAG_HILO if args.hilo else 0) | hoist
    plan = E.Plan(prep.tn, prep.tree, prec=args.prec, max_slice_batch=batch, flags=flags)
    S = plan.n_slices_total
    ids = np.arange(S, dtype=np.int64)
    if args.autotune:  # per-step tensor-core launch forms, timed before (outside) the measurement
        plan.autotune(ids, reps=3)
    if args.profile_region:
        # for ncu --profile-from-start off: three warm-up calls, then one call
        # (one slice batch) between cudaProfilerStart and cudaProfilerStop
        amps = torch.empty((plan.G, plan.J), dtype=torch.complex128, device="cuda")
        for _ in range(3):
            plan.contract(ids, out=amps)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
        plan.contract(ids, out=amps)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        if rank == 0:
            print(json.dumps({"profile_region": True, "sum_abs_amplitudes": float(amps.abs().sum())}), flush=True)
        plan.close()
        return
    base_np = w.block_base()
    pos = w.open_bit_pos()
    base = torch.as_tensor(base_np, device="cuda")
    amps = torch.empty((plan.G, plan.J), dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    info = plan.info
    useful_per_slice = info["useful_flops_per_slice"]

    from paper_2406_18889_gb300 import multirank as MR

    def step():
        if split_slices:
            if MR.contract_partitioned(plan, ids, dist, world, rank, out=amps) is None:
                return None
        else:
            plan.contract(ids, out=amps)
        idx, p = E.topk(amps, w.k, 1.0, base, pos)
        x = E.xeb(p, w.n_qubits)  # f = 1: the selected p are the strings' probabilities
        return idx, p, x

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clk = ClockSampler(local).__enter__()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall0, t_win = time.perf_counter(), time.time()
    for i in range(args.steps):
        flush.zero_()  # evict L2 (129 MB) between steps; not inside the timed events
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk.timed(t_win, time.time())
    if dist:
        dist.barrier()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    ms = max_over_ranks(ms, dist, "cuda")
    slices = float(S * args.steps) if split_slices else sum_over_ranks(float(S * args.steps), dist, "cuda")
    value = slices / (ms / 1e3)

    if args.only_timed:
        clk.__exit__()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "slices/s",
                              "ms_per_step": ms / args.steps, "only_timed": True}), flush=True)
        plan.close()
        return
    # e2e: same step through the C ABI with host buffers (pinned), copies inside the timing
    h_base = torch.as_tensor(base_np).pin_memory()
    h_idx = torch.empty((w.G, w.k), dtype=torch.int64).pin_memory()
    h_p = torch.empty((w.G, w.k), dtype=torch.float64).pin_memory()
    h_ids = torch.as_tensor(ids).pin_memory()
    d_base = torch.empty_like(base)

    def e2e_step():
        d_base.copy_(h_base, non_blocking=True)
        # slice ids travel host -> device inside the call
        if split_slices:
            if MR.contract_partitioned(plan, h_ids.numpy(), dist, world, rank, out=amps) is None:
                torch.cuda.synchronize()
                return None
        else:
            plan.contract(h_ids.numpy(), out=amps)
        idx, p = E.topk(amps, w.k, 1.0, d_base, pos)
        x = E.xeb(p, w.n_qubits)
        h_idx.copy_(idx, non_blocking=True)
        h_p.copy_(p, non_blocking=True)
        torch.cuda.synchronize()
        return x

    for _ in range(2):
        e2e_step()
    e2e_ms = 0.0
    for i in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t_win = time.time()
        e2e_step()
        e2e_ms += 1e3 * (time.perf_counter() - t0)
        clk.timed(t_win, time.time())
    clk.__exit__()
    e2e_ms = max_over_ranks(e2e_ms, dist, "cuda")

    e2e_value = slices / (e2e_ms / 1e3)
    h2d = h_base.numel() * 8 + S * 8
    d2h = (h_idx.numel() + h_p.numel()) * 8 + 8

    # per-kernel roofline: one profiled pass (events around every launch)
    # (this rank's own slices: all of them, or its share when slices are split)
    mine = MR.partition(ids, rank, world) if split_slices else ids
    prof = B.tn_contract_slices_profile(plan.handle, mine, amps.data_ptr(), 0, plan.workspace.data_ptr(),
                                        plan.workspace.numel(), stream.cuda_stream)
    alu = fp32_peak_measured(B)
    roofline, per_kind = roofline_from_profile(prof, (args.path, args.prec, batch, bool(args.hilo),
                                                      bool(args.hoist)), alu)
    executed_per_slice = float(prof["flops"].sum()) / max(len(mine), 1)
    permute = permute_bandwidth(B, torch, stream)
    # recorded kernels + slice-id uploads (one launch per 256 ids of each batch) + top-k + XEB
    n_batches = -(-len(mine) // batch)
    launches_per_step = prof["n_launches"] + n_batches * (-(-batch // 256)) + 2
    # complex64 accuracy on the tensor cores: fp16 hi + lo operands, K accumulated
    # one k tile at a time in FP32 (relative L2 8.7e-6 on this workload, the
    # complex64 path's 8.4e-6; tests/test_gpu_precision.py holds it to 1e-5)
    fine_value = None
    if args.prec != "c64" and not args.no_c64:
        planf = E.Plan(prep.tn, prep.tree, prec="fp16", max_slice_batch=batch,
                       flags=B.TN_FLAG_HILO | B.TN_FLAG_FINE_ACC | hoist)
        for _ in range(2):
            planf.contract(ids, out=amps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            planf.contract(ids, out=amps)
        e1.record(stream)
        torch.cuda.synchronize()
        fine_value = S * 3 / (e0.elapsed_time(e1) / 1e3)
        planf.close()
    # bf16 with split products on every tensor-core step, and only where the
    # calibration says their 16-bit error moves the amplitudes (TN_FLAG_HILO_AUTO, 3e-3)
    split = None
    if args.prec != "c64" and not args.no_c64:
        split = {"note": "bf16 tensor-core operands; hi + lo split products on every tensor-core step, or on "
                         "those TN_FLAG_HILO_AUTO picks for relative L2 <= 3e-3 on the calibration batch "
                         "(contraction only)"}
        for name, fl, kw in (("all_steps", B.TN_FLAG_HILO, {}), ("auto", B.TN_FLAG_HILO_AUTO, {"hilo_tol": 3e-3})):
            pl = E.Plan(prep.tn, prep.tree, prec="bf16", max_slice_batch=batch, flags=fl | hoist, **kw)
            for _ in range(2):
                pl.contract(ids, out=amps)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                pl.contract(ids, out=amps)
            e1.record(stream)
            torch.cuda.synchronize()
            pr = pl.precision()
            split[name] = {"value": S * 3 / (e0.elapsed_time(e1) / 1e3), "unit": "slices/s",
                           "n_tc_steps": pr["n_tc_steps"], "n_hilo_steps": pr["n_hilo_steps"]}
            if name == "auto":
                split[name].update({"calibration_rel_l2": pr["rel_l2_chosen"],
                                    "calibration_rel_l2_without_split": pr["rel_l2_none"]})
            pl.close()
    tuned = None
    if args.tune and args.prec != "c64":
        # operand type, slice batch, split placement and launch forms picked by timing under 3e-3
        tplan, rows = E.tune_plan(prep.tn, prep.tree, tol=3e-3, batches=(16, 32, 64), flags=hoist, reps=3)
        tplan.close()
        tuned = {"note": "engine.tune_plan: fp16 / bf16 x slice batch, split products placed by calibration "
                         "(TN_FLAG_HILO_AUTO, 3e-3), tensor-core launch forms tuned; the fastest within the bar "
                         "is chosen (contraction only)", "candidates": rows}
    c64_value = None
    if args.prec != "c64" and not args.no_c64:
        plan64 = E.Plan(prep.tn, prep.tree, prec="c64", max_slice_batch=batch, flags=hoist)
        for _ in range(3):
            plan64.contract(ids, out=amps)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            plan64.contract(ids, out=amps)
        e1.record(stream)
        torch.cuda.synchronize()
        c64_slices = 5.0 * S if split_slices else sum_over_ranks(5.0 * S, dist, "cuda")
        c64_value = c64_slices / (max_over_ranks(e0.elapsed_time(e1), dist, "cuda") / 1e3)
        plan64.close()
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        w0 = rank_workload(0)
        v = oracle_slices_per_s(w0, oracle_wires(w0), [0, 1])
        cpu = {"value": v, "unit": "slices/s", "cores": host_cores(), "kind": "oracle",
               "sample": ORACLE_SAMPLE.replace("1 slice of 64 per step", "2 of the 64 slices")}
    line = {
        "metric": METRIC, "value": value, "unit": "slices/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if split_slices else "weak", "vs_baseline": None,
        "dtype": "complex64" if args.prec == "c64" else
                 f"{args.prec} tensor-core operands, fp32 accumulate, complex64 elsewhere",
        "data": "synthetic",
        "config": bench_config(args, world),
        "useful_tflops": value * executed_per_slice / 1e12,
        "useful_flops_note": "flops the step's kernels execute (8 per complex multiply-add), per slice: "
                             "slice-independent subtrees run once per batch and are shared by its slices",
        "complex64_path": None if c64_value is None else {
            "value": c64_value, "unit": "slices/s", "speedup": value / c64_value,
            "useful_tflops": c64_value * executed_per_slice / 1e12, "fp32_peak_tflops": alu[0],
            "alu_frac": c64_value * executed_per_slice / 1e12 / alu[0], "fp32_peak_source": alu[1],
            "note": "same workload and batch through the complex64 CUDA-core path (contraction only)"},
        "complex64_accuracy_tensor_core_path": None if fine_value is None else {
            "value": fine_value, "unit": "slices/s",
            "vs_complex64_path": None if c64_value is None else fine_value / c64_value,
            "note": "fp16 hi+lo operands, K accumulated one k tile at a time in FP32 (TN_FLAG_HILO | "
                    "TN_FLAG_FINE_ACC): complex64 accuracy on the tensor cores (contraction only)"},
        "bf16_split_precision": split,
        "tuned": tuned,
        "useful_flops_per_slice": executed_per_slice,
        "subnetwork_flops": useful_per_slice,
        "subnetwork_flops_note": "8 x complex multiply-adds of one sub-network along the tree, every step "
                                 "counted (the paper's Table I convention)",
        "wall_s": wall,
        "roofline": roofline,
        "permute": permute,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "slices/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "clocks": clk.summary(),
        "gpu_launches": int(launches_per_step * args.steps),
    }
    print(json.dumps(line), flush=True)
    plan.close()


def run_uneven(args):
    """The 64 uneven circuits contracted in one tn_contract_slices_batched call
    (every slice of every circuit, FP64 sums per circuit), on one GPU.
    --path time plans the flop-refined trees here: the slice batch of each
    plan is the library's choice, not known when the tree is searched."""
    refined = args.path != "greedy"
    import torch
    import workloads as W
    from paper_2406_18889_gb300 import binding as B
    from paper_2406_18889_gb300 import engine as E
    torch.cuda.set_device(0)
    ws = W.configs.uneven_batch(64)
    t0 = time.perf_counter()
    preps = [E.prepare(w, restarts=1, refine=refined, method="both" if refined else "greedy",
                       workers=host_cores() if refined else 0) for w in ws]
    plan_s = time.perf_counter() - t0
    flags = ((B.TN_FLAG_HILO if args.hilo else 0) | (B.TN_FLAG_HILO_AUTO if args.hilo_auto else 0) |
             (B.TN_FLAG_HOIST_INVARIANT if args.hoist else 0))
    # each plan's slice batch chosen by the library from a 16 GiB budget (and its slice count)
    cap = 16 << 30
    plans = [E.Plan(p.tn, p.tree, prec=args.prec, flags=flags, own_workspace=False, max_slice_batch=0,
                    mem_cap_bytes=cap, hilo_tol=3e-3) for p in preps]
    outs = [torch.empty((w.G, 1 << w.l), dtype=torch.complex128, device="cuda") for w in ws]
    counts = [p.n_slices_total for p in plans]
    # the workspace for the most concurrent branches that fit in half the free memory
    free = torch.cuda.mem_get_info()[0]
    branches, wsz = 1, 0
    for k in range(8, 0, -1):
        wsz = B.tn_batched_workspace_bytes([p.handle for p in plans], counts, k)
        branches = k
        if wsz <= free // 2:
            break
    wsb = torch.empty(max(wsz, 256), dtype=torch.uint8, device="cuda")
    ids = [np.arange(p.n_slices_total, dtype=np.int64) for p in plans]
    slices = sum(len(x) for x in ids)
    flops = sum(p.info["useful_flops_per_slice"] * len(x) for p, x in zip(plans, ids))
    stream = torch.cuda.current_stream()

    def call():
        B.tn_contract_slices_batched([p.handle for p in plans], ids, [o.data_ptr() for o in outs], 0,
                                     wsb.data_ptr(), wsz, stream.cuda_stream)

    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({
        "metric": "uneven 64-circuit batch slices/s on 1 GB300", "value": slices / (ms / 1e3),
        "unit": "slices/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "dtype": args.prec, "data": "synthetic",
        "config": {"workload": "64 seeded circuits, 4x4..4x7 grids, depth 10..16, 2^2..2^8 slices, "
                               "l = 8, G = 16 (16..28 qubits)", "circuits": len(ws), "slices": slices,
                   "slice_batch": "per plan, from a 16 GiB budget: " + ",".join(
                       str(p.max_slice_batch) for p in plans),
                   "graph_branches": branches, "workspace_bytes": wsz,
                   "hilo": "auto (3e-3)" if args.hilo_auto else args.hilo,
                   "path": "greedy and bisection + subtree reconfiguration" if refined else "greedy",
                   "l2": "not flushed (one batched call)"},
        "useful_tflops": flops / (ms / 1e3) / 1e12, "host_planning_s": plan_s}), flush=True)
    for p in plans:
        p.close()


def run_sycamore(args):
    """The 53-qubit Sycamore-shaped circuit, 20 cycles (l = 10 open qubits, G = 16
    blocks, k = 1 per block): a bisection-search plan (refined by subtree
    reconfiguration unless --path greedy) under a 2^32-element cap,
    a few seeded slices timed one by one, and the extrapolated time to 1e6
    samples at the fidelity whose top-1 XEB is 0.002 (Eq. 4: F = 0.002 /
    (H_1024 - 1); slices needed per block batch = F x 2^(sliced bonds))."""
    refined = args.path != "greedy"
    import math
    import torch
    import workloads as W
    from paper_2406_18889_gb300 import binding as B
    from paper_2406_18889_gb300 import engine as E
    from paper_2406_18889_gb300 import network as N
    from paper_2406_18889_gb300 import pathfind as P
    torch.cuda.set_device(0)
    w = W.workload("sycamore53_d20", cycles=20, l=10, G=16)
    tn = N.circuit_network(w.circuit, w.open_qubits, w.closed_qubits, w.closed_bits)
    t0 = time.perf_counter()
    tree = P.plan_tree(tn, cap_log2=32, restarts=1, method="partition", refine=refined,
                       workers=host_cores() if refined else 0)
    plan_s = time.perf_counter() - t0
    flags = B.TN_FLAG_HOIST_INVARIANT | (B.TN_FLAG_HILO_AUTO if args.hilo_auto and args.prec != "c64" else 0)
    plan = E.Plan(tn, tree, prec=args.prec, flags=flags, max_slice_batch=1, hilo_tol=2e-3)
    s = len(tree.sliced_edges)
    ids = W.draw_slice_subset(1 << min(s, 62), 1 + args.steps, seed=20)
    amps = plan.contract(ids[:1])  # warm-up: graph capture
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(1, 1 + args.steps):
        plan.contract(ids[i:i + 1], out=amps, accumulate=True)
    e1.record(stream)
    torch.cuda.synchronize()
    t_slice = e0.elapsed_time(e1) / args.steps / 1e3
    useful = plan.info["useful_flops_per_slice"]
    # error of the timed precision on the last timed slice, against the complex64 path
    precision = None
    if args.prec != "c64":
        one = plan.contract(ids[-1:])
        plan64 = E.Plan(tn, tree, prec="c64", flags=B.TN_FLAG_HOIST_INVARIANT, max_slice_batch=1)
        ref = plan64.contract(ids[-1:])
        plan64.close()
        torch.cuda.synchronize()
        rel = float(torch.linalg.vector_norm(one - ref) / torch.linalg.vector_norm(ref))
        pr = plan.precision()
        precision = {"rel_l2_vs_complex64_one_slice": rel, "split_steps": pr["n_hilo_steps"],
                     "tensor_core_steps": pr["n_tc_steps"], "calibration_rel_l2": pr["rel_l2_chosen"]}
    F = 0.002 / (sum(1.0 / j for j in range(1, 1025)) - 1.0)
    slices_per_batch = F * 2.0 ** s
    batches = 1e6 / w.G
    print(json.dumps({
        "metric": "53-qubit 20-cycle sliced contraction: seconds per slice on 1 GB300", "value": t_slice,
        "unit": "s/slice", "higher_is_better": False, "steps": args.steps, "dtype": args.prec,
        "data": "synthetic", "config": {"workload": "53-qubit Sycamore-shaped diagonal grid, 20 cycles, l = 10, "
                                                  "G = 16, k = 1 per block", "cap_log2": 32, "sliced_bonds": s,
                                        "path": "recursive bisection + subtree reconfiguration" if refined
                                        else "recursive bisection"},
        "useful_tflops": useful / t_slice / 1e12, "useful_flops_per_slice": useful, "precision": precision,
        "path_cost_complex_macs": tree.cost_per_slice * 2.0 ** s, "host_planning_s": plan_s,
        "extrapolation_1e6_samples": {"fidelity_F": F, "slices_per_block_batch": slices_per_batch,
                                      "block_batches": batches,
                                      "seconds": slices_per_batch * batches * t_slice,
                                      "note": "the total is set by the path's cost per slice x 2^sliced bonds"}}),
          flush=True)
    plan.close()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp16", choices=["c64", "bf16", "fp16"])
    ap.add_argument("--hilo", action="store_true", help="split-precision (hi + lo) tensor-core steps")
    ap.add_argument("--hilo-auto", action="store_true",
                    help="split products only where the calibration needs them for relative L2 <= 3e-3")
    ap.add_argument("--no-c64", action="store_true", help="skip timing the complex64 path alongside")
    ap.add_argument("--hoist", action="store_true",
                    help="contract slice-independent subtrees once, at plan creation, instead of once in every "
                         "batch (the default: every step does all of its batch's work)")
    ap.add_argument("--tune", action="store_true",
                    help="also run the plan tuner (operand type, slice batch, split placement, launch forms)")
    ap.add_argument("--serial-graph", action="store_true",
                    help="one chain of launches per batch graph instead of concurrent branches")
    ap.add_argument("--path", default="time", choices=["time", "refined", "greedy"],
                    help="contraction tree: time (default; flop-refined greedy and bisection trees re-optimised "
                         "for the estimated time of one slice batch: multiply-adds plus the elements moved), "
                         "refined (fewest multiply-adds) or greedy")
    ap.add_argument("--autotune", action="store_true",
                    help="time the tensor-core steps' launch forms on one batch first and keep the fastest")
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--partition", default="slices", choices=["slices", "blocks"],
                    help="N > 1: split the slices of one problem over the GPUs and reduce their FP64 partials "
                         "(slices, strong scaling), or give every GPU its own blocks (blocks, weak scaling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-region", action="store_true",
                    help="one contraction between cudaProfilerStart/Stop after warm-up (ncu --profile-from-start off)")
    ap.add_argument("--only-timed", action="store_true",
                    help="run warm-up and timed steps only (for ncu launch lists)")
    ap.add_argument("--workload", default="grid4x6_d14", choices=["grid4x6_d14", "uneven64", "sycamore53_d20"],
                    help="uneven64: the 64-circuit batch (4x4..4x7 grids, depth 10..16, 2^2..2^8 "
                         "slices, l = 8, G = 16) in one batched call, timed as total slices / call time")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "uneven64":
        run_uneven(args)
    elif args.workload == "sycamore53_d20":
        run_sycamore(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
