"""User-facing layer: circuit workload -> plan -> amplitudes -> top-k -> XEB.

PyTorch provides device memory and streams only; every contraction, the
FP64 slice sum, top-k and XEB run in the library's CUDA kernels through the C
ABI (``binding``).
"""
from __future__ import annotations

import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from . import binding as B
from .network import TensorNetwork, circuit_network
from .pathfind import Tree, plan_tree

PREC = {"c64": B.TN_PREC_C64, "bf16": B.TN_PREC_BF16, "fp16": B.TN_PREC_FP16}


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required (the library has no CPU path)")
    return torch


def flatten_network(tn: TensorNetwork):
    rank = [len(e) for e in tn.leaf_edges]
    edges = [e for es in tn.leaf_edges for e in es]
    data = np.concatenate([d.reshape(-1) for d in tn.leaf_data]) if tn.leaf_data else np.zeros(0, complex)
    return rank, edges, data


class Plan:
    """A contraction plan living on the current CUDA device."""

    def __init__(self, tn: TensorNetwork, tree: Tree, prec: str = "c64", flags: int = 0,
                 max_slice_batch: int = 64, mem_cap_bytes: int = 0, stream=None,
                 own_workspace: bool = True, hilo_steps=None, hilo_tol: float = 0.0):
        """``max_slice_batch = 0`` lets the library choose the batch from the
        memory budget; ``hilo_steps`` (per step 0/1) or ``flags`` with
        ``TN_FLAG_HILO_AUTO`` (target ``hilo_tol``) place split-precision
        products on chosen tensor-core steps."""
        torch = _torch()
        self.tn, self.tree = tn, tree
        self.n_slices_total = 1 << len(tree.sliced_edges)
        rank, edges, data = flatten_network(tn)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.handle = B.tn_plan_create(rank, edges, tn.edge_dim, data, tn.open_edges, tn.block_edge,
                                       np.asarray(tree.pairs, dtype=np.int32).reshape(-1),
                                       tree.sliced_edges, PREC[prec], flags, max_slice_batch,
                                       mem_cap_bytes, s.cuda_stream, hilo_steps=hilo_steps, hilo_tol=hilo_tol)
        self.info = B.tn_plan_query(self.handle)
        self.prec, self.flags = prec, flags
        self.max_slice_batch = B.tn_plan_slice_batch(self.handle)
        self.G = tn.n_blocks
        self.J = 1
        for e in tn.open_edges:
            self.J *= tn.edge_dim[e]
        # plans run back to back in one batched call share the caller's workspace
        self.workspace = torch.empty(max(self.info["workspace_bytes"], 256), dtype=torch.uint8,
                                     device="cuda") if own_workspace else None

    def steps(self) -> dict:
        return B.tn_plan_steps(self.handle)

    def precision(self) -> dict:
        return B.tn_plan_precision(self.handle)

    def contract(self, slice_ids: Optional[Sequence[int]] = None, out=None, accumulate: bool = False,
                 stream=None):
        """amps [G, 2^l] complex128 = sum over the given slices (all when None)."""
        torch = _torch()
        if slice_ids is None:
            slice_ids = np.arange(self.n_slices_total, dtype=np.int64)
        if out is None:
            out = torch.empty((self.G, self.J), dtype=torch.complex128, device="cuda")
        s = stream if stream is not None else torch.cuda.current_stream()
        if self.workspace is None:
            raise ValueError("plan created without a workspace: use tn_contract_slices_batched")
        B.tn_contract_slices(self.handle, slice_ids, out.data_ptr(), int(accumulate),
                             self.workspace.data_ptr(), self.workspace.numel(), s.cuda_stream)
        return out

    def autotune(self, slice_ids: Optional[Sequence[int]] = None, reps: int = 3, cache: Optional[str] = None,
                 stream=None) -> np.ndarray:
        """Launch forms of the tensor-core steps (tile width, row halves),
        timed on one batch of slices (the first ``max_slice_batch`` of
        ``slice_ids``, default the first slices) by ``tn_plan_autotune``.  With
        ``cache`` (a JSON file of forms keyed by precision, flags and step shape),
        forms found there are set without timing, and newly tuned ones are added
        to the file.  Returns int32 [n_steps, 2] (zeros: step not tuned)."""
        import json
        torch = _torch()
        st = self.steps()
        kinds = st["kinds"]
        keys = [f"{self.prec}/{self.flags}/{st['batch'][t]}x{st['m'][t]}x{st['n'][t]}x{st['k'][t]}/{kinds[t]}"
                for t in range(len(kinds))]
        tuned = [t for t in range(len(kinds)) if (kinds[t] & 8) and not (kinds[t] & 4)]
        known = {}
        if cache and os.path.exists(cache):
            with open(cache) as fh:
                known = json.load(fh)
        if tuned and all(keys[t] in known for t in tuned):
            forms = np.zeros((len(kinds), 2), np.int32)
            for t in tuned:
                forms[t] = known[keys[t]]
            try:
                B.tn_plan_set_tuning(self.handle, forms)
                return forms
            except B.TNError:
                pass  # a stale entry: tune again
        if slice_ids is None:
            slice_ids = np.arange(min(self.max_slice_batch, self.n_slices_total), dtype=np.int64)
        ids = np.asarray(slice_ids, dtype=np.int64)[: self.max_slice_batch]
        if self.workspace is None:
            raise ValueError("plan created without a workspace")
        s = stream if stream is not None else torch.cuda.current_stream()
        out = torch.empty((self.G, self.J), dtype=torch.complex128, device="cuda")
        forms = B.tn_plan_autotune(self.handle, ids, out.data_ptr(), self.workspace.data_ptr(),
                                   self.workspace.numel(), s.cuda_stream, reps)
        if cache and tuned:
            for t in tuned:
                known[keys[t]] = [int(x) for x in forms[t]]
            tmp = cache + ".tmp"
            with open(tmp, "w") as fh:
                json.dump(known, fh, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return forms

    def close(self):
        if getattr(self, "handle", None):
            B.tn_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune_plan(tn: TensorNetwork, tree: Tree, tol: float = 3e-3, precs: Sequence[str] = ("fp16", "bf16"),
              batches: Sequence[int] = (16, 32, 64), flags: int = 0, slice_ids=None, reps: int = 3,
              launch_forms: bool = True):
    """Split choices and launch forms picked by timing, under an accuracy bar.

    Every candidate -- 16-bit operand type x slice batch -- is planned with
    its split-precision (hi + lo) products placed by calibration
    (``TN_FLAG_HILO_AUTO``: the fewest tensor-core steps split so that the
    calibration batch's relative L2 against a complex64 pass is <= ``tol``),
    its tensor-core launch forms tuned (``Plan.autotune``), then timed over
    ``slice_ids`` (default all slices; ``reps`` calls after one warm-up).  The
    fastest candidate whose calibrated error meets ``tol`` is kept.  Returns
    (plan, table): the chosen plan, open, and one row per candidate (prec,
    batch, slices_per_s, rel_l2, n_hilo_steps, n_tc_steps, chosen)."""
    torch = _torch()
    rows, best, best_plan = [], None, None
    n_total = 1 << len(tree.sliced_edges)
    ids = np.arange(n_total, dtype=np.int64) if slice_ids is None else np.asarray(slice_ids, dtype=np.int64)
    for prec in precs:
        for b in batches:
            plan = Plan(tn, tree, prec=prec, flags=flags | B.TN_FLAG_HILO_AUTO, max_slice_batch=b, hilo_tol=tol)
            if launch_forms:
                plan.autotune(ids, reps=2)
            out = torch.empty((plan.G, plan.J), dtype=torch.complex128, device="cuda")
            plan.contract(ids, out=out)
            s = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                plan.contract(ids, out=out)
            e1.record(s)
            torch.cuda.synchronize()
            pr = plan.precision()
            row = dict(prec=prec, batch=plan.max_slice_batch, slices_per_s=len(ids) * reps / (e0.elapsed_time(e1) / 1e3),
                       rel_l2=pr["rel_l2_chosen"], n_hilo_steps=pr["n_hilo_steps"], n_tc_steps=pr["n_tc_steps"],
                       chosen=False)
            rows.append(row)
            ok = 0 <= row["rel_l2"] <= tol
            if ok and (best is None or row["slices_per_s"] > best["slices_per_s"]):
                if best_plan is not None:
                    best_plan.close()
                best, best_plan = row, plan
            else:
                plan.close()
    if best is None:
        raise ValueError("no candidate meets the accuracy bar")
    best["chosen"] = True
    return best_plan, rows


def contract_checkpointed(plan: "Plan", slice_ids, path: str, chunk: Optional[int] = None, out=None,
                          on_chunk=None):
    """Sum the given slices in chunks, saving (ids, number finished, FP64 partial
    sum) to the .npz file `path` after every chunk; a checkpoint already at
    `path` for the same slice list is resumed from where it stopped.  Chunks are
    processed in order and each adds into the FP64 sum, so a resumed run gives
    the same bits as an uninterrupted one.  `on_chunk(i, n_done)` is called
    after chunk i is saved (progress; an exception there leaves a valid
    checkpoint behind)."""
    torch = _torch()
    ids = np.ascontiguousarray(np.asarray(slice_ids, dtype=np.int64))
    chunk = int(chunk or plan.max_slice_batch)
    if out is None:
        out = torch.empty((plan.G, plan.J), dtype=torch.complex128, device="cuda")
    done = 0
    if os.path.exists(path):
        ck = np.load(path)
        if not np.array_equal(ck["ids"], ids):
            raise ValueError(f"checkpoint {path} belongs to another slice list")
        done = int(ck["done"])
        out.copy_(torch.as_tensor(ck["amps"], device=out.device))
    i = done // chunk
    while done < len(ids):
        part = ids[done:done + chunk]
        plan.contract(part, out=out, accumulate=done > 0)
        done += len(part)
        tmp = path + ".tmp.npz"
        np.savez(tmp, ids=ids, done=np.int64(done), amps=out.cpu().numpy())
        os.replace(tmp, path)
        if on_chunk is not None:
            on_chunk(i, done)
        i += 1
    if len(ids) == 0:
        plan.contract([], out=out)
    return out


def topk(amps, k: int, inv_f: float, block_base, open_bit_pos, global_mode: bool = False, stream=None):
    """(idx int64, p float64) device tensors: [G, k] per block or [k] global."""
    torch = _torch()
    G, Bsz = amps.shape
    shape = (k,) if global_mode else (G, k)
    idx = torch.empty(shape, dtype=torch.int64, device="cuda")
    p = torch.empty(shape, dtype=torch.float64, device="cuda")
    base = block_base if hasattr(block_base, "data_ptr") else torch.as_tensor(
        np.asarray(block_base, dtype=np.int64), device="cuda")
    s = stream if stream is not None else torch.cuda.current_stream()
    B.tn_topk_postprocess(amps.data_ptr(), G, Bsz, k, inv_f, int(global_mode), base.data_ptr(),
                          np.asarray(open_bit_pos, dtype=np.int64), idx.data_ptr(), p.data_ptr(),
                          s.cuda_stream)
    return idx, p


def xeb(q, n_qubits: int, stream=None) -> float:
    torch = _torch()
    q = q.reshape(-1).contiguous()
    s = stream if stream is not None else torch.cuda.current_stream()
    return B.tn_xeb(q.data_ptr(), q.numel(), n_qubits, s.cuda_stream)


@dataclass
class Prepared:
    tn: TensorNetwork
    tree: Tree


def prepare(workload, n_sliced: Optional[int] = None, restarts: int = 4, seed: int = 0,
            sliced_wires: Optional[Sequence] = None, method: str = "greedy", refine: bool = False,
            workers: int = 0, objective: str = "flops", batch_log2: Optional[int] = None) -> Prepared:
    """Network + contraction tree of a workload (host planning, once per circuit).
    ``method`` / ``refine`` / ``workers`` / ``objective`` / ``batch_log2`` select the
    path search (``pathfind.plan_tree``)."""
    tn = circuit_network(workload.circuit, workload.open_qubits, workload.closed_qubits,
                         workload.closed_bits)
    sliced = None
    if sliced_wires is not None:
        sliced = [tn.edge_of_wire[tuple(w)] for w in sliced_wires]
    s = workload.n_sliced if n_sliced is None else n_sliced
    tree = plan_tree(tn, n_sliced=s, restarts=restarts, seed=seed, sliced=sliced, method=method, refine=refine,
                     workers=workers, objective=objective, batch_log2=batch_log2)
    return Prepared(tn, tree)
