"""Thin ctypes binding of the C ABI in include/tn.h (argument marshalling only).

Every function has the C name and forwards plain host arrays (numpy) and
device pointers (ints) to the library; all contraction work happens in the
library's CUDA kernels.  Loading fails loudly when the library has not been
built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
from pathlib import Path
from typing import Optional, Sequence

import numpy as np

LIB_PATH = Path(__file__).resolve().parent / "_build" / "libtn.so"

TN_OK = 0
(TN_ERR_INVALID_ARG, TN_ERR_OOM, TN_ERR_CUDA, TN_ERR_TIMEOUT, TN_ERR_UNSUPPORTED,
 TN_ERR_NUMERIC) = 1, 2, 3, 4, 5, 6
STATUS_NAMES = {0: "TN_OK", 1: "TN_ERR_INVALID_ARG", 2: "TN_ERR_OOM", 3: "TN_ERR_CUDA",
                4: "TN_ERR_TIMEOUT", 5: "TN_ERR_UNSUPPORTED", 6: "TN_ERR_NUMERIC"}
TN_PREC_C64, TN_PREC_BF16, TN_PREC_FP16 = 0, 1, 2
TN_FLAG_HOIST_INVARIANT = 0x1
TN_FLAG_NO_GRAPH = 0x2
TN_FLAG_PLAN_ONLY = 0x4
TN_FLAG_HILO = 0x8
TN_FLAG_FINE_ACC = 0x20
TN_FLAG_HILO_AUTO = 0x40
TN_FLAG_SERIAL_GRAPH = 0x80

EXPORTS = ("tn_plan_create", "tn_plan_destroy", "tn_plan_query", "tn_plan_steps",
           "tn_contract_slices", "tn_contract_slices_batched", "tn_contract_slices_profile",
           "tn_topk_postprocess", "tn_xeb", "tn_contract_slices_noalloc", "tn_selftest_gemm_tc", "tn_plan_status",
           "tn_permute", "tn_selftest_bounded_wait", "tn_selftest_fp32_peak", "tn_plan_autotune",
           "tn_plan_set_tuning", "tn_plan_slice_batch", "tn_plan_precision", "tn_batched_workspace_bytes", "tn_sum_partials", "tn_last_error",
           "tn_version")


class TNError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class NetworkDesc(ctypes.Structure):
    _fields_ = [("n_leaves", ctypes.c_int32), ("n_edges", ctypes.c_int32),
                ("leaf_rank", ctypes.POINTER(ctypes.c_int32)),
                ("leaf_edges", ctypes.POINTER(ctypes.c_int32)),
                ("edge_dim", ctypes.POINTER(ctypes.c_int64)),
                ("leaf_data", ctypes.c_void_p),
                ("n_open", ctypes.c_int32), ("open_edges", ctypes.POINTER(ctypes.c_int32)),
                ("block_edge", ctypes.c_int32)]


class TreeDesc(ctypes.Structure):
    _fields_ = [("n_steps", ctypes.c_int32), ("pairs", ctypes.POINTER(ctypes.c_int32)),
                ("n_sliced", ctypes.c_int32), ("sliced_edges", ctypes.POINTER(ctypes.c_int32))]


class PlanOptions(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("max_slice_batch", ctypes.c_int32), ("mem_cap_bytes", ctypes.c_int64),
                ("hilo_steps", ctypes.POINTER(ctypes.c_uint8)), ("hilo_tol", ctypes.c_double)]


_lib: Optional[ctypes.CDLL] = None


def load() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_2406_18889_gb300.build.build() first "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(str(LIB_PATH))
    vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    p_i64 = ctypes.POINTER(ctypes.c_int64)
    p_i32 = ctypes.POINTER(ctypes.c_int32)
    lib.tn_plan_create.argtypes = [ctypes.POINTER(NetworkDesc), ctypes.POINTER(TreeDesc),
                                   ctypes.POINTER(PlanOptions), vp, ctypes.POINTER(vp)]
    lib.tn_plan_destroy.argtypes = [vp]
    lib.tn_plan_query.argtypes = [vp, p_i64, p_i64, p_i64, p_i64]
    lib.tn_plan_steps.argtypes = [vp, i32, p_i64, p_i64, p_i64, p_i64, p_i32, p_i32]
    lib.tn_contract_slices.argtypes = [vp, p_i64, i64, vp, ctypes.c_int, vp, u64, vp]
    lib.tn_contract_slices_batched.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(p_i64), p_i64,
                                               ctypes.POINTER(vp), ctypes.c_int, vp, u64, vp]
    lib.tn_contract_slices_profile.argtypes = [vp, p_i64, i64, vp, ctypes.c_int, vp, u64, vp, i32, p_i32,
                                               ctypes.POINTER(ctypes.c_float),
                                               ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_double), p_i32]
    lib.tn_topk_postprocess.argtypes = [vp, i64, i64, i32, ctypes.c_double, ctypes.c_int, vp, p_i64,
                                        i32, vp, vp, vp]
    lib.tn_xeb.argtypes = [vp, i64, i32, ctypes.POINTER(ctypes.c_double), vp]
    lib.tn_contract_slices_noalloc.argtypes = [vp, p_i64, i64, vp, ctypes.c_int, vp]
    lib.tn_plan_status.argtypes = [vp, vp]
    lib.tn_permute.argtypes = [vp, vp, i32, p_i32, i32, vp]
    lib.tn_selftest_gemm_tc.argtypes = [i64, i64, i64, i64, i32, ctypes.c_uint64,
                                        ctypes.POINTER(ctypes.c_double), vp]
    lib.tn_selftest_bounded_wait.argtypes = [ctypes.c_uint64, vp]
    lib.tn_selftest_fp32_peak.argtypes = [ctypes.POINTER(ctypes.c_double), vp]
    lib.tn_plan_autotune.argtypes = [vp, p_i64, i64, vp, vp, u64, vp, i32, p_i32]
    lib.tn_plan_set_tuning.argtypes = [vp, p_i32, i32]
    lib.tn_plan_slice_batch.argtypes = [vp, p_i32]
    lib.tn_sum_partials.argtypes = [vp, i64, i64, vp, ctypes.c_int, vp]
    lib.tn_batched_workspace_bytes.argtypes = [ctypes.POINTER(vp), i32, p_i64, i32, p_i64]
    p_f64 = ctypes.POINTER(ctypes.c_double)
    lib.tn_plan_precision.argtypes = [vp, p_f64, p_f64, p_i32, p_i32]
    for name in EXPORTS[:-2]:
        getattr(lib, name).restype = ctypes.c_int
    lib.tn_last_error.restype = ctypes.c_char_p
    lib.tn_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status: int):
    if status != TN_OK:
        raise TNError(status, load().tn_last_error().decode())


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _p(arr: np.ndarray, ctype):
    return arr.ctypes.data_as(ctypes.POINTER(ctype))


def tn_plan_create(leaf_rank, leaf_edges, edge_dim, leaf_data, open_edges, block_edge: int,
                   pairs, sliced_edges, prec: int = TN_PREC_C64, flags: int = 0,
                   max_slice_batch: int = 1, mem_cap_bytes: int = 0, stream: int = 0,
                   hilo_steps=None, hilo_tol: float = 0.0) -> int:
    rank, edges, dims = _i32(leaf_rank), _i32(leaf_edges), _i64(edge_dim)
    data = np.ascontiguousarray(np.asarray(leaf_data, dtype=np.complex128))
    opens, pr, sl = _i32(open_edges), _i32(pairs).reshape(-1), _i32(sliced_edges)
    net = NetworkDesc(len(rank), len(dims), _p(rank, ctypes.c_int32), _p(edges, ctypes.c_int32),
                      _p(dims, ctypes.c_int64), data.ctypes.data, len(opens),
                      _p(opens, ctypes.c_int32), int(block_edge))
    tree = TreeDesc(len(pr) // 2, _p(pr, ctypes.c_int32), len(sl), _p(sl, ctypes.c_int32))
    hl = None if hilo_steps is None else np.ascontiguousarray(np.asarray(hilo_steps, dtype=np.uint8))
    opt = PlanOptions(int(prec), int(flags), int(max_slice_batch), int(mem_cap_bytes),
                      None if hl is None else _p(hl, ctypes.c_uint8), float(hilo_tol))
    out = ctypes.c_void_p()
    _check(load().tn_plan_create(ctypes.byref(net), ctypes.byref(tree), ctypes.byref(opt),
                                 ctypes.c_void_p(stream), ctypes.byref(out)))
    return out.value


def tn_plan_destroy(plan: int) -> None:
    _check(load().tn_plan_destroy(ctypes.c_void_p(plan)))


def tn_plan_slice_batch(plan: int) -> int:
    b = ctypes.c_int32()
    _check(load().tn_plan_slice_batch(ctypes.c_void_p(plan), ctypes.byref(b)))
    return b.value


def tn_plan_precision(plan: int) -> dict:
    e1, e0 = ctypes.c_double(), ctypes.c_double()
    ntc, nhl = ctypes.c_int32(), ctypes.c_int32()
    _check(load().tn_plan_precision(ctypes.c_void_p(plan), ctypes.byref(e1), ctypes.byref(e0), ctypes.byref(ntc),
                                    ctypes.byref(nhl)))
    return dict(rel_l2_chosen=e1.value, rel_l2_none=e0.value, n_tc_steps=ntc.value, n_hilo_steps=nhl.value)


def tn_plan_query(plan: int) -> dict:
    v = [ctypes.c_int64() for _ in range(4)]
    _check(load().tn_plan_query(ctypes.c_void_p(plan), *[ctypes.byref(x) for x in v]))
    return dict(useful_flops_per_slice=v[0].value, algo_bytes_per_slice=v[1].value,
                peak_intermediate_bytes=v[2].value, workspace_bytes=v[3].value)


def tn_plan_steps(plan: int) -> dict:
    n = ctypes.c_int32()
    _check(load().tn_plan_steps(ctypes.c_void_p(plan), 0, None, None, None, None, None, ctypes.byref(n)))
    cnt = n.value
    b, m, nn, k = (np.zeros(cnt, np.int64) for _ in range(4))
    kinds = np.zeros(cnt, np.int32)
    _check(load().tn_plan_steps(ctypes.c_void_p(plan), cnt, _p(b, ctypes.c_int64), _p(m, ctypes.c_int64),
                                _p(nn, ctypes.c_int64), _p(k, ctypes.c_int64), _p(kinds, ctypes.c_int32),
                                ctypes.byref(n)))
    return dict(batch=b, m=m, n=nn, k=k, kinds=kinds)


def tn_plan_autotune(plan: int, slice_ids, amps_ptr: int, ws_ptr: int, ws_bytes: int, stream: int = 0,
                     reps: int = 3) -> np.ndarray:
    """Tunes the tensor-core steps' launch forms; returns int32 [n_steps, 2]
    (tile width, row halves; zeros for steps that are not tuned)."""
    ids = _i64(slice_ids)
    n = ctypes.c_int32()
    _check(load().tn_plan_steps(ctypes.c_void_p(plan), 0, None, None, None, None, None, ctypes.byref(n)))
    forms = np.zeros((n.value, 2), np.int32)
    _check(load().tn_plan_autotune(ctypes.c_void_p(plan), _p(ids, ctypes.c_int64), len(ids),
                                   ctypes.c_void_p(amps_ptr), ctypes.c_void_p(ws_ptr), int(ws_bytes),
                                   ctypes.c_void_p(stream), int(reps), _p(forms, ctypes.c_int32)))
    return forms


def tn_plan_set_tuning(plan: int, forms) -> None:
    f = np.ascontiguousarray(np.asarray(forms, dtype=np.int32).reshape(-1, 2))
    _check(load().tn_plan_set_tuning(ctypes.c_void_p(plan), _p(f, ctypes.c_int32), f.shape[0]))


def tn_contract_slices(plan: int, slice_ids, amps_ptr: int, accumulate: int, ws_ptr: int, ws_bytes: int,
                       stream: int = 0) -> None:
    ids = _i64(slice_ids)
    _check(load().tn_contract_slices(ctypes.c_void_p(plan), _p(ids, ctypes.c_int64), len(ids),
                                     ctypes.c_void_p(amps_ptr), int(accumulate), ctypes.c_void_p(ws_ptr),
                                     int(ws_bytes), ctypes.c_void_p(stream)))


def tn_contract_slices_profile(plan: int, slice_ids, amps_ptr: int, accumulate: int, ws_ptr: int,
                               ws_bytes: int, stream: int = 0, max_records: int = 1 << 16) -> dict:
    ids = _i64(slice_ids)
    kind = np.zeros(max_records, np.int32)
    ms = np.zeros(max_records, np.float32)
    flops = np.zeros(max_records, np.float64)
    nbytes = np.zeros(max_records, np.float64)
    n = ctypes.c_int32()
    _check(load().tn_contract_slices_profile(
        ctypes.c_void_p(plan), _p(ids, ctypes.c_int64), len(ids), ctypes.c_void_p(amps_ptr), int(accumulate),
        ctypes.c_void_p(ws_ptr), int(ws_bytes), ctypes.c_void_p(stream), max_records,
        _p(kind, ctypes.c_int32), _p(ms, ctypes.c_float), _p(flops, ctypes.c_double),
        _p(nbytes, ctypes.c_double), ctypes.byref(n)))
    c = min(n.value, max_records)
    return dict(kind=kind[:c], ms=ms[:c], flops=flops[:c], bytes=nbytes[:c], n_launches=n.value)


def tn_contract_slices_batched(plans: Sequence[int], slice_ids: Sequence, amps_ptrs: Sequence[int],
                               accumulate: int, ws_ptr: int, ws_bytes: int, stream: int = 0) -> None:
    n = len(plans)
    id_arrays = [_i64(s) for s in slice_ids]
    VP = ctypes.c_void_p * n
    PP = ctypes.POINTER(ctypes.c_int64) * n
    counts = _i64([len(a) for a in id_arrays])
    _check(load().tn_contract_slices_batched(
        VP(*[ctypes.c_void_p(p) for p in plans]), n, PP(*[_p(a, ctypes.c_int64) for a in id_arrays]),
        _p(counts, ctypes.c_int64), VP(*[ctypes.c_void_p(a) for a in amps_ptrs]), int(accumulate),
        ctypes.c_void_p(ws_ptr), int(ws_bytes), ctypes.c_void_p(stream)))


def tn_batched_workspace_bytes(plans: Sequence[int], n_slices: Sequence[int], max_branches: int = 8) -> int:
    n = len(plans)
    arr = (ctypes.c_void_p * max(n, 1))(*[ctypes.c_void_p(p) for p in plans])
    ns = _i64(n_slices)
    out = ctypes.c_int64()
    _check(load().tn_batched_workspace_bytes(arr, n, _p(ns, ctypes.c_int64), int(max_branches), ctypes.byref(out)))
    return out.value


def tn_sum_partials(parts_ptr: int, n_parts: int, n_amps: int, out_ptr: int, accumulate: int = 0,
                    stream: int = 0) -> None:
    _check(load().tn_sum_partials(ctypes.c_void_p(parts_ptr), int(n_parts), int(n_amps), ctypes.c_void_p(out_ptr),
                                  int(accumulate), ctypes.c_void_p(stream)))


def tn_topk_postprocess(amps_ptr: int, G: int, B: int, k: int, inv_f: float, global_mode: int,
                        block_base_ptr: int, open_bit_pos, out_idx_ptr: int, out_p_ptr: int,
                        stream: int = 0) -> None:
    pos = _i64(open_bit_pos)
    _check(load().tn_topk_postprocess(ctypes.c_void_p(amps_ptr), int(G), int(B), int(k), float(inv_f),
                                      int(global_mode), ctypes.c_void_p(block_base_ptr),
                                      _p(pos, ctypes.c_int64), len(pos), ctypes.c_void_p(out_idx_ptr),
                                      ctypes.c_void_p(out_p_ptr), ctypes.c_void_p(stream)))


def tn_xeb(q_ptr: int, n_sel: int, n_qubits: int, stream: int = 0) -> float:
    out = ctypes.c_double()
    _check(load().tn_xeb(ctypes.c_void_p(q_ptr), int(n_sel), int(n_qubits), ctypes.byref(out),
                         ctypes.c_void_p(stream)))
    return out.value


def tn_contract_slices_noalloc(plan: int, slice_ids, amps_ptr: int, accumulate: int, stream: int = 0) -> None:
    """Same contraction as tn_contract_slices, using the library's static 64 MiB
    device workspace instead of a caller-allocated one (no device allocation)."""
    ids = _i64(slice_ids)
    _check(load().tn_contract_slices_noalloc(ctypes.c_void_p(plan), _p(ids, ctypes.c_int64), len(ids),
                                             ctypes.c_void_p(amps_ptr), int(accumulate),
                                             ctypes.c_void_p(stream)))


def tn_selftest_bounded_wait(limit_ns: int, stream: int = 0) -> None:
    """Raises TNError(TN_ERR_TIMEOUT) when the device wait gave up (the expected outcome)."""
    _check(load().tn_selftest_bounded_wait(ctypes.c_uint64(int(limit_ns)), ctypes.c_void_p(stream)))


def tn_selftest_fp32_peak(stream: int = 0) -> float:
    out = ctypes.c_double()
    _check(load().tn_selftest_fp32_peak(ctypes.byref(out), ctypes.c_void_p(stream)))
    return out.value


def tn_selftest_gemm_tc(nbt: int, M: int, N: int, K: int, prec: int, seed: int = 1, stream: int = 0) -> float:
    out = ctypes.c_double()
    _check(load().tn_selftest_gemm_tc(int(nbt), int(M), int(N), int(K), int(prec), int(seed),
                                      ctypes.byref(out), ctypes.c_void_p(stream)))
    return out.value


def tn_plan_status(plan: int, stream: int = 0) -> None:
    _check(load().tn_plan_status(ctypes.c_void_p(plan), ctypes.c_void_p(stream)))


def tn_permute(in_ptr: int, out_ptr: int, out_bit, elem_bytes: int, stream: int = 0) -> None:
    ob = _i32(out_bit)
    _check(load().tn_permute(ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), len(ob), _p(ob, ctypes.c_int32),
                             int(elem_bytes), ctypes.c_void_p(stream)))


def tn_last_error() -> str:
    return load().tn_last_error().decode()


def tn_version() -> str:
    return load().tn_version().decode()
