"""Batched uneven circuits (64 seeded circuits, 4x4..4x7 grids, depth 10..16,
2^2..2^8 slices, l = 8, G = 16): a subset -- six circuits of up to 24 qubits and
one 28-qubit circuit -- is contracted in one tn_contract_slices_batched call
(one captured graph with concurrent branches) and each circuit is checked
against its own FP64 state vector, in complex64, fp16 and bf16 (split
products placed by calibration).  Slice batches are chosen from free memory."""
import numpy as np
import pytest

import workloads as W
from oracle import statevector as sv
from parity_checks import assert_amplitudes_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_18889_gb300 import engine
    return engine


def _subset():
    ws = W.configs.uneven_batch(64)
    small = [w for w in ws if w.n_qubits <= 24][:6]
    big = [ws[12]]  # 4x7 grid (28 qubits), 10 cycles, 2^6 slices
    assert big[0].n_qubits == 28
    return small + big


@pytest.fixture(scope="module")
def circuits(E):
    ws = _subset()
    refs = []
    for w in ws:
        psi = sv.simulate(w.circuit)
        ref, _ = sv.block_amplitudes(psi, w.n_qubits, w.open_qubits, w.closed_qubits, w.closed_bits)
        refs.append(ref)
        del psi
    preps = [E.prepare(w, restarts=1) for w in ws]
    return ws, refs, preps


def _run_batched(E, plans, ids, outs, ws_bytes=None):
    import torch
    from paper_2406_18889_gb300 import binding as B
    need = B.tn_batched_workspace_bytes([p.handle for p in plans], [len(x) for x in ids])
    wsz = need if ws_bytes is None else ws_bytes
    wsb = torch.empty(max(wsz, 256), dtype=torch.uint8, device="cuda")
    B.tn_contract_slices_batched([p.handle for p in plans], ids, [o.data_ptr() for o in outs], 0,
                                 wsb.data_ptr(), wsz, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return need


@pytest.mark.parametrize("prec,tol", [("c64", 1e-5), ("fp16", 3e-3), ("bf16", 3e-3)])
def test_uneven_batch_against_statevectors(E, circuits, prec, tol):
    import torch
    from paper_2406_18889_gb300 import binding as B
    ws, refs, preps = circuits
    assert len({w.n_qubits for w in ws}) >= 3 and len({w.n_sliced for w in ws}) >= 2
    flags = B.TN_FLAG_HOIST_INVARIANT | (B.TN_FLAG_HILO_AUTO if prec == "bf16" else 0)
    plans = [E.Plan(p.tn, p.tree, prec=prec, flags=flags, max_slice_batch=0, mem_cap_bytes=8 << 30,
                    own_workspace=False, hilo_tol=tol)
             for p in preps]
    outs = [torch.empty((w.G, 1 << w.l), dtype=torch.complex128, device="cuda") for w in ws]
    ids = [np.arange(p.n_slices_total) for p in plans]
    _run_batched(E, plans, ids, outs)
    for w, o, ref in zip(ws, outs, refs):
        assert_amplitudes_close(o.cpu().numpy(), ref, tol, w.name)
    for p in plans:
        p.close()


def test_batched_graph_replay_and_branches(E, circuits):
    # the cached graph replays the same result; new slice ids are captured anew;
    # a workspace holding one region runs the plans on one branch, bit for bit
    import torch
    ws, refs, preps = circuits
    ws, refs, preps = ws[:6], refs[:6], preps[:6]
    plans = [E.Plan(p.tn, p.tree, prec="fp16", max_slice_batch=8, own_workspace=False) for p in preps]
    outs = [torch.empty((w.G, 1 << w.l), dtype=torch.complex128, device="cuda") for w in ws]
    ids = [np.arange(p.n_slices_total) for p in plans]
    _run_batched(E, plans, ids, outs)
    first = [o.cpu().numpy() for o in outs]
    for o in outs:
        o.fill_(float("nan"))
    _run_batched(E, plans, ids, outs)  # replay
    assert all(np.array_equal(a, o.cpu().numpy()) for a, o in zip(first, outs))
    half = [x[: max(1, len(x) // 2)] for x in ids]
    _run_batched(E, plans, half, outs)  # different slices: a new graph
    for p, h, o in zip(plans, half, outs):
        single = torch.empty_like(o)
        p.workspace = torch.empty(max(p.info["workspace_bytes"], 256), dtype=torch.uint8, device="cuda")
        p.contract(h, out=single)
        assert np.array_equal(single.cpu().numpy(), o.cpu().numpy())
    one_region = max(p.info["workspace_bytes"] for p in plans)
    _run_batched(E, plans, ids, outs, ws_bytes=(one_region + 255) // 256 * 256)
    assert all(np.array_equal(a, o.cpu().numpy()) for a, o in zip(first, outs))
    for w, o, ref in zip(ws, outs, refs):
        assert_amplitudes_close(o.cpu().numpy(), ref, 3e-3, w.name)
    for p in plans:
        p.close()
