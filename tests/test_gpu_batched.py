"""Batched uneven circuits (64 seeded circuits, 4x4..4x7 grids, depth 10..16,
2^2..2^8 slices, l = 8, G = 16): a subset of up to 24 qubits is contracted in
one tn_contract_slices_batched call and each circuit is checked against its
own FP64 state vector."""
import numpy as np
import pytest

import workloads as W
from oracle import postprocess as pp
from parity_checks import assert_amplitudes_close
from oracle import statevector as sv

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


def _subset(max_qubits=24, count=6):
    ws = [w for w in W.configs.uneven_batch(64) if w.n_qubits <= max_qubits]
    return ws[:count]


@pytest.mark.parametrize("prec,tol", [("c64", 1e-5), ("fp16", 3e-3)])
def test_uneven_batch_against_statevectors(E, prec, tol):
    import torch
    from paper_2406_18889_gb300 import binding as B
    ws = _subset()
    assert len({w.n_qubits for w in ws}) >= 2 and len({w.n_sliced for w in ws}) >= 2
    preps = [E.prepare(w, restarts=1) for w in ws]
    plans = [E.Plan(p.tn, p.tree, prec=prec, max_slice_batch=16) for p in preps]
    outs = [torch.empty((w.G, 1 << w.l), dtype=torch.complex128, device="cuda") for w in ws]
    wsz = max(p.workspace.numel() for p in plans)
    wsb = torch.empty(wsz, dtype=torch.uint8, device="cuda")
    B.tn_contract_slices_batched([p.handle for p in plans], [np.arange(p.n_slices_total) for p in plans],
                                 [o.data_ptr() for o in outs], 0, wsb.data_ptr(), wsz,
                                 torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for w, o in zip(ws, outs):
        psi = sv.simulate(w.circuit)
        ref, _ = sv.block_amplitudes(psi, w.n_qubits, w.open_qubits, w.closed_qubits, w.closed_bits)
        assert_amplitudes_close(o.cpu().numpy(), ref, tol, w.name)
