"""The refined contraction tree of the 24-qubit, 14-cycle workload (greedy and
bisection trees re-optimised by subtree reconfiguration, six sliced bonds
chosen two at a time): the bench's default plan.  Its steps are skinnier than
the greedy tree's (batched 4096 x 4096 x 16 x 16, 2^23 x 4 x 4), which is where
the narrow-tile epilogue groups, 16-byte epilogue stores, row-paired
tensor-core steps and the small-K row kernel run.  All 64 slices against the
FP64 state vector, complex64 and fp16, and the fp16 selection's XEB."""
import os

import numpy as np
import pytest

from oracle import postprocess as pp
from oracle import statevector as sv
from parity_checks import assert_amplitudes_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def refined(sv_grid4x6):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_18889_gb300 import engine as E
    w, psi = sv_grid4x6
    prep = E.prepare(w, refine=True, method="both", workers=len(os.sched_getaffinity(0)))
    greedy = E.prepare(w)
    assert prep.tree.cost_per_slice < 0.2 * greedy.tree.cost_per_slice  # ~10x fewer MACs per sub-network
    assert len(prep.tree.sliced_edges) == 6
    ref, _ = sv.block_amplitudes(psi, w.n_qubits, w.open_qubits, w.closed_qubits, w.closed_bits)
    return E, w, psi, ref, prep


@pytest.mark.parametrize("prec,tol", [("c64", 1e-5), ("fp16", 3e-3)])
def test_refined_tree_against_statevector(refined, prec, tol):
    import torch
    from paper_2406_18889_gb300 import binding as B
    E, w, psi, ref, prep = refined
    plan = E.Plan(prep.tn, prep.tree, prec=prec, flags=B.TN_FLAG_HOIST_INVARIANT, max_slice_batch=64)
    kinds = plan.steps()["kinds"]
    if prec == "fp16":
        assert ((kinds & 8) > 0).sum() >= 4
        assert ((kinds & 256) > 0).sum() >= 1, "no row-paired tensor-core step"
    amps = plan.contract()
    B.tn_plan_status(plan.handle, torch.cuda.current_stream().cuda_stream)
    assert_amplitudes_close(amps.cpu().numpy(), ref, tol, f"refined tree, {prec}")
    base = torch.as_tensor(w.block_base(), device="cuda")
    idx, _ = E.topk(amps, w.k, 1.0, base, w.open_bit_pos())
    ri, _ = pp.topk_blocks(ref, w.k, 1.0, w.block_base(), w.open_bit_pos())
    x = pp.xeb(pp.ideal_probabilities_at(psi, idx.cpu().numpy()), w.n_qubits)
    x_ref = pp.xeb(pp.ideal_probabilities_at(psi, ri), w.n_qubits)
    assert abs(x - x_ref) <= 0.01 * abs(x_ref), (x, x_ref)
    plan.close()


def test_refined_tree_batches_agree(refined):
    # slice batch 16 (four batches) against batch 64: the same per-slice
    # amplitudes summed in FP64 in another grouping
    from paper_2406_18889_gb300 import binding as B
    E, w, psi, ref, prep = refined
    a = E.Plan(prep.tn, prep.tree, prec="fp16", flags=B.TN_FLAG_HOIST_INVARIANT, max_slice_batch=16)
    got = a.contract().cpu().numpy()
    assert_amplitudes_close(got, ref, 3e-3, "refined tree, fp16, batch 16")
    a.close()
