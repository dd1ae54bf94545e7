"""Reduced-precision path (fp16 / bf16 tensor cores, FP32 accumulate, per-tensor
power-of-two exponents, optional hi+lo split) against the FP64 oracle.

Bars: relative L2 of the amplitudes <= 3e-3 (fp16; bf16 with hi+lo), and the
XEB of the per-block top-k selection within 1% of the oracle's selection (all
reduced-precision variants, plain bf16 included; its amplitude error is only
held to a loose 2e-2 and reported).
"""
import numpy as np
import pytest

import workloads as W
from oracle import einsum_tn as et
from oracle import postprocess as pp
from parity_checks import assert_amplitudes_close
from oracle import statevector as sv

pytestmark = pytest.mark.gpu

LOWP_TOL = 3e-3


@pytest.fixture(scope="module")
def E():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_18889_gb300 import engine
    return engine


@pytest.fixture(scope="module")
def grid(E, sv_grid4x6):
    w, psi = sv_grid4x6
    ref, _ = sv.block_amplitudes(psi, w.n_qubits, w.open_qubits, w.closed_qubits, w.closed_bits)
    ri, _ = pp.topk_blocks(ref, w.k, 1.0, w.block_base(), w.open_bit_pos())
    x_ref = pp.xeb(pp.ideal_probabilities_at(psi, ri), w.n_qubits)
    return w, psi, ref, x_ref, E.prepare(w)


CASES = [("fp16", 0, LOWP_TOL), ("bf16", 8, LOWP_TOL), ("fp16", 8, LOWP_TOL), ("bf16", 0, 2e-2)]


@pytest.mark.parametrize("prec,flags,tol", CASES, ids=[f"{p}{'+hilo' if f else ''}" for p, f, _ in CASES])
def test_reduced_precision_amplitudes_and_xeb(E, grid, prec, flags, tol):
    import torch
    from paper_2406_18889_gb300 import binding as B
    w, psi, ref, x_ref, prep = grid
    plan = E.Plan(prep.tn, prep.tree, prec=prec, flags=flags, max_slice_batch=64)
    st = plan.steps()
    assert ((st["kinds"] & 8) > 0).sum() >= 1, "no step ran on the tensor cores"
    amps = plan.contract()
    B.tn_plan_status(plan.handle, torch.cuda.current_stream().cuda_stream)
    got = amps.cpu().numpy()
    assert_amplitudes_close(got, ref, tol, f"{prec} flags {flags}")
    base = torch.as_tensor(w.block_base(), device="cuda")
    idx, _ = E.topk(amps, w.k, 1.0, base, w.open_bit_pos())
    x = pp.xeb(pp.ideal_probabilities_at(psi, idx.cpu().numpy()), w.n_qubits)
    assert abs(x - x_ref) <= 0.01 * abs(x_ref), (x, x_ref)
    plan.close()


def test_reduced_precision_partial_fraction(E):
    # a seeded subset of slices in fp16 with seeded sliced wire segments, against the
    # oracle's own sliced contraction of the same segments
    w = W.workload("grid4x6_d14", cols=5, cycles=10, l=8, G=16)
    rng = np.random.default_rng(21)
    cands = [(q, t) for q in range(w.n_qubits) for t in range(1, w.circuit.n_ops_on(q))]
    bonds = [cands[i] for i in sorted(rng.choice(len(cands), size=5, replace=False))]
    prep = E.prepare(w, sliced_wires=bonds)
    ids = W.draw_slice_subset(32, 12, seed=9)
    plan = E.Plan(prep.tn, prep.tree, prec="fp16", max_slice_batch=8)
    got = plan.contract(ids).cpu().numpy()
    net = et.build_network(w.circuit, w.open_qubits, w.closed_qubits, w.closed_bits)
    ref = et.contract(net, bonds, ids)
    assert_amplitudes_close(got, ref, LOWP_TOL)


def test_reduced_precision_deterministic(E, grid):
    w, psi, ref, x_ref, prep = grid
    plan = E.Plan(prep.tn, prep.tree, prec="fp16", max_slice_batch=32)
    a = plan.contract().cpu().numpy()
    b = plan.contract().cpu().numpy()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("prec,flags,tol", [
    ("fp16", "hilo", 2e-5), ("bf16", "hilo", 3e-5), ("fp16", "hilo+fine", 1e-5)],
    ids=["fp16+hilo", "bf16+hilo", "fp16+hilo+fine"])
def test_chunked_accumulation_accuracy(E, grid, prec, flags, tol):
    # the tensor cores' own accumulation error grows with K; split products
    # accumulate K in chunks summed in FP32 registers (4 k tiles, or 1 with
    # TN_FLAG_FINE_ACC, which meets the complex64 bar of 1e-5)
    from paper_2406_18889_gb300 import binding as B
    w, psi, ref, x_ref, prep = grid
    f = B.TN_FLAG_HILO | (B.TN_FLAG_FINE_ACC if "fine" in flags else 0)
    plan = E.Plan(prep.tn, prep.tree, prec=prec, flags=f | B.TN_FLAG_HOIST_INVARIANT, max_slice_batch=64)
    got = plan.contract().cpu().numpy()
    assert_amplitudes_close(got, ref, tol, f"{prec} {flags}")


def test_hilo_auto_places_split_products_by_calibration(E, grid):
    # bf16 misses 3e-3 without any split product; TN_FLAG_HILO_AUTO splits only
    # the tensor-core steps with the largest share of the calibration error
    import torch
    from paper_2406_18889_gb300 import binding as B
    w, psi, ref, x_ref, prep = grid
    plan = E.Plan(prep.tn, prep.tree, prec="bf16", flags=B.TN_FLAG_HILO_AUTO | B.TN_FLAG_HOIST_INVARIANT,
                  max_slice_batch=64, hilo_tol=LOWP_TOL)
    pr = plan.precision()
    assert pr["rel_l2_none"] > LOWP_TOL and pr["rel_l2_chosen"] <= LOWP_TOL, pr
    assert 1 <= pr["n_hilo_steps"] < pr["n_tc_steps"], pr
    kinds = plan.steps()["kinds"]
    assert ((kinds & 16) > 0).sum() == pr["n_hilo_steps"]
    amps = plan.contract()
    assert_amplitudes_close(amps.cpu().numpy(), ref, LOWP_TOL, "bf16 auto hi+lo")
    base = torch.as_tensor(w.block_base(), device="cuda")
    idx, _ = E.topk(amps, w.k, 1.0, base, w.open_bit_pos())
    x = pp.xeb(pp.ideal_probabilities_at(psi, idx.cpu().numpy()), w.n_qubits)
    assert abs(x - x_ref) <= 0.01 * abs(x_ref), (x, x_ref)
    # the same placement given explicitly reproduces the plan bit for bit
    mask = ((kinds & 16) > 0).astype(np.uint8)
    plan2 = E.Plan(prep.tn, prep.tree, prec="bf16", flags=B.TN_FLAG_HOIST_INVARIANT, max_slice_batch=64,
                   hilo_steps=mask)
    assert np.array_equal(plan2.contract().cpu().numpy(), amps.cpu().numpy())
    plan.close()
    plan2.close()


def test_slice_batch_from_free_memory(E, grid):
    # max_slice_batch = 0: the library picks the batch from the device's free memory
    w, psi, ref, x_ref, prep = grid
    plan = E.Plan(prep.tn, prep.tree, prec="fp16", max_slice_batch=0)
    assert plan.max_slice_batch == 64  # all 64 slices fit a GB300 at once
    assert_amplitudes_close(plan.contract().cpu().numpy(), ref, LOWP_TOL)
    plan.close()
