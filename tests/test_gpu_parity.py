"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (complex64 path): relative L2 <= 1e-5 of amplitudes; top-k on the
same FP64 amplitudes bit-exact; XEB within 1e-12 relative of the oracle's.
"""
import numpy as np
import pytest

import workloads as W
from oracle import einsum_tn as et
from oracle import postprocess as pp
from parity_checks import assert_amplitudes_close
from oracle import statevector as sv

pytestmark = pytest.mark.gpu

C64_TOL = 1e-5


@pytest.fixture(scope="module")
def E():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_18889_gb300 import engine
    return engine


def _sv_blocks(w, psi=None):
    psi = sv.simulate(w.circuit) if psi is None else psi
    amps, _ = sv.block_amplitudes(psi, w.n_qubits, w.open_qubits, w.closed_qubits, w.closed_bits)
    return amps, psi


def _random_bonds(circuit, k, seed):
    rng = np.random.default_rng(seed)
    cands = [(q, t) for q in range(circuit.n_qubits) for t in range(1, circuit.n_ops_on(q))]
    pick = rng.choice(len(cands), size=k, replace=False)
    return [cands[i] for i in sorted(pick)]


def test_grid3x4_all_amplitudes(E):
    w = W.workload("grid3x4_d8")
    prep = E.prepare(w)
    plan = E.Plan(prep.tn, prep.tree, max_slice_batch=1)
    got = plan.contract().cpu().numpy()
    ref, _ = _sv_blocks(w)
    assert got.shape == (1, 4096)
    assert_amplitudes_close(got, ref, C64_TOL)


@pytest.mark.parametrize("batch", [64, 16])
def test_grid4x6_all_slices(E, sv_grid4x6, batch):
    w, psi = sv_grid4x6
    prep = E.prepare(w)
    assert len(prep.tree.sliced_edges) == 6
    plan = E.Plan(prep.tn, prep.tree, max_slice_batch=batch)
    got = plan.contract().cpu().numpy()
    ref, _ = _sv_blocks(w, psi)
    assert_amplitudes_close(got, ref, C64_TOL)


@pytest.mark.parametrize("prec,tol", [("c64", C64_TOL), ("fp16", 3e-3)])
def test_grid4x6_whole_state_vector(E, sv_grid4x6, prec, tol):
    """The 24-qubit, 14-cycle circuit with all 2^14 closed bitstrings as blocks:
    the 64 slices' blocks then hold every amplitude of the state vector."""
    import torch
    from paper_2406_18889_gb300 import binding as B
    w0, psi = sv_grid4x6
    w = W.workload("grid4x6_d14", G=1 << 14)
    assert all(a.qubits == b.qubits and np.array_equal(a.matrix, b.matrix)
               for a, b in zip(w.circuit.ops, w0.circuit.ops))
    prep = E.prepare(w)
    plan = E.Plan(prep.tn, prep.tree, prec=prec, flags=B.TN_FLAG_HOIST_INVARIANT, max_slice_batch=16)
    amps = plan.contract()
    got = amps.cpu().numpy()
    assert got.shape == (1 << 14, 1 << 10)
    ref, _ = _sv_blocks(w, psi)
    assert_amplitudes_close(got, ref, tol)
    # the blocks partition the state vector: total probability 1 (unit norm)
    assert abs(float(np.sum(np.abs(got) ** 2)) - 1.0) <= 2 * tol
    if prec == "c64":
        # global top-k over all 2^24 strings, bit-exact on the oracle's amplitudes
        base = torch.as_tensor(w.block_base(), device="cuda")
        gi, gp = E.topk(torch.as_tensor(ref, device="cuda"), 1000, 1.0, base, w.open_bit_pos(), global_mode=True)
        ri, rp = pp.topk_global(ref, 1000, 1.0, w.block_base(), w.open_bit_pos())
        assert np.array_equal(gi.cpu().numpy(), ri) and np.array_equal(gp.cpu().numpy(), rp)
        # and they are the 1000 most probable strings of the state vector itself
        q = pp.probabilities(psi.reshape(1, -1), 1.0).reshape(-1)
        assert np.array_equal(np.sort(ri), np.sort(np.argsort(-q, kind="stable")[:1000]))


@pytest.mark.parametrize("prec", ["c64", "fp16"])
def test_hoisted_invariant_subtrees(E, sv_grid4x6, prec):
    # slice-independent subtrees contracted once at plan creation give the same sum
    from paper_2406_18889_gb300 import binding as B
    w, psi = sv_grid4x6
    prep = E.prepare(w)
    plan = E.Plan(prep.tn, prep.tree, prec=prec, flags=B.TN_FLAG_HOIST_INVARIANT, max_slice_batch=32)
    kinds = plan.steps()["kinds"]
    assert ((kinds & 4) > 0).sum() > 0
    got = plan.contract().cpu().numpy()
    ref, _ = _sv_blocks(w, psi)
    assert_amplitudes_close(got, ref, C64_TOL if prec == "c64" else 3e-3)


@pytest.mark.parametrize("batch,n_run", [(8, 19), (4, 4), (16, 1)])
def test_partial_fraction_ragged_batches(E, batch, n_run):
    # f < 1: the sum over a seeded subset of sub-networks, against the oracle's own
    # sliced contraction of the same wire segments (slices run in ragged batches)
    w = W.workload("grid3x4_d8", cycles=10, l=5, G=8)
    bonds = _random_bonds(w.circuit, 5, seed=11)
    prep = E.prepare(w, sliced_wires=bonds)
    ids = W.draw_slice_subset(32, n_run, seed=5)
    plan = E.Plan(prep.tn, prep.tree, max_slice_batch=batch)
    got = plan.contract(ids).cpu().numpy()
    net = et.build_network(w.circuit, w.open_qubits, w.closed_qubits, w.closed_bits)
    ref = et.contract(net, bonds, ids)
    assert_amplitudes_close(got, ref, C64_TOL)


def test_accumulate_and_empty(E):
    torch = pytest.importorskip("torch")
    w = W.workload("grid3x4_d8", l=6, G=8)
    bonds = _random_bonds(w.circuit, 3, seed=4)
    prep = E.prepare(w, sliced_wires=bonds)
    plan = E.Plan(prep.tn, prep.tree, max_slice_batch=4)
    full = plan.contract().cpu().numpy()
    out = plan.contract([0, 1, 2])
    plan.contract([3, 4, 5, 6, 7], out=out, accumulate=True)
    assert_amplitudes_close(out.cpu().numpy(), full, C64_TOL)
    plan.contract([], out=out)  # zero slices, overwrite -> zeros
    assert torch.count_nonzero(out).item() == 0


def test_duplicate_slices_count_twice(E):
    w = W.workload("grid3x4_d8", l=6, G=8)
    bonds = _random_bonds(w.circuit, 3, seed=6)
    prep = E.prepare(w, sliced_wires=bonds)
    plan = E.Plan(prep.tn, prep.tree, max_slice_batch=4)
    one = plan.contract([5]).cpu().numpy()
    two = plan.contract([5, 5]).cpu().numpy()
    assert np.max(np.abs(two - 2 * one)) <= 1e-6 * np.max(np.abs(one))


def test_deterministic(E):
    w = W.workload("grid3x4_d8", cycles=10, l=6, G=8)
    prep = E.prepare(w, n_sliced=4)
    plan = E.Plan(prep.tn, prep.tree, max_slice_batch=8)
    a = plan.contract().cpu().numpy()
    b = plan.contract().cpu().numpy()
    assert np.array_equal(a, b)


def test_invalid_slice_rejected_before_work(E):
    torch = pytest.importorskip("torch")
    from paper_2406_18889_gb300.binding import TNError
    w = W.workload("grid3x4_d8", l=6, G=8)
    prep = E.prepare(w, n_sliced=2)
    plan = E.Plan(prep.tn, prep.tree, max_slice_batch=4)
    out = torch.full((8, 64), 7.0, dtype=torch.complex128, device="cuda")
    with pytest.raises(TNError):
        plan.contract([0, 4], out=out)  # 4 >= 2^2
    assert torch.all(out == 7.0).item()


def test_batched_plans_match_single(E):
    ws = [W.workload("grid3x4_d8", l=6, G=8, seed=s) for s in (1, 2, 3)]
    preps = [E.prepare(w, n_sliced=2 + i) for i, w in enumerate(ws)]
    plans = [E.Plan(p.tn, p.tree, max_slice_batch=4) for p in preps]
    singles = [p.contract().cpu().numpy() for p in plans]
    import torch
    from paper_2406_18889_gb300 import binding as B
    outs = [torch.empty((8, 64), dtype=torch.complex128, device="cuda") for _ in plans]
    wsz = max(p.workspace.numel() for p in plans)
    wsb = torch.empty(wsz, dtype=torch.uint8, device="cuda")
    B.tn_contract_slices_batched([p.handle for p in plans], [np.arange(p.n_slices_total) for p in plans],
                                 [o.data_ptr() for o in outs], 0, wsb.data_ptr(), wsz,
                                 torch.cuda.current_stream().cuda_stream)
    for o, s in zip(outs, singles):
        assert np.array_equal(o.cpu().numpy(), s)


# ------------------------------------------------------------------ post-processing
def test_topk_bit_exact_on_oracle_amplitudes(E, sv_grid4x6):
    import torch
    w, psi = sv_grid4x6
    amps, _ = _sv_blocks(w, psi)
    d = torch.as_tensor(amps, device="cuda")
    base = torch.as_tensor(w.block_base(), device="cuda")
    for inv_f in (1.0, 64.0 / 5.0):
        idx, p = E.topk(d, 64, inv_f, base, w.open_bit_pos())
        ri, rp = pp.topk_blocks(amps, 64, inv_f, w.block_base(), w.open_bit_pos())
        assert np.array_equal(idx.cpu().numpy(), ri)
        assert np.array_equal(p.cpu().numpy(), rp)
        gi, gp = E.topk(d, 200, inv_f, base, w.open_bit_pos(), global_mode=True)
        rgi, rgp = pp.topk_global(amps, 200, inv_f, w.block_base(), w.open_bit_pos())
        assert np.array_equal(gi.cpu().numpy(), rgi) and np.array_equal(gp.cpu().numpy(), rgp)


@pytest.mark.parametrize("seed", range(3))
def test_topk_ties_and_edges(E, seed):
    import torch
    rng = np.random.default_rng(seed)
    G, l = 5, 7
    vals = np.array([0.0, 0.125, -0.125, 0.25j, 0.5, -0.5j])
    amps = vals[rng.integers(0, len(vals), size=(G, 1 << l))]
    base = (np.sort(rng.choice(1 << 12, size=G, replace=False)).astype(np.int64)) << l
    pos = np.arange(l - 1, -1, -1)
    d = torch.as_tensor(amps, device="cuda")
    db = torch.as_tensor(base, device="cuda")
    for k in (1, 9, 128):
        idx, p = E.topk(d, k, 2.0, db, pos)
        ri, rp = pp.topk_blocks(amps, k, 2.0, base, pos)
        assert np.array_equal(idx.cpu().numpy(), ri) and np.array_equal(p.cpu().numpy(), rp)
    idx, p = E.topk(d, 512, 2.0, db, pos, global_mode=True)
    ri, rp = pp.topk_global(amps, 512, 2.0, base, pos)
    assert np.array_equal(idx.cpu().numpy(), ri) and np.array_equal(p.cpu().numpy(), rp)


def test_xeb_matches_oracle(E, sv_grid4x6):
    import torch
    w, psi = sv_grid4x6
    rng = np.random.default_rng(2)
    idx = rng.choice(1 << w.n_qubits, size=5000, replace=False)
    q = pp.ideal_probabilities_at(psi, idx)
    got = E.xeb(torch.as_tensor(q, device="cuda"), w.n_qubits)
    ref = pp.xeb(q, w.n_qubits)
    assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref))


def test_end_to_end_topk_and_xeb(E, sv_grid4x6):
    import torch
    w, psi = sv_grid4x6
    prep = E.prepare(w)
    plan = E.Plan(prep.tn, prep.tree, max_slice_batch=64)
    amps = plan.contract()
    base = torch.as_tensor(w.block_base(), device="cuda")
    idx, p = E.topk(amps, w.k, 1.0, base, w.open_bit_pos())
    ref_amps, _ = _sv_blocks(w, psi)
    ri, rp = pp.topk_blocks(ref_amps, w.k, 1.0, w.block_base(), w.open_bit_pos())
    gi = idx.cpu().numpy()
    # sets equal except where the oracle's p is within the amplitude tolerance of the k-th value
    tol = 2 * C64_TOL * rp.max()
    for g in range(w.G):
        diff = set(gi[g]) ^ set(ri[g])
        thresh = rp[g, -1]
        for s in diff:
            q = pp.ideal_probabilities_at(psi, np.array([s]))[0]
            assert abs(q - thresh) <= tol
    q_gpu = torch.as_tensor(pp.ideal_probabilities_at(psi, gi), device="cuda")
    x_gpu = E.xeb(q_gpu, w.n_qubits)
    x_ref = pp.xeb(pp.ideal_probabilities_at(psi, ri), w.n_qubits)
    assert abs(x_gpu - x_ref) <= 0.01 * abs(x_ref)
