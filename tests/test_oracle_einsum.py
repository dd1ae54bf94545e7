"""Pins for oracle O2 (naive tensor-network contractor with slicing)."""
import copy

import numpy as np
import pytest

import workloads as W
from oracle import einsum_tn as et
from oracle import statevector as sv
from oracle import postprocess as pp


def _with_projectors(circuit, fixes):
    """Circuit with |v><v| inserted on qubit q after its t-th operation for every
    (q, t, v) in ``fixes``: the state-vector meaning of fixing that wire segment."""
    c = copy.deepcopy(circuit)
    count = [0] * c.n_qubits
    ops = []
    pending = {(q, t): v for (q, t, v) in fixes}

    def emit_after(q):
        key = (q, count[q])
        if key in pending:
            p = np.zeros((2, 2), dtype=complex)
            p[pending[key], pending[key]] = 1
            ops.append(W.Op((q,), p, "proj"))

    for q in range(c.n_qubits):
        emit_after(q)
    for op in c.ops:
        ops.append(op)
        for q in op.qubits:
            count[q] += 1
            emit_after(q)
    c.ops = ops
    return c


def _sv_blocks(w, circuit=None):
    psi = sv.simulate(circuit or w.circuit, backend="numpy")
    amps, _ = sv.block_amplitudes(psi, w.n_qubits, w.open_qubits, w.closed_qubits, w.closed_bits)
    return amps


@pytest.mark.parametrize("l,G", [(12, 1), (6, 8), (3, 16)])
def test_unsliced_matches_statevector(l, G):
    w = W.workload("grid3x4_d8", l=l, G=G)
    net = et.build_network(w.circuit, w.open_qubits, w.closed_qubits, w.closed_bits)
    assert pp.relative_l2(et.contract(net), _sv_blocks(w)) < 1e-12


def _some_bonds(circuit, k, seed):
    """k distinct internal wire segments (q, t) with 1 <= t < #ops on q."""
    rng = np.random.default_rng(seed)
    cands = [(q, t) for q in range(circuit.n_qubits) for t in range(1, circuit.n_ops_on(q))]
    pick = rng.choice(len(cands), size=k, replace=False)
    return [cands[i] for i in sorted(pick)]


def test_sliced_sum_equals_unsliced():
    # slicing identity: the network is the sum of its sub-networks over all assignments
    w = W.workload("grid3x4_d8", l=6, G=8)
    net = et.build_network(w.circuit, w.open_qubits, w.closed_qubits, w.closed_bits)
    bonds = _some_bonds(w.circuit, 4, seed=1)
    full = et.contract(net)
    sliced = et.contract(net, bonds)
    assert pp.relative_l2(sliced, full) < 1e-12
    assert pp.relative_l2(sliced, _sv_blocks(w)) < 1e-12


def test_each_slice_is_projected_statevector():
    # sub-network sigma = circuit with projectors |v_i><v_i| on the sliced wire segments
    w = W.workload("grid3x4_d8", l=5, G=4)
    net = et.build_network(w.circuit, w.open_qubits, w.closed_qubits, w.closed_bits)
    bonds = _some_bonds(w.circuit, 3, seed=2)
    per = et.contract_each_slice(net, bonds, [0, 3, 5, 6])
    for row, sigma in zip(per, [0, 3, 5, 6]):
        fixes = [(q, t, (sigma >> i) & 1) for i, (q, t) in enumerate(bonds)]
        ref = _sv_blocks(w, _with_projectors(w.circuit, fixes))
        assert np.max(np.abs(row - ref)) < 1e-13


def test_partial_fraction_is_sum_of_chosen_slices():
    w = W.workload("grid3x4_d8", l=6, G=8)
    net = et.build_network(w.circuit, w.open_qubits, w.closed_qubits, w.closed_bits)
    bonds = _some_bonds(w.circuit, 3, seed=3)
    chosen = [1, 4, 6]
    partial = et.contract(net, bonds, chosen)
    ref = 0
    for sigma in chosen:
        fixes = [(q, t, (sigma >> i) & 1) for i, (q, t) in enumerate(bonds)]
        ref = ref + _sv_blocks(w, _with_projectors(w.circuit, fixes))
    assert np.max(np.abs(partial - ref)) < 1e-13


def test_rejects_bad_slices():
    w = W.workload("grid3x4_d8", l=6, G=8)
    net = et.build_network(w.circuit, w.open_qubits, w.closed_qubits, w.closed_bits)
    last = w.circuit.n_ops_on(0)
    with pytest.raises(ValueError):
        et.contract(net, [(w.open_qubits[0], w.circuit.n_ops_on(w.open_qubits[0]))])  # output leg
    with pytest.raises(ValueError):
        et.contract(net, [(0, 1)], [2])  # slice id out of range
    assert last > 1


def test_pair_contract_hyperindex_kept():
    # C[g, a, c] = sum_b A[g, a, b] B[g, b, c] with g shared and kept
    rng = np.random.default_rng(0)
    A = rng.normal(size=(3, 2, 4)) + 0j
    B = rng.normal(size=(3, 4, 5)) + 0j
    dims = {"g": 3, "a": 2, "b": 4, "c": 5}
    C, lc = et.pair_contract(A, ("g", "a", "b"), B, ("g", "b", "c"), keep={"g", "a", "c"}, dims=dims)
    ref = np.einsum("gab,gbc->gac", A, B)
    assert lc == ("g", "a", "c") and np.allclose(C, ref, atol=1e-14)
