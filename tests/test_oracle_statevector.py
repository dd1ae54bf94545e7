"""Pins for oracle O1 (state vector): brute force, closed forms, invariants."""
import copy

import numpy as np
import pytest

import workloads as W
from oracle import statevector as sv
from oracle import postprocess as pp


def _full_operator(op, n):
    """Brute-force 2^n x 2^n matrix of one gate: U on its qubits, identity elsewhere."""
    N = 1 << n
    U = np.zeros((N, N), dtype=complex)
    qs = op.qubits
    others = [q for q in range(n) if q not in qs]
    bit = lambda x, q: (x >> (n - 1 - q)) & 1  # noqa: E731
    for x in range(N):
        for y in range(N):
            if any(bit(x, q) != bit(y, q) for q in others):
                continue
            o = 0
            i = 0
            for q in qs:
                o = 2 * o + bit(x, q)
                i = 2 * i + bit(y, q)
            U[x, y] = op.matrix[o, i]
    return U


@pytest.mark.parametrize("rows,cols,cycles,seed", [(1, 2, 3, 1), (2, 2, 4, 2), (1, 4, 5, 3)])
def test_matches_brute_force_unitary(rows, cols, cycles, seed):
    c = W.grid_circuit(rows, cols, cycles, seed)
    n = c.n_qubits
    psi_ref = np.zeros(1 << n, dtype=complex)
    psi_ref[0] = 1
    for op in c.ops:
        psi_ref = _full_operator(op, n) @ psi_ref
    assert np.max(np.abs(sv.simulate(c, backend="numpy") - psi_ref)) < 1e-13
    assert np.max(np.abs(sv.simulate(c, backend="c") - psi_ref)) < 1e-13


def test_two_qubit_gate_on_reversed_qubits():
    # a non-symmetric 4x4 on (q_a, q_b) = (2, 0) against brute force
    rng = np.random.default_rng(0)
    m = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
    c = W.Circuit(n_qubits=3, cycles=0, layout="test")
    c.ops = [W.Op((0,), W.SQRT_X, "x"), W.Op((1,), W.SQRT_Y, "y"), W.Op((2, 0), m, "m")]
    psi_ref = np.zeros(8, dtype=complex)
    psi_ref[0] = 1
    for op in c.ops:
        psi_ref = _full_operator(op, 3) @ psi_ref
    assert np.max(np.abs(sv.simulate(c, backend="numpy") - psi_ref)) < 1e-13
    assert np.max(np.abs(sv.simulate(c, backend="c") - psi_ref)) < 1e-13


def test_product_state_closed_form():
    # single-qubit gates only: the state is the Kronecker product of U_q |0>
    c = W.grid_circuit(2, 3, 6, seed=5)
    c.ops = [op for op in c.ops if len(op.qubits) == 1]
    per_q = [np.array([1, 0], dtype=complex) for _ in range(6)]
    for op in c.ops:
        q = op.qubits[0]
        per_q[q] = op.matrix @ per_q[q]
    ref = per_q[0]
    for v in per_q[1:]:
        ref = np.kron(ref, v)
    assert np.max(np.abs(sv.simulate(c) - ref)) < 1e-14


def test_norm_preserved_every_op():
    w = W.workload("grid3x4_d8")
    norms = sv.layer_norms(w.circuit)
    assert max(abs(x - 1) for x in norms) < 1e-12


def test_c_and_numpy_agree_medium():
    c = W.grid_circuit(3, 5, 10, seed=11)
    a = sv.simulate(c, backend="numpy")
    b = sv.simulate(c, backend="c")
    assert pp.relative_l2(b, a) < 1e-13


def test_block_amplitudes_index_layout():
    c = W.grid_circuit(2, 3, 4, seed=9)
    psi = sv.simulate(c)
    opens, closed = [3, 5], [0, 1, 2, 4]
    bits = np.array([[1, 0, 1, 1], [0, 1, 1, 0]], dtype=np.uint8)
    amps, idx = sv.block_amplitudes(psi, 6, opens, closed, bits)
    # block 0, j = 0b10: open qubit 3 = 1, qubit 5 = 0; closed 0,1,2,4 = 1,0,1,1
    # bits q0..q5 = 1 0 1 1 1 0 -> 0b101110
    assert idx[0, 2] == 0b101110
    assert amps[0, 2] == psi[0b101110]


def test_porter_thomas_deep_circuit(sv_grid4x6):
    w, psi = sv_grid4x6
    N = 1 << w.n_qubits
    x = N * (psi.real ** 2 + psi.imag ** 2)
    assert abs(x.mean() - 1.0) < 1e-9  # norm
    assert abs((x ** 2).mean() - 2.0) < 0.1  # Haar value 2N/(N+1)
    from scipy import stats
    ks = stats.kstest(x[:: 16], "expon").statistic
    assert ks < 0.01
