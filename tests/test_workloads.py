"""Pins for the seeded input generator: gate matrices and circuit structure."""
import numpy as np
import pytest

import workloads as W


def _phase_equal(a, b, tol=1e-14):
    """a == e^{i t} b for some global phase t."""
    k = np.argmax(np.abs(b))
    ph = a.flat[k] / b.flat[k]
    return abs(abs(ph) - 1) < tol and np.max(np.abs(a - ph * b)) < tol


X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)


@pytest.mark.parametrize("u", list(W.ONE_QUBIT_GATES) + [W.fsim(np.pi / 2, np.pi / 6)])
def test_gates_unitary(u):
    eye = np.eye(u.shape[0])
    assert np.max(np.abs(u.conj().T @ u - eye)) <= 1e-14


def test_square_roots():
    # sqrt(X)^2 = X, sqrt(Y)^2 = Y, sqrt(W)^2 = W up to a global phase
    Wm = (X + Y) / np.sqrt(2)
    assert _phase_equal(W.SQRT_X @ W.SQRT_X, X)
    assert _phase_equal(W.SQRT_Y @ W.SQRT_Y, Y)
    assert _phase_equal(W.SQRT_W @ W.SQRT_W, Wm)


def test_fsim_special_cases():
    assert np.allclose(W.fsim(0.0, 0.0), np.eye(4), atol=1e-15)
    f = W.fsim(np.pi / 2, np.pi / 6)
    # |01> -> -i |10>, |10> -> -i |01>, |11> -> e^{-i pi/6} |11>
    e01 = np.zeros(4); e01[1] = 1
    out = f @ e01
    assert abs(out[2] + 1j) < 1e-15 and abs(out[1]) < 1e-15
    assert abs(f[3, 3] - np.exp(-1j * np.pi / 6)) < 1e-15
    # symmetric under exchanging the two qubits
    swap = np.eye(4)[[0, 2, 1, 3]]
    assert np.allclose(swap @ f @ swap, f, atol=1e-15)


@pytest.mark.parametrize("rows,cols", [(3, 4), (4, 6), (4, 7), (5, 6)])
def test_rect_patterns_are_matchings_covering_grid(rows, cols):
    pat = W.rect_couplers(rows, cols)
    all_edges = set()
    for letter, edges in pat.items():
        qs = [q for e in edges for q in e]
        assert len(qs) == len(set(qs)), f"pattern {letter} is not a matching"
        all_edges |= {tuple(sorted(e)) for e in edges}
    grid = set()
    for r in range(rows):
        for c in range(cols):
            q = r * cols + c
            if c + 1 < cols:
                grid.add((q, q + 1))
            if r + 1 < rows:
                grid.add((q, q + cols))
    assert all_edges == grid


def test_diag_grid_53_qubits():
    n, pat = W.diag_couplers()
    assert n == 53
    for letter, edges in pat.items():
        qs = [q for e in edges for q in e]
        assert len(qs) == len(set(qs))
    degree = np.zeros(n, dtype=int)
    for edges in pat.values():
        for a, b in edges:
            degree[a] += 1
            degree[b] += 1
    assert degree.max() <= 4 and degree.min() >= 1


def test_circuit_gate_rule_and_counts():
    c = W.grid_circuit(4, 6, 14, seed=7)
    n = 24
    oneq = [op for op in c.ops if len(op.qubits) == 1]
    assert len(oneq) == n * 15  # 14 cycles + final layer
    per_q = {q: [op.name for op in oneq if op.qubits[0] == q] for q in range(n)}
    for q, names in per_q.items():
        assert all(a != b for a, b in zip(names, names[1:])), "same gate twice in a row"
    pat = W.rect_couplers(4, 6)
    twoq = [op for op in c.ops if len(op.qubits) == 2]
    expected = sum(len(pat[W.PATTERN_ORDER[i % 8]]) for i in range(14))
    assert len(twoq) == expected
    # deterministic in the seed
    c2 = W.grid_circuit(4, 6, 14, seed=7)
    assert [op.name for op in c.ops] == [op.name for op in c2.ops]


def test_closed_bitstrings_distinct_and_seeded():
    b = W.draw_closed_bitstrings(14, 64, seed=3)
    assert b.shape == (64, 14)
    assert len({r.tobytes() for r in b}) == 64
    assert np.array_equal(b, W.draw_closed_bitstrings(14, 64, seed=3))
    with pytest.raises(ValueError):
        W.draw_closed_bitstrings(3, 9, seed=0)


def test_block_base_and_open_positions():
    w = W.workload("grid4x6_d14")
    base = w.block_base()
    pos = w.open_bit_pos()
    assert list(pos) == list(range(9, -1, -1))  # open qubits 14..23 -> bits 9..0
    assert np.all(base & ((1 << 10) - 1) == 0)
    # closed qubit 0 is the MSB
    assert np.array_equal((base >> 23) & 1, w.closed_bits[:, 0])


def test_slice_subset():
    s = W.draw_slice_subset(64, 16, seed=1)
    assert len(set(s.tolist())) == 16 and s.min() >= 0 and s.max() < 64
    assert list(s) == sorted(s)


def test_uneven_batch_shapes():
    ws = W.configs.uneven_batch(8)
    for w in ws:
        assert 16 <= w.n_qubits <= 28 and w.l == 8 and w.G == 16
        assert 2 <= w.n_sliced <= 8 and 10 <= w.circuit.cycles <= 16

