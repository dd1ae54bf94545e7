"""O1: FP64 state-vector simulator (test infrastructure only).

The exact amplitude of bitstring s is <s|C|0^n>: start from |0^n> and apply
every gate of the circuit in order (paper Fig. 1: layers of random
single-qubit gates and two-qubit couplers).  Qubit 0 is the most significant
bit of the n-bit index, i.e. the state is a C-ordered array with axes
q0 ... q_{n-1}.

Each gate acts as psi'[.., o, ..] = sum_i U[o, i] psi[.., i, ..] on its
qubits' axes.  Two implementations of that one formula:

* ``apply_1q`` / ``apply_2q``: NumPy, the sum written out term by term over the
  gate's basis states on reshaped views (terms whose matrix entry is exactly
  zero add nothing and are skipped).  Slow but transparent; used for n <= 20.
* ``csrc/statevector.c``: the same sum as plain C loops over amplitude pairs or
  quadruples (OpenMP over independent groups), for 20 < n <= 30.

``simulate`` picks the C loops above 20 qubits; tests check that both agree.
"""
from __future__ import annotations

import ctypes
from typing import Iterable, Optional

import numpy as np


def zero_state(n: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def apply_1q(psi: np.ndarray, n: int, q: int, u: np.ndarray) -> np.ndarray:
    """psi' = (I x .. x U_q x .. x I) psi for a 2x2 U[out, in] on qubit q."""
    v = psi.reshape(1 << q, 2, 1 << (n - q - 1))
    out = np.zeros_like(v)
    for o in range(2):
        for i in range(2):
            if u[o, i] != 0:
                out[:, o, :] += u[o, i] * v[:, i, :]
    return out.reshape(-1)


def apply_2q(psi: np.ndarray, n: int, qa: int, qb: int, u: np.ndarray) -> np.ndarray:
    """Apply a 4x4 U[out, in] whose basis is |q_a q_b> (q_a most significant)."""
    lo, hi = min(qa, qb), max(qa, qb)
    v = psi.reshape(1 << lo, 2, 1 << (hi - lo - 1), 2, 1 << (n - hi - 1))
    out = np.zeros_like(v)

    def view(arr, bit_a, bit_b):
        b_lo, b_hi = (bit_a, bit_b) if qa == lo else (bit_b, bit_a)
        return arr[:, b_lo, :, b_hi, :]

    for oa in range(2):
        for ob in range(2):
            dst = view(out, oa, ob)
            for ia in range(2):
                for ib in range(2):
                    m = u[2 * oa + ob, 2 * ia + ib]
                    if m != 0:
                        dst += m * view(v, ia, ib)
    return out.reshape(-1)


def simulate_c(circuit) -> np.ndarray:
    """Full final state via the plain-C loops (same formula as apply_1q/apply_2q)."""
    from .build import load
    lib = load()
    n = circuit.n_qubits
    psi = np.empty(1 << n, dtype=np.complex128)
    dp = ctypes.POINTER(ctypes.c_double)
    ptr = psi.ctypes.data_as(dp)
    lib.sv_zero_state(ptr, n)
    for op in circuit.ops:
        u = np.ascontiguousarray(op.matrix, dtype=np.complex128)
        if len(op.qubits) == 1:
            lib.sv_apply_1q(ptr, n, op.qubits[0], u.ctypes.data_as(dp))
        elif len(op.qubits) == 2:
            lib.sv_apply_2q(ptr, n, op.qubits[0], op.qubits[1], u.ctypes.data_as(dp))
        else:
            raise ValueError("only 1- and 2-qubit gates")
    return psi


def simulate(circuit, check_norm_every: Optional[int] = None,
             backend: Optional[str] = None) -> np.ndarray:
    """Full final state of ``circuit`` as a complex128 vector of length 2^n."""
    n = circuit.n_qubits
    if backend is None:
        backend = "c" if n > 20 and not check_norm_every else "numpy"
    if backend == "c":
        return simulate_c(circuit)
    psi = zero_state(n)
    for k, op in enumerate(circuit.ops):
        if len(op.qubits) == 1:
            psi = apply_1q(psi, n, op.qubits[0], op.matrix)
        elif len(op.qubits) == 2:
            psi = apply_2q(psi, n, op.qubits[0], op.qubits[1], op.matrix)
        else:
            raise ValueError("only 1- and 2-qubit gates")
        if check_norm_every and (k + 1) % check_norm_every == 0:
            nrm = float(np.vdot(psi, psi).real)
            if abs(nrm - 1.0) > 1e-10:
                raise AssertionError(f"norm drifted to {nrm} after op {k}")
    return psi


def layer_norms(circuit) -> list:
    """||psi||^2 after every op (the state must stay normalised: unitary gates)."""
    n = circuit.n_qubits
    psi = zero_state(n)
    norms = []
    for op in circuit.ops:
        if len(op.qubits) == 1:
            psi = apply_1q(psi, n, op.qubits[0], op.matrix)
        else:
            psi = apply_2q(psi, n, op.qubits[0], op.qubits[1], op.matrix)
        norms.append(float(np.vdot(psi, psi).real))
    return norms


def block_amplitudes(psi: np.ndarray, n: int, open_qubits: Iterable[int],
                     closed_qubits: Iterable[int], closed_bits: np.ndarray) -> np.ndarray:
    """amps[g, j] = psi[s(g, j)]: block g fixes the closed qubits to closed_bits[g];
    j runs over the open qubits' values, first open qubit = most significant bit of j
    (paper Sec. III: groups of 2^l correlated bitstrings)."""
    open_qubits = list(open_qubits)
    closed_qubits = list(closed_qubits)
    l = len(open_qubits)
    G = closed_bits.shape[0]
    j = np.arange(1 << l, dtype=np.int64)
    open_part = np.zeros(1 << l, dtype=np.int64)
    for i, q in enumerate(open_qubits):
        open_part |= ((j >> (l - 1 - i)) & 1) << (n - 1 - q)
    base = np.zeros(G, dtype=np.int64)
    for c, q in enumerate(closed_qubits):
        base |= closed_bits[:, c].astype(np.int64) << (n - 1 - q)
    idx = base[:, None] | open_part[None, :]
    return psi[idx], idx
