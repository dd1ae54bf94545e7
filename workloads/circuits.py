"""Seeded synthetic random-circuit workloads (inputs only).

This module produces the *inputs* that both the FP64 oracle and the GPU path
consume: the gate list of a 2D-grid random circuit, the closed-qubit
bitstrings of each correlated block, and seeded subsets of slice ids.  It holds
none of the method's arithmetic (no contraction, no probabilities, no XEB).

Circuit family (paper, Fig. 1 and Sec. I): cycles of random single-qubit gates
drawn from {sqrt(X), sqrt(Y), sqrt(W)} followed by two-qubit fSim couplers on
one of the coupler patterns A/B/C/D, in the order ABCDCDAB.  The paper names
the single-qubit gate set only; the readings taken for the matrices, the draw
rule, the coupler patterns and the bit order are:

* sqrt(X) = [[1,-i],[-i,1]]/sqrt2, sqrt(Y) = [[1,-1],[1,1]]/sqrt2,
  sqrt(W) = [[1,-sqrt(i)],[sqrt(-i),1]]/sqrt2 with W = (X+Y)/sqrt2.
* fSim(theta, phi) on |q_a q_b> = diag-block [[1,0,0,0],[0,c,-is,0],[0,-is,c,0],
  [0,0,0,e^{-i phi}]] with c = cos(theta), s = sin(theta); theta = pi/2,
  phi = pi/6.  The matrix is symmetric under exchanging q_a and q_b.
* First layer: uniform over the three gates.  Every later layer: uniform over
  the two gates that differ from the previous gate on that qubit.  Draws are
  cycle-major, qubits ascending, from numpy's PCG64.  One final single-qubit
  layer follows the last cycle.
* Rectangular R x C grid, qubit q = r*C + c.  A = horizontal couplers
  (r,c)-(r,c+1) with r+c even, B = horizontal with r+c odd, C = vertical
  (r,c)-(r+1,c) with r+c even, D = vertical with r+c odd.
* Diagonal (Sycamore-shaped) grid: rows i of 6 sites; site (i,j) couples
  "down-right" to (i+1, j + (i odd)) and "down-left" to (i+1, j - (i even)).
  A/B = down-right from even/odd rows, C/D = down-left from even/odd rows.
  One corner site is removed to reach 53 qubits.
* Qubit 0 is the most significant bit of an n-bit index.

Ops are stored as (qubits, matrix) with matrix[out, in] in the computational
basis of the listed qubits, first listed qubit = most significant.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

PATTERN_ORDER = "ABCDCDAB"

_S2 = 1.0 / np.sqrt(2.0)
SQRT_X = _S2 * np.array([[1, -1j], [-1j, 1]], dtype=np.complex128)
SQRT_Y = _S2 * np.array([[1, -1], [1, 1]], dtype=np.complex128)
SQRT_W = _S2 * np.array(
    [[1, -np.exp(1j * np.pi / 4)], [np.exp(-1j * np.pi / 4), 1]], dtype=np.complex128
)
ONE_QUBIT_GATES = (SQRT_X, SQRT_Y, SQRT_W)
ONE_QUBIT_NAMES = ("sqrtX", "sqrtY", "sqrtW")


def fsim(theta: float, phi: float) -> np.ndarray:
    """fSim(theta, phi) as a 4x4 matrix on |q_a q_b> (q_a most significant)."""
    c, s = np.cos(theta), np.sin(theta)
    m = np.zeros((4, 4), dtype=np.complex128)
    m[0, 0] = 1.0
    m[1, 1] = c
    m[1, 2] = -1j * s
    m[2, 1] = -1j * s
    m[2, 2] = c
    m[3, 3] = np.exp(-1j * phi)
    return m


@dataclass
class Op:
    qubits: Tuple[int, ...]
    matrix: np.ndarray  # [2^len(qubits), 2^len(qubits)], [out, in]
    name: str


@dataclass
class Circuit:
    n_qubits: int
    cycles: int
    layout: str  # "rect RxC" or "diag"
    ops: List[Op] = field(default_factory=list)
    couplers: dict = field(default_factory=dict)  # pattern letter -> list of (a, b)

    def n_ops_on(self, q: int) -> int:
        return sum(1 for op in self.ops if q in op.qubits)


def rect_couplers(rows: int, cols: int) -> dict:
    """Coupler patterns A/B/C/D of a rectangular grid (each pattern a matching)."""
    pat = {k: [] for k in "ABCD"}
    for r in range(rows):
        for c in range(cols):
            q = r * cols + c
            if c + 1 < cols:
                pat["A" if (r + c) % 2 == 0 else "B"].append((q, q + 1))
            if r + 1 < rows:
                pat["C" if (r + c) % 2 == 0 else "D"].append((q, q + cols))
    return pat


def diag_couplers(rows: int = 9, cols: int = 6, removed: Tuple[int, int] = (0, 0)):
    """Coupler patterns of a diagonal-coupler grid; returns (n_qubits, patterns)."""
    sites = [(i, j) for i in range(rows) for j in range(cols) if (i, j) != removed]
    index = {s: k for k, s in enumerate(sites)}
    pat = {k: [] for k in "ABCD"}
    for (i, j) in sites:
        dr = (i + 1, j + (1 if i % 2 == 1 else 0))
        dl = (i + 1, j - (1 if i % 2 == 0 else 0))
        if dr in index:
            pat["A" if i % 2 == 0 else "B"].append((index[(i, j)], index[dr]))
        if dl in index:
            pat["C" if i % 2 == 0 else "D"].append((index[(i, j)], index[dl]))
    return len(sites), pat


def _one_qubit_layer(rng: np.random.Generator, prev: List[int]) -> List[int]:
    out = []
    for p in prev:
        if p < 0:
            out.append(int(rng.integers(0, 3)))
        else:
            others = [g for g in range(3) if g != p]
            out.append(others[int(rng.integers(0, 2))])
    return out


def make_circuit(n_qubits: int, patterns: dict, cycles: int, seed: int, layout: str,
                 theta: float = np.pi / 2, phi: float = np.pi / 6,
                 final_layer: bool = True) -> Circuit:
    rng = np.random.Generator(np.random.PCG64(seed))
    circ = Circuit(n_qubits=n_qubits, cycles=cycles, layout=layout, couplers=patterns)
    two_q = fsim(theta, phi)
    prev = [-1] * n_qubits
    layers = cycles + (1 if final_layer else 0)
    for cyc in range(layers):
        prev = _one_qubit_layer(rng, prev)
        for q, g in enumerate(prev):
            circ.ops.append(Op((q,), ONE_QUBIT_GATES[g].copy(), ONE_QUBIT_NAMES[g]))
        if cyc < cycles:
            letter = PATTERN_ORDER[cyc % len(PATTERN_ORDER)]
            for (a, b) in patterns[letter]:
                circ.ops.append(Op((a, b), two_q.copy(), "fsim"))
    return circ


def grid_circuit(rows: int, cols: int, cycles: int, seed: int, **kw) -> Circuit:
    return make_circuit(rows * cols, rect_couplers(rows, cols), cycles, seed,
                        f"rect {rows}x{cols}", **kw)


def sycamore_like_circuit(cycles: int, seed: int, **kw) -> Circuit:
    n, pat = diag_couplers()
    return make_circuit(n, pat, cycles, seed, "diag 9x6-1", **kw)


def open_qubits_default(n_qubits: int, l: int) -> List[int]:
    """The last l qubits in row-major order (a corner patch), ascending."""
    return list(range(n_qubits - l, n_qubits))


def draw_closed_bitstrings(n_closed: int, G: int, seed: int) -> np.ndarray:
    """G distinct uniformly drawn closed-qubit bitstrings, [G, n_closed] uint8.

    Bits are listed for the closed qubits in ascending qubit order.  Distinct
    draws avoid double-counting a bitstring in top-k and XEB.
    """
    if n_closed == 0:
        if G != 1:
            raise ValueError("with no closed qubits there is exactly one block")
        return np.zeros((1, 0), dtype=np.uint8)
    if n_closed < 63 and G > (1 << n_closed):
        raise ValueError("more blocks than distinct closed bitstrings")
    rng = np.random.Generator(np.random.PCG64(seed))
    seen = set()
    rows = []
    while len(rows) < G:
        bits = rng.integers(0, 2, size=n_closed, dtype=np.uint8)
        key = bits.tobytes()
        if key in seen:
            continue
        seen.add(key)
        rows.append(bits)
    return np.stack(rows)


def draw_slice_subset(n_total: int, n_run: int, seed: int) -> np.ndarray:
    """A seeded subset of n_run distinct slice ids out of n_total, ascending int64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ids = rng.choice(n_total, size=n_run, replace=False)
    return np.sort(ids.astype(np.int64))


def block_base_index(closed_qubits: Sequence[int], closed_bits: np.ndarray,
                     n_qubits: int) -> np.ndarray:
    """n-bit index (qubit 0 = MSB) of each block with all open bits zero, int64 [G]."""
    base = np.zeros(closed_bits.shape[0], dtype=np.int64)
    for col, q in enumerate(closed_qubits):
        base |= closed_bits[:, col].astype(np.int64) << np.int64(n_qubits - 1 - q)
    return base


def open_bit_positions(open_qubits: Sequence[int], n_qubits: int) -> np.ndarray:
    """Bit position (0 = LSB of the n-bit index) of each open qubit, int64 [l]."""
    return np.array([n_qubits - 1 - q for q in open_qubits], dtype=np.int64)
