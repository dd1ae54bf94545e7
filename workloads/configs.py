"""The synthetic workloads: grids, depths, open qubits, blocks, slices and k.

Each workload is fully determined by its seed.  Workload i uses seed
2406188890 + i; circuit j of the uneven batch uses that seed + 100*j.  The
circuit, the closed bitstrings and any slice subset draw from independent
child streams of the seed.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from .circuits import (Circuit, draw_closed_bitstrings, grid_circuit, open_qubits_default,
                       sycamore_like_circuit, block_base_index, open_bit_positions)

SEED0 = 2406188890


@dataclass
class Workload:
    name: str
    circuit: Circuit
    open_qubits: List[int]
    closed_qubits: List[int]
    closed_bits: np.ndarray  # [G, n_closed] uint8, closed qubits ascending
    n_sliced: int            # number of sliced bond indices (S = 2^n_sliced slices)
    k: int                   # top-k per block
    seed: int

    @property
    def n_qubits(self) -> int:
        return self.circuit.n_qubits

    @property
    def G(self) -> int:
        return int(self.closed_bits.shape[0])

    @property
    def l(self) -> int:
        return len(self.open_qubits)

    @property
    def n_slices(self) -> int:
        return 1 << self.n_sliced

    def block_base(self) -> np.ndarray:
        return block_base_index(self.closed_qubits, self.closed_bits, self.n_qubits)

    def open_bit_pos(self) -> np.ndarray:
        return open_bit_positions(self.open_qubits, self.n_qubits)


def _children(seed: int, n: int = 3):
    ss = np.random.SeedSequence(seed)
    return [int(c.generate_state(1, dtype=np.uint64)[0] & ((1 << 63) - 1)) for c in ss.spawn(n)]


def make_workload(name: str, circuit: Circuit, l: int, G: int, n_sliced: int, k: int,
                  seed: int, open_qubits: Optional[List[int]] = None) -> Workload:
    n = circuit.n_qubits
    opens = list(open_qubits) if open_qubits is not None else open_qubits_default(n, l)
    closed = [q for q in range(n) if q not in set(opens)]
    bits_seed = _children(seed)[1]
    bits = draw_closed_bitstrings(len(closed), G, bits_seed)
    return Workload(name, circuit, opens, closed, bits, n_sliced, k, seed)


def rect_workload(name: str, rows: int, cols: int, cycles: int, l: int, G: int,
                  n_sliced: int, k: int, seed: int) -> Workload:
    circ = grid_circuit(rows, cols, cycles, _children(seed)[0])
    return make_workload(name, circ, l, G, n_sliced, k, seed)


def slice_subset_seed(seed: int) -> int:
    return _children(seed)[2]


def uneven_batch(n_circuits: int = 64, seed: int = SEED0 + 4) -> List[Workload]:
    """64 circuits: grids 4x{4..7}, depth U{10..16}, 2^U{2..8} slices, l = 8, G = 16, k = 16."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for j in range(n_circuits):
        cols = int(rng.integers(4, 8))
        depth = int(rng.integers(10, 17))
        s = int(rng.integers(2, 9))
        out.append(rect_workload(f"uneven[{j}] 4x{cols} d{depth} s{s}", 4, cols, depth,
                                 l=8, G=16, n_sliced=s, k=16, seed=seed + 100 * j))
    return out


CONFIGS = {
    # 3x4 grid, 8 cycles, every qubit open, one block, no slicing
    "grid3x4_d8": dict(rows=3, cols=4, cycles=8, l=12, G=1, n_sliced=0, k=64, seed=SEED0 + 1),
    # 4x6 grid, 14 cycles, 6 sliced bonds (64 slices), 10 open qubits, 64 blocks, k = 64
    "grid4x6_d14": dict(rows=4, cols=6, cycles=14, l=10, G=64, n_sliced=6, k=64, seed=SEED0 + 2),
}


def workload(name: str, **override) -> Workload:
    if name == "sycamore53_d20":
        seed = override.get("seed", SEED0 + 5)
        circ = sycamore_like_circuit(override.get("cycles", 20), _children(seed)[0])
        return make_workload(name, circ, override.get("l", 10), override.get("G", 16),
                             override.get("n_sliced", 0), override.get("k", 16), seed)
    cfg = dict(CONFIGS[name])
    cfg.update(override)
    return rect_workload(name, **cfg)
