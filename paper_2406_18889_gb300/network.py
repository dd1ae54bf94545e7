"""Circuit -> tensor network (host side, once per circuit).

Builds the network whose contraction gives the amplitudes of k groups of 2^l
correlated bitstrings (arXiv 2406.18889, Sec. III "Composition of our
algorithm"): the l open qubits keep their output legs, every closed qubit ends
in a projector onto its sampled bit that carries the shared group (block)
index g, a hyper-edge kept to the output (the "compute only the entries that
feed the wanted bitstrings" approach the paper adopts for the last stem
stages, Sec. III "Optimizing tensor contraction").

Edges are integers.  Wire edges are also named by (qubit, t): the segment of
qubit q after its t-th operation (t = 0 leaves the initial |0>), which is how
sliced edges are named across the library and its callers.

Leaf data stays complex128 on the host; the library converts it to the device
precision when it copies it.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Sequence, Tuple

import numpy as np


@dataclass
class TensorNetwork:
    edge_dim: List[int] = field(default_factory=list)
    leaf_edges: List[Tuple[int, ...]] = field(default_factory=list)
    leaf_data: List[np.ndarray] = field(default_factory=list)  # complex128, axes = leaf_edges
    open_edges: List[int] = field(default_factory=list)        # output order, first = MSB of j
    block_edge: int = -1                                         # g, or -1 when there is one block
    wire_of_edge: Dict[int, Tuple[int, int]] = field(default_factory=dict)
    edge_of_wire: Dict[Tuple[int, int], int] = field(default_factory=dict)
    n_qubits: int = 0
    n_blocks: int = 1

    def new_edge(self, dim: int) -> int:
        self.edge_dim.append(int(dim))
        return len(self.edge_dim) - 1

    def add_leaf(self, edges: Sequence[int], data: np.ndarray) -> int:
        data = np.ascontiguousarray(data, dtype=np.complex128)
        if tuple(data.shape) != tuple(self.edge_dim[e] for e in edges):
            raise ValueError("leaf shape does not match its edges")
        self.leaf_edges.append(tuple(int(e) for e in edges))
        self.leaf_data.append(data)
        return len(self.leaf_edges) - 1

    @property
    def n_leaves(self) -> int:
        return len(self.leaf_edges)

    def output_edges(self) -> List[int]:
        return ([self.block_edge] if self.block_edge >= 0 else []) + list(self.open_edges)


def circuit_network(circuit, open_qubits: Sequence[int], closed_qubits: Sequence[int],
                    closed_bits: np.ndarray) -> TensorNetwork:
    """The amplitude network <s_g, j| C |0^n> for every block g and open value j."""
    n = circuit.n_qubits
    tn = TensorNetwork(n_qubits=n)
    cur: List[int] = []
    t_of = [0] * n

    def wire_edge(q):
        e = tn.new_edge(2)
        tn.wire_of_edge[e] = (q, t_of[q])
        tn.edge_of_wire[(q, t_of[q])] = e
        return e

    for q in range(n):
        cur.append(wire_edge(q))
        tn.add_leaf([cur[q]], np.array([1.0, 0.0]))
    for op in circuit.ops:
        if len(op.qubits) == 1:
            (q,) = op.qubits
            src = cur[q]
            t_of[q] += 1
            dst = wire_edge(q)
            tn.add_leaf([dst, src], op.matrix)
            cur[q] = dst
        elif len(op.qubits) == 2:
            qa, qb = op.qubits
            ia, ib = cur[qa], cur[qb]
            t_of[qa] += 1
            t_of[qb] += 1
            oa, ob = wire_edge(qa), wire_edge(qb)
            tn.add_leaf([oa, ob, ia, ib], np.asarray(op.matrix).reshape(2, 2, 2, 2))
            cur[qa], cur[qb] = oa, ob
        else:
            raise ValueError("only 1- and 2-qubit gates")
    G = int(closed_bits.shape[0])
    tn.n_blocks = G
    closed_qubits = list(closed_qubits)
    if closed_qubits:
        g = tn.new_edge(G)
        tn.block_edge = g
        for c, q in enumerate(closed_qubits):
            proj = np.zeros((G, 2))
            proj[np.arange(G), closed_bits[:, c].astype(np.int64)] = 1.0
            tn.add_leaf([g, cur[q]], proj)
    elif G != 1:
        raise ValueError("no closed qubits means one block")
    tn.open_edges = [cur[q] for q in open_qubits]
    return tn
