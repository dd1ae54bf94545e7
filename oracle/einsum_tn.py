"""O2: naive FP64 tensor-network contractor with slicing (test infrastructure only).

Builds its own tensor network from the circuit's gate list and contracts it
pairwise in complex128.  It follows these passages of arXiv 2406.18889:

* Sec. III "Composition of our algorithm": amplitudes are computed for k groups
  of 2^l correlated bitstrings -- the l open qubits run over all values, the
  other qubits are fixed to one sampled bitstring per group.  Here each closed
  qubit ends in a projector P_q[g, b] = [b == s_g(q)] that carries the shared
  group index g (a hyper-index kept to the output).
* Sec. III "Optimizing tensor contraction": slicing fixes the value of chosen
  edges; the network equals the sum of its sliced sub-networks over every
  assignment of those values (for two edges i, j:
  TN = TN_{00} + TN_{01} + TN_{10} + TN_{11}).
* Sec. III "Composition of our algorithm": the approximate amplitude contracts
  only a fraction f of the sub-networks and sums them.

Network: one rank-1 tensor |0> per qubit, one tensor per gate (U[out, in] for
one qubit, U[o_a, o_b, i_a, i_b] for two), one projector per closed qubit.
The wire segment of qubit q after its t-th operation is the edge ('w', q, t)
(t = 0 leaves the initial |0>).  Sliced edges are named by these labels; slice
id sigma fixes sliced edge i to bit i of sigma, (sigma >> i) & 1.

Each pairwise step is the plain definition of a contraction: labels shared by
both operands are summed unless another tensor or the output still needs them
(then they are carried as a batch index); the step is computed as a batched
matrix product after transposing the operands.  The pairwise order comes from
this module's own greedy rule (smallest growth first); the order changes only
rounding, not the result.
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass
from typing import Dict, Hashable, List, Optional, Sequence, Tuple

import numpy as np

G_LABEL = ("g",)


def wire(q: int, t: int) -> Tuple:
    return ("w", int(q), int(t))


@dataclass
class Network:
    arrays: List[np.ndarray]
    labels: List[Tuple[Hashable, ...]]
    dims: Dict[Hashable, int]
    output: Tuple[Hashable, ...]
    n_blocks: int
    n_open: int


def build_network(circuit, open_qubits: Sequence[int], closed_qubits: Sequence[int],
                  closed_bits: np.ndarray) -> Network:
    n = circuit.n_qubits
    arrays, labels = [], []
    dims: Dict[Hashable, int] = {}
    seg = [0] * n
    for q in range(n):
        arrays.append(np.array([1.0, 0.0], dtype=np.complex128))
        labels.append((wire(q, 0),))
        dims[wire(q, 0)] = 2
    for op in circuit.ops:
        if len(op.qubits) == 1:
            (q,) = op.qubits
            a, b = wire(q, seg[q] + 1), wire(q, seg[q])
            arrays.append(np.asarray(op.matrix, dtype=np.complex128).copy())
            labels.append((a, b))
            dims[a] = 2
            seg[q] += 1
        else:
            qa, qb = op.qubits
            oa, ob = wire(qa, seg[qa] + 1), wire(qb, seg[qb] + 1)
            ia, ib = wire(qa, seg[qa]), wire(qb, seg[qb])
            arrays.append(np.asarray(op.matrix, dtype=np.complex128).reshape(2, 2, 2, 2).copy())
            labels.append((oa, ob, ia, ib))
            dims[oa] = dims[ob] = 2
            seg[qa] += 1
            seg[qb] += 1
    G = int(closed_bits.shape[0])
    closed_qubits = list(closed_qubits)
    if closed_qubits:
        dims[G_LABEL] = G
        for c, q in enumerate(closed_qubits):
            p = np.zeros((G, 2), dtype=np.complex128)
            p[np.arange(G), closed_bits[:, c].astype(np.int64)] = 1.0
            arrays.append(p)
            labels.append((G_LABEL, wire(q, seg[q])))
        output = (G_LABEL,) + tuple(wire(q, seg[q]) for q in open_qubits)
    else:
        if G != 1:
            raise ValueError("no closed qubits means a single block")
        output = tuple(wire(q, seg[q]) for q in open_qubits)
    return Network(arrays, labels, dims, output, G, len(list(open_qubits)))


def _size(lbls, dims) -> float:
    s = 1.0
    for x in lbls:
        s *= dims[x]
    return s


def _result_labels(la, lb, occ, output, i, j):
    out = []
    for x in la:
        if x in lb and x not in output and occ[x] <= {i, j}:
            continue
        out.append(x)
    for x in lb:
        if x not in la:
            out.append(x)
    return tuple(out)


def greedy_path(labels: Sequence[Tuple], dims: Dict, output: Sequence) -> List[Tuple[int, int]]:
    """Pairwise order: repeatedly contract the pair (sharing a label) whose result
    grows the total size least; SSA ids (inputs 0..T-1, step t creates T+t)."""
    output = set(output)
    live = {i: tuple(l) for i, l in enumerate(labels)}
    occ: Dict[Hashable, set] = {}
    for i, l in live.items():
        for x in l:
            occ.setdefault(x, set()).add(i)
    heap = []

    def push(i, j):
        if i > j:
            i, j = j, i
        lc = _result_labels(live[i], live[j], occ, output, i, j)
        sc = _size(lc, dims)
        score = sc - _size(live[i], dims) - _size(live[j], dims)
        heapq.heappush(heap, (score, sc, i, j))

    seen = set()
    for x, ids in occ.items():
        ids = sorted(ids)
        for a in range(len(ids)):
            for b in range(a + 1, len(ids)):
                if (ids[a], ids[b]) not in seen:
                    seen.add((ids[a], ids[b]))
                    push(ids[a], ids[b])
    path = []
    nxt = len(labels)
    while len(live) > 1:
        if heap:
            score, sc, i, j = heapq.heappop(heap)
            if i not in live or j not in live:
                continue
        else:  # disconnected components: join the two smallest by outer product
            ids = sorted(live, key=lambda t: (_size(live[t], dims), t))
            i, j = sorted(ids[:2])
        lc = _result_labels(live[i], live[j], occ, output, i, j)
        path.append((i, j))
        for x in live[i] + live[j]:
            occ[x].discard(i)
            occ[x].discard(j)
        del live[i], live[j]
        k = nxt
        nxt += 1
        live[k] = lc
        nbrs = set()
        for x in lc:
            nbrs |= occ[x]
            occ[x].add(k)
        for m in sorted(nbrs):
            push(m, k)
    return path


def pair_contract(A: np.ndarray, la: Tuple, B: np.ndarray, lb: Tuple, keep: set,
                  dims: Dict) -> Tuple[np.ndarray, Tuple]:
    """C[batch, fa, fb] = sum_k A[batch, fa, k] B[batch, k, fb] (definition of a
    pairwise contraction with hyper-indices kept when ``keep`` still needs them)."""
    shared = [x for x in la if x in lb]
    batch = [x for x in shared if x in keep]
    summed = [x for x in shared if x not in keep]
    fa = [x for x in la if x not in lb]
    fb = [x for x in lb if x not in la]
    for x in fa + fb:
        if x not in keep:
            raise ValueError(f"dangling label {x}")
    p = lambda ls: int(np.prod([dims[x] for x in ls], dtype=np.int64)) if ls else 1  # noqa: E731
    At = A.transpose([la.index(x) for x in batch + fa + summed]).reshape(p(batch), p(fa), p(summed))
    Bt = B.transpose([lb.index(x) for x in batch + summed + fb]).reshape(p(batch), p(summed), p(fb))
    C = np.matmul(At, Bt)
    lc = tuple(batch + fa + fb)
    return C.reshape([dims[x] for x in lc]), lc


def contract_arrays(arrays: Sequence[np.ndarray], labels: Sequence[Tuple], dims: Dict,
                    output: Sequence, path: Optional[List[Tuple[int, int]]] = None) -> np.ndarray:
    """Contract a whole network (no slicing) and return it in ``output`` order."""
    output = tuple(output)
    if path is None:
        path = greedy_path(labels, dims, output)
    live = {i: (a, tuple(l)) for i, (a, l) in enumerate(zip(arrays, labels))}
    nxt = len(arrays)
    for (i, j) in path:
        A, la = live.pop(i)
        B, lb = live.pop(j)
        keep = set(output)
        for (_, l) in live.values():
            keep.update(l)
        C, lc = pair_contract(A, la, B, lb, keep, dims)
        live[nxt] = (C, lc)
        nxt += 1
    if len(live) != 1:
        raise ValueError("path did not reduce the network to one tensor")
    (C, lc), = live.values()
    if set(lc) != set(output):
        raise ValueError(f"result labels {lc} differ from output {output}")
    return C.transpose([lc.index(x) for x in output])


def _fix(arrays, labels, dims, sliced, sigma):
    """Slice sigma: fix sliced edge i to (sigma >> i) & 1 in every tensor holding it."""
    arrs, lbls = [], []
    fixed = {lab: (int(sigma) >> i) & 1 for i, lab in enumerate(sliced)}
    for a, l in zip(arrays, labels):
        for lab, v in fixed.items():
            if lab in l:
                ax = l.index(lab)
                a = np.take(a, v, axis=ax)
                l = l[:ax] + l[ax + 1:]
        arrs.append(a)
        lbls.append(l)
    return arrs, lbls


def _as_label(x) -> Tuple:
    """A sliced edge given as (q, t) or as a wire label ('w', q, t)."""
    x = tuple(x)
    if len(x) == 3 and x[0] == "w":
        return wire(x[1], x[2])
    if len(x) == 2:
        return wire(x[0], x[1])
    raise ValueError(f"bad sliced edge {x}")


def _check_sliced(net: Network, sliced):
    for lab in sliced:
        holders = [i for i, l in enumerate(net.labels) if lab in l]
        if lab in net.output or len(holders) != 2:
            raise ValueError(f"{lab} is not an internal bond")


def _as_blocks(net: Network, C: np.ndarray) -> np.ndarray:
    return C.reshape(net.n_blocks, 1 << net.n_open)


def contract(net: Network, sliced: Sequence = (), slice_ids: Optional[Sequence[int]] = None
             ) -> np.ndarray:
    """amps[g, j] = sum over the chosen slices sigma of TN_sigma (all 2^s slices when
    ``slice_ids`` is None, which gives the exact amplitudes)."""
    per = contract_each_slice(net, sliced, slice_ids)
    return per.sum(axis=0)


def contract_each_slice(net: Network, sliced: Sequence = (),
                        slice_ids: Optional[Sequence[int]] = None) -> np.ndarray:
    """[n_slices, G, 2^l]: each chosen sliced sub-network contracted on its own."""
    sliced = [_as_label(x) for x in sliced]
    _check_sliced(net, sliced)
    if slice_ids is None:
        slice_ids = range(1 << len(sliced))
    slice_ids = list(slice_ids)
    out = np.zeros((len(slice_ids), net.n_blocks, 1 << net.n_open), dtype=np.complex128)
    path = None
    for n_i, sigma in enumerate(slice_ids):
        if not 0 <= int(sigma) < (1 << len(sliced)):
            raise ValueError("slice id out of range")
        arrs, lbls = _fix(net.arrays, net.labels, net.dims, sliced, sigma)
        if path is None:
            path = greedy_path(lbls, net.dims, net.output)
        out[n_i] = _as_blocks(net, contract_arrays(arrs, lbls, net.dims, net.output, path))
    return out


def amplitudes(circuit, open_qubits, closed_qubits, closed_bits, sliced=(), slice_ids=None):
    """Convenience: build the network and contract the chosen slices, [G, 2^l]."""
    net = build_network(circuit, open_qubits, closed_qubits, closed_bits)
    return contract(net, sliced, slice_ids)
