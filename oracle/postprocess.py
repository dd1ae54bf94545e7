"""Post-processing of amplitudes in FP64 (test infrastructure only).

* Probabilities (paper Fig. 5 caption and Sec. III): the probability assigned to
  bitstring s after contracting a fraction f of the sub-networks is
  p(s) = |phi(s)|^2 / f.  Here it is computed as (re*re + im*im) * inv_f, each
  operation rounded separately in IEEE FP64 (inv_f = 1/f is an input), so that
  any other implementation making the same three roundings gets identical bits.
* Top-k (Sec. III "Composition of our algorithm"): keep the k strings with the
  largest p(s).  Order: p descending, then full n-bit index ascending (the
  paper does not say how ties break; this is the reading taken).  Per block
  (each group of 2^l correlated strings) or over all groups at once.
* Linear XEB (Eq. 1): F_XEB(S) = N/|S| * sum_{s in S} q(s) - 1, N = 2^n, q the
  ideal probability.
* Numerical fidelity (Fig. 3 caption: fidelity from approximate and exact
  amplitudes; no formula given): the normalised overlap
  |<a|e>|^2 / (<a|a><e|e>) over the computed strings.
* MCMC sampling (Sec. III, Eq. 3: samples drawn from the approximate p over a
  candidate set score an XEB equal to the fidelity F): Metropolis chains over
  the candidates with uniform proposals, accepting a move x -> y with
  probability min(1, p(y) / p(x)), so that p (normalised) is the stationary
  distribution.  The paper does not state its chain; this is the plainest one.
"""
from __future__ import annotations

import numpy as np


def probabilities(amps: np.ndarray, inv_f: float) -> np.ndarray:
    re = np.ascontiguousarray(amps.real, dtype=np.float64)
    im = np.ascontiguousarray(amps.imag, dtype=np.float64)
    return (re * re + im * im) * np.float64(inv_f)


def full_indices(block_base: np.ndarray, open_bit_pos: np.ndarray, l: int) -> np.ndarray:
    """idx[g, j]: n-bit index of block g's j-th string; bit (l-1-i) of j is open qubit i."""
    j = np.arange(1 << l, dtype=np.int64)
    part = np.zeros(1 << l, dtype=np.int64)
    for i in range(l):
        part |= ((j >> (l - 1 - i)) & 1) << np.int64(open_bit_pos[i])
    return np.asarray(block_base, dtype=np.int64)[:, None] | part[None, :]


def _order(p: np.ndarray, idx: np.ndarray) -> np.ndarray:
    # primary key: p descending; secondary: index ascending
    return np.lexsort((idx, -p))


def topk_blocks(amps: np.ndarray, k: int, inv_f: float, block_base: np.ndarray,
                open_bit_pos: np.ndarray):
    """Per-block top-k: returns (idx [G, k] int64, p [G, k] float64), each row sorted."""
    G, B = amps.shape
    l = int(round(np.log2(B)))
    if k > B:
        raise ValueError("k larger than the block")
    p = probabilities(amps, inv_f)
    idx = full_indices(block_base, open_bit_pos, l)
    out_i = np.empty((G, k), dtype=np.int64)
    out_p = np.empty((G, k), dtype=np.float64)
    for g in range(G):
        o = _order(p[g], idx[g])[:k]
        out_i[g] = idx[g][o]
        out_p[g] = p[g][o]
    return out_i, out_p


def topk_global(amps: np.ndarray, k: int, inv_f: float, block_base: np.ndarray,
                open_bit_pos: np.ndarray):
    """Top-k over every string of every block: (idx [k], p [k]), sorted."""
    G, B = amps.shape
    l = int(round(np.log2(B)))
    p = probabilities(amps, inv_f).reshape(-1)
    idx = full_indices(block_base, open_bit_pos, l).reshape(-1)
    if k > p.size:
        raise ValueError("k larger than the candidate set")
    o = _order(p, idx)[:k]
    return idx[o], p[o]


def xeb(q: np.ndarray, n_qubits: int) -> float:
    """Eq. (1): 2^n / |S| * sum q(s) - 1."""
    q = np.asarray(q, dtype=np.float64).reshape(-1)
    if q.size == 0:
        raise ValueError("empty selection")
    return float(np.ldexp(1.0, n_qubits) / q.size * q.sum() - 1.0)


def ideal_probabilities_at(psi: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """q(s) = |<s|C|0>|^2 of the full state vector at the given indices."""
    a = psi[np.asarray(idx, dtype=np.int64)]
    return a.real * a.real + a.imag * a.imag


def numerical_fidelity(approx: np.ndarray, exact: np.ndarray) -> float:
    a = np.asarray(approx, dtype=np.complex128).reshape(-1)
    e = np.asarray(exact, dtype=np.complex128).reshape(-1)
    return float(abs(np.vdot(a, e)) ** 2 / (np.vdot(a, a).real * np.vdot(e, e).real))


def relative_l2(x: np.ndarray, ref: np.ndarray) -> float:
    x = np.asarray(x, dtype=np.complex128).reshape(-1)
    ref = np.asarray(ref, dtype=np.complex128).reshape(-1)
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def metropolis(p: np.ndarray, n_chains: int, n_steps: int, burn: int, rng: np.random.Generator) -> np.ndarray:
    """Candidate indices sampled with probability proportional to p (Eq. 3's
    MCMC baseline): n_chains independent Metropolis chains, each started at a
    uniform candidate; at every step a uniform proposal y replaces the state x
    when u * p(x) < p(y) for u uniform in [0, 1) (so always when p(y) >= p(x),
    and with probability p(y) / p(x) otherwise).  Returns the states of the
    steps after the first ``burn``, chain-major within each step:
    n_chains * (n_steps - burn) indices."""
    p = np.asarray(p, dtype=np.float64).reshape(-1)
    if p.size == 0 or n_chains <= 0 or not 0 <= burn < n_steps:
        raise ValueError("empty candidate set or no sampled steps")
    if np.any(p < 0) or not np.any(p > 0):
        raise ValueError("p must be non-negative with some positive entry")
    x = rng.integers(0, p.size, size=n_chains)
    out = []
    for t in range(n_steps):
        y = rng.integers(0, p.size, size=n_chains)
        u = rng.random(n_chains)
        x = np.where(u * p[x] < p[y], y, x)
        if t >= burn:
            out.append(x.copy())
    return np.concatenate(out)
