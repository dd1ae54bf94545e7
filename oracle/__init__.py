"""FP64 CPU oracle for sliced tensor-network random-circuit sampling.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
benchmark's CPU-baseline leg may import this package; the library's product
path never does, and this package imports nothing from the library.

Contents (each function cites the passage of arXiv 2406.18889 it follows):

* ``statevector``  -- O1: exact amplitudes <s|C|0^n> by applying every gate to
  a complex128 state vector in circuit order.
* ``einsum_tn``    -- O2: an independent tensor network built from the gate
  list, contracted pairwise in FP64, with slicing (Sec. III "Optimizing tensor
  contraction", the slicing identity TN = sum over fixed edge values) and
  partial contraction of a fraction f of the slices (Sec. III "Composition of
  our algorithm").
* ``postprocess``  -- probabilities |phi|^2/f (Fig. 5), per-block and global
  top-k (Sec. III), linear XEB (Eq. 1), numerical fidelity, Metropolis
  sampling from p (the MCMC baseline of Eq. 3).
* ``theory``       -- the paper's closed forms: Porter-Thomas moments
  (App. A), ideal and approximate top-k XEB (Eqs. 2 and 4) and the exact
  finite-size order-statistics expectation used to pin them.

Every function here is pinned by ``-m "not gpu"`` tests against facts that do
not come from this package (closed forms, brute force, invariants).
"""
from . import statevector, einsum_tn, postprocess, theory  # noqa: F401
