"""Element-wise amplitude parity used by the GPU tests.

A single relative L2 over all G * 2^l amplitudes dilutes a localised error:
one wrong block of 1024 among 64 moves it by 1/8 of that block's error, one
wrong element by 1/256.  So, beside the global relative L2 <= tol:

* every block (row) g has relative L2 <= tol on its own;
* every element's error is at most K_ELEM * tol times the RMS amplitude of its
  block.  With a per-element error of RMS tol * rms (what a relative L2 of tol
  means), the largest of up to 2^24 complex errors stays below ~6 of those
  RMS units (the tail of the error modulus falls as exp(-x^2)); K_ELEM = 8
  keeps the check free of false alarms while a wrong element -- whose error
  is of the order of the amplitudes themselves -- fails it by a factor of
  ~1 / (8 tol).
"""
from __future__ import annotations

import numpy as np

K_ELEM = 8.0


def parity_report(got, ref) -> dict:
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    g2 = got.reshape(ref.shape[0], -1) if ref.ndim > 1 else got.reshape(1, -1)
    r2 = ref.reshape(ref.shape[0], -1) if ref.ndim > 1 else ref.reshape(1, -1)
    d = g2 - r2
    rn = np.linalg.norm(r2, axis=1)
    dn = np.linalg.norm(d, axis=1)
    glob = float(np.linalg.norm(d) / np.linalg.norm(r2))
    nz = rn > 0
    per_block = float(np.max(dn[nz] / rn[nz])) if nz.any() else 0.0
    rms = rn / np.sqrt(r2.shape[1])
    elem = float(np.max(np.abs(d[nz]).max(axis=1) / rms[nz])) if nz.any() else 0.0
    # blocks whose reference is exactly zero must come out exactly zero
    zero_blocks_ok = bool(np.all(dn[~nz] == 0))
    return {"global": glob, "max_block": per_block, "max_elem_over_rms": elem, "zero_blocks_ok": zero_blocks_ok}


def assert_amplitudes_close(got, ref, tol: float, what: str = "") -> dict:
    """Global relative L2, per-block relative L2 and per-element error against
    the block RMS, all held to `tol` (elements to K_ELEM * tol)."""
    r = parity_report(got, ref)
    assert r["global"] <= tol, (what, "global relative L2", r)
    assert r["max_block"] <= tol, (what, "worst block's relative L2", r)
    assert r["max_elem_over_rms"] <= K_ELEM * tol, (what, "worst element's error / block RMS", r)
    assert r["zero_blocks_ok"], (what, "a block that is zero in the reference is not", r)
    return r
