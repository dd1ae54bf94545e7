"""Build and load the oracle's plain-C helpers (test infrastructure only).

``build()`` compiles ``csrc/*.c`` with gcc into ``_build/liboracle_sv.so``.
Flags: -O2, OpenMP, and -ffp-contract=off so that no multiply-add is fused
(the same arithmetic on x86-64 and aarch64 hosts).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from pathlib import Path

HERE = Path(__file__).resolve().parent
SRC = HERE / "csrc" / "statevector.c"
OUT_DIR = HERE / "_build"
LIB = OUT_DIR / "liboracle_sv.so"

_lib = None


def build(force: bool = False) -> Path:
    OUT_DIR.mkdir(exist_ok=True)
    if LIB.exists() and not force and LIB.stat().st_mtime >= SRC.stat().st_mtime:
        return LIB
    tmp = OUT_DIR / f"liboracle_sv.{os.getpid()}.so"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           str(SRC), "-o", str(tmp)]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def load():
    global _lib
    if _lib is None:
        path = build()
        lib = ctypes.CDLL(str(path))
        dp = ctypes.POINTER(ctypes.c_double)
        lib.sv_apply_1q.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
        lib.sv_apply_2q.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        lib.sv_zero_state.argtypes = [dp, ctypes.c_int]
        for f in (lib.sv_apply_1q, lib.sv_apply_2q, lib.sv_zero_state):
            f.restype = None
        _lib = lib
    return _lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
