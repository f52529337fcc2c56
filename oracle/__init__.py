"""Oracle for the stencil sweeps and the learned tuner's network -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  The CUDA library never calls it and shares no code with it; the product path fails
loudly when its CUDA extension is missing instead of falling back here.

Contents:
* ``sweep(...)``     -- the plain FP64 naive time-stepping sweep (``girih_oracle.c``), the exact
                        definition of what the temporally blocked GPU sweep computes.
* ``brute``          -- an independent per-point evaluator driven by a table of (offset, coefficient)
                        terms, used to cross-check the C loop nests on tiny grids.
* ``mlp``            -- FP64 forward/backward/optimiser steps of the tuner's 3-layer network.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "girih_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, no FP contraction, OpenMP for the timed baseline)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC",
               "-o", _LIB, _SRC]
        subprocess.run(cmd, check=True)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_sweep.restype = ctypes.c_int
        lib.oracle_sweep.argtypes = [ctypes.c_int] + [ctypes.c_int64] * 5 + [ctypes.c_void_p] * 4 + [ctypes.c_int]
        _lib = lib
    return _lib


RADIUS = {0: 1, 1: 1, 2: 4, 3: 4, 4: 4, 5: 1, 6: 1}


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def sweep(stencil: int, u: np.ndarray, u_prev: np.ndarray, coeffs, c, T: int, nx: int, ny: int, nz: int,
          nthreads: int = 1) -> None:
    """Advance (u, u_prev) by T steps in place, FP64.  Arrays are padded [nz+2R][ny+2R][ldx]."""
    lib = _load()
    R = RADIUS[stencil]
    for a in (u, u_prev):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"] and a.ndim == 3
        assert a.shape[0] == nz + 2 * R and a.shape[1] == ny + 2 * R
    ldx = u.shape[2]
    cc = np.ascontiguousarray(np.asarray(c, dtype=np.float64)) if c is not None and len(c) else None
    co = None if coeffs is None else np.ascontiguousarray(coeffs, dtype=np.float64)
    rc = lib.oracle_sweep(stencil, nx, ny, nz, ldx, T, _ptr(u), _ptr(u_prev), _ptr(co), _ptr(cc), nthreads)
    if rc != 0:
        raise ValueError("oracle_sweep rejected its arguments")
