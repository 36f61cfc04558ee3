"""The C build of the frozen-velocity oracle step (oracle/c/lmep_oracle.c).

TEST INFRASTRUCTURE ONLY (tests/, bench.py's CPU-baseline leg).  The same
steps as ``oracle.lmep.frozen_step`` -- window, Lagrange derivative matrices,
re-centred local matrix, Pade scaling and squaring (Higham 2005), harvested
row, dot product -- in plain FP64 C with OpenMP over the grid points, so that
the oracle can be timed on all host cores and can check every point of a
full-size step.  Pinned against the numpy oracle and Thm. 1 in
tests/test_oracle_c.py.  ``build()`` compiles it with gcc; nothing here
touches the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "c", "lmep_oracle.c")
LIB = os.path.join(HERE, "c", "liblmep_oracle.so")
BC = {"periodic": 0, "dirichlet": 1, "neumann": 2}

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle library with gcc (-O3, OpenMP, no machine-specific flags)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp"
        subprocess.run(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c99", SRC, "-o", tmp, "-lm"],
                       check=True, capture_output=True, text=True)
        os.replace(tmp, LIB)
    return LIB


def load() -> C.CDLL:
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(LIB)
        lib.lmep_oracle_frozen_step.argtypes = [
            C.c_int64, C.c_double, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
            C.c_double, C.c_double, C.c_double, C.c_double, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int]
        lib.lmep_oracle_frozen_step.restype = C.c_int
        lib.lmep_oracle_threads.restype = C.c_int
        _lib = lib
    return _lib


def frozen_step(p, u, points=None, threads: int = 0) -> np.ndarray:
    """One frozen-velocity step of Problem p from state u at `points` (all points if None)."""
    lib = load()
    u = np.ascontiguousarray(u, dtype=np.float64)
    if points is None:
        pts, npts = None, p.N
    else:
        pts = np.ascontiguousarray(points, dtype=np.int64)
        npts = len(pts)
    out = np.empty(npts, dtype=np.float64)
    rc = lib.lmep_oracle_frozen_step(p.N, p.h, BC[p.bc], p.n, int(p.departure_centring), p.dt, p.c0, p.c1, p.c2,
                                     p.c3, p.frozen_adv, p.bc_lo, p.bc_hi, u.ctypes.data,
                                     None if pts is None else pts.ctypes.data, npts, out.ctypes.data, threads)
    if rc != 0:
        raise ValueError("unsupported stencil width")
    return out


def threads() -> int:
    return int(load().lmep_oracle_threads())
