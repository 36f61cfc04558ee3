"""Shared helpers of the GPU tests: translate a workload Problem into the
library's Grid/Operator and compare results with stated tolerances."""
import numpy as np

import workloads as wl

# Parity tolerances (stated in the parity tests' docstrings):
TOL_FP64 = 1e-12     # FP64 path, relative (weights: ||dw||_inf / ||w||_1; states: rel l_inf)
TOL_MIXED = 1e-5     # FP32 form (FP32 products/apply, FP64 solve and squarings)


def tol(precision):
    return TOL_FP64 if precision == "fp64" else TOL_MIXED


def grid_of(p: wl.Problem):
    from paper_2603_15964_gb300 import Grid
    return Grid(N=p.N, h=p.h, bc=p.bc, n=p.n, departure_centring=p.departure_centring,
                bc_lo=p.bc_lo, bc_hi=p.bc_hi, window_shift=p.window_shift)


def op_of(p: wl.Problem):
    from paper_2603_15964_gb300 import Operator
    return Operator(c0=p.c0, c1=p.c1, c2=p.c2, c3=p.c3, frozen_adv=p.frozen_adv)


def weight_err(got, want):
    """max over rows of ||dw||_inf / ||w||_1."""
    got = np.asarray(got, dtype=np.float64).reshape(-1, want.shape[-1])
    want = np.asarray(want, dtype=np.float64).reshape(-1, want.shape[-1])
    den = np.maximum(np.sum(np.abs(want), axis=1), 1e-300)
    return float(np.max(np.max(np.abs(got - want), axis=1) / den))


def rel_linf(got, want):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    return float(np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-300))
