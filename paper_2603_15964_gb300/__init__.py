"""GB300 (sm_103a) Local Matrix Exponential Propagator -- Python binding.

The functions below carry the names of the C entry points of include/lmep.h
and only marshal arguments (torch tensors -> device pointers, current CUDA
stream).  Every step of the computation runs in the library's CUDA kernels;
nothing here computes on the host and there is no fallback path.

Method: V. Bayona, "Unifying Finite Differences and Semi-Lagrangian Schemes
via Localized Matrix Exponentials" (Sec. 2.1: localisation, local
exponential, harvest; Sec. 3.1: augmented local matrix and ETD stepping).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import BC, EXPM, NONLIN, PREC, SCHEME, LmepError  # noqa: F401

__all__ = ["Grid", "Operator", "Handle", "lmep_build_operator", "lmep_expm", "lmep_harvest_weights",
           "lmep_harvest_scheme_weights", "scheme_rows",
           "lmep_step", "lmep_batch_workspace_bytes", "lmep_batch_prepare", "lmep_step_batched",
           "lmep_step_batched_once", "lmep_frozen_set_workspace_bytes", "lmep_frozen_set_prepare",
           "lmep_frozen_set_refresh", "lmep_frozen_set_step_once", "frozen_set_offsets",
           "lmep_adjoint_scratch_bytes", "lmep_adjoint_step", "lmep_adjoint_step_noalloc", "lmep_frozen_stats", "lmep_set_expm_method", "lmep_set_wait_limit", "lmep_sync_status",
           "lmep_fma_peak", "lmep_amplification", "lmep_harvest_nodes", "lmep_step_nodes",
           "state_dtype", "LmepError"]


@dataclass(frozen=True)
class Grid:
    """Uniform grid and stencil (lmep_grid)."""

    N: int
    h: float
    bc: str = "periodic"
    n: int = 5
    departure_centring: bool = False
    bc_lo: float = 0.0
    bc_hi: float = 0.0
    batch: int = 1
    window_shift: int = 0

    def c(self) -> _lib.LmepGrid:
        return _lib.LmepGrid(self.N, self.h, BC[self.bc], self.n, int(self.departure_centring), self.batch,
                             self.window_shift, 0, self.bc_lo, self.bc_hi)


@dataclass(frozen=True)
class Operator:
    """L = c0 + c1 d/dx + c2 d^2/dx^2 + c3 d^3/dx^3 - frozen_adv u_i d/dx (lmep_operator)."""

    c0: float = 0.0
    c1: float = 0.0
    c2: float = 0.0
    c3: float = 0.0
    frozen_adv: float = 0.0

    def c(self) -> _lib.LmepOperator:
        return _lib.LmepOperator(self.c0, self.c1, self.c2, self.c3, self.frozen_adv)


def state_dtype(precision: str) -> torch.dtype:
    return torch.float64 if precision == "fp64" else torch.float32


def _ptr(t) -> C.c_void_p:
    if t is None:
        return C.c_void_p(None)
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("tensors passed to the LMEP library must be contiguous CUDA tensors")
    return C.c_void_p(t.data_ptr())


def _state_ptr(t) -> C.c_void_p:
    """A state buffer: a contiguous CUDA tensor, or a contiguous pinned host tensor (read and written by the
    kernels in place through unified addressing)."""
    if not t.is_cuda and t.is_contiguous() and t.is_pinned():
        return C.c_void_p(t.data_ptr())
    return _ptr(t)


def _stream(stream=None) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Handle:
    """Owns an lmep_handle (device status block) on the current device."""

    def __init__(self):
        lib = _lib.load()
        h = C.c_void_p()
        _lib.check(lib.lmep_create(C.byref(h)), "lmep_create")
        self._h = h
        self._keep = []  # host arrays referenced by prepared batch workspaces

    @property
    def ptr(self) -> C.c_void_p:
        return self._h

    def close(self):
        if self._h:
            _lib.load().lmep_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lmep_build_operator(h: Handle, grid: Grid, op: Operator, dt: float, n_phi: int, u, i0: int, count: int,
                        M, start, row, stream=None) -> None:
    _lib.call("lmep_build_operator", h.ptr, C.byref(grid.c()), C.byref(op.c()), dt, n_phi, _ptr(u), i0, count,
              _ptr(M), _ptr(start), _ptr(row), _stream(stream))


def lmep_expm(h: Handle, A, d: int, E, precision: str = "fp64", ms=None, stream=None) -> None:
    P = A.numel() // (d * d)
    _lib.call("lmep_expm", h.ptr, _ptr(A), P, d, _ptr(E), PREC[precision], _ptr(ms), _stream(stream))


def lmep_harvest_weights(h: Handle, grid: Grid, op: Operator, dt: float, n_phi: int, u_frozen, W,
                         precision: str = "fp64", stream=None) -> None:
    _lib.call("lmep_harvest_weights", h.ptr, C.byref(grid.c()), C.byref(op.c()), dt, n_phi, _ptr(u_frozen),
              _ptr(W), PREC[precision], _stream(stream))


def scheme_rows(scheme: str) -> int:
    """Weight rows per row class that lmep_step reads for a scheme."""
    return {"linear": 1, "etd1": 2, "etdrk2": 3, "etdrk4": 6}[scheme]


def lmep_harvest_scheme_weights(h: Handle, grid: Grid, op: Operator, dt: float, scheme: str, W,
                                precision: str = "fp64", stream=None) -> None:
    _lib.call("lmep_harvest_scheme_weights", h.ptr, C.byref(grid.c()), C.byref(op.c()), dt, SCHEME[scheme], _ptr(W),
              PREC[precision], _stream(stream))


def lmep_step(h: Handle, grid: Grid, op: Operator, scheme: str, nonlin: str, dt: float, W, u, work,
              nsteps: int, precision: str = "fp64", stream=None) -> None:
    _lib.call("lmep_step", h.ptr, C.byref(grid.c()), C.byref(op.c()), SCHEME[scheme], NONLIN[nonlin], dt,
              _ptr(W), _ptr(u), _ptr(work), nsteps, PREC[precision], _stream(stream))


def _batch_desc(Ns, hs, bcs, n, scheme, nonlin, dt, op: Operator, tile=0, block=0, ctas_per_sm=0):
    B = len(Ns)
    N_arr = (C.c_int64 * B)(*[int(v) for v in Ns])
    h_arr = (C.c_double * B)(*[float(v) for v in hs])
    bc_arr = (C.c_int32 * B)(*[BC[b] if isinstance(b, str) else int(b) for b in bcs])
    d = _lib.LmepBatchDesc(B, N_arr, h_arr, bc_arr, n, SCHEME[scheme], NONLIN[nonlin], tile, block, ctas_per_sm,
                           dt, op.c())
    return d, (N_arr, h_arr, bc_arr)


def lmep_batch_workspace_bytes(Ns, hs, bcs, n, scheme, nonlin, dt, op: Operator, precision="mixed", tile=0,
                               block=0, ctas_per_sm=0) -> int:
    d, keep = _batch_desc(Ns, hs, bcs, n, scheme, nonlin, dt, op, tile, block, ctas_per_sm)
    out = C.c_size_t()
    _lib.call("lmep_batch_workspace_bytes", C.byref(d), PREC[precision], C.byref(out))
    return int(out.value)


def lmep_batch_prepare(h: Handle, Ns, hs, bcs, n, scheme, nonlin, dt, op: Operator, workspace,
                       precision="mixed", tile=0, block=0, ctas_per_sm=0, stream=None) -> None:
    d, keep = _batch_desc(Ns, hs, bcs, n, scheme, nonlin, dt, op, tile, block, ctas_per_sm)
    _lib.call("lmep_batch_prepare", h.ptr, C.byref(d), _ptr(workspace), workspace.numel() * workspace.element_size(),
              PREC[precision], _stream(stream))


def lmep_step_batched(h: Handle, workspace, u, work, nsteps: int, stream=None) -> None:
    _lib.call("lmep_step_batched", h.ptr, _ptr(workspace), _ptr(u), _ptr(work), nsteps, _stream(stream))


def lmep_step_batched_once(h: Handle, workspace, u_in, u_out, stream=None) -> None:
    _lib.call("lmep_step_batched_once", h.ptr, _ptr(workspace), _ptr(u_in), _ptr(u_out), _stream(stream))


def _set_desc(grids, ops, dts, block=0, points_per_thread=0):
    B = len(grids)
    g_arr = (_lib.LmepGrid * B)(*[g.c() for g in grids])
    o_arr = (_lib.LmepOperator * B)(*[o.c() for o in ops])
    t_arr = (C.c_double * B)(*[float(t) for t in dts])
    d = _lib.LmepFrozenSetDesc(B, g_arr, o_arr, t_arr, block, points_per_thread)
    return d, (g_arr, o_arr, t_arr)


def frozen_set_offsets(Ns) -> list:
    """Start of every instance in a frozen set's state: prefix sums of N_b rounded up to 4."""
    offs = [0]
    for v in Ns:
        offs.append(offs[-1] + (int(v) + 3) // 4 * 4)
    return offs


def lmep_frozen_set_workspace_bytes(grids, ops, dts, precision="mixed", block=0, points_per_thread=0) -> int:
    d, keep = _set_desc(grids, ops, dts, block, points_per_thread)
    out = C.c_size_t()
    _lib.call("lmep_frozen_set_workspace_bytes", C.byref(d), PREC[precision], C.byref(out))
    return int(out.value)


def lmep_frozen_set_prepare(h: Handle, grids, ops, dts, workspace, precision="mixed", block=0, points_per_thread=0,
                            stream=None) -> None:
    d, keep = _set_desc(grids, ops, dts, block, points_per_thread)
    _lib.call("lmep_frozen_set_prepare", h.ptr, C.byref(d), _ptr(workspace),
              workspace.numel() * workspace.element_size(), PREC[precision], _stream(stream))


def lmep_frozen_set_refresh(h: Handle, workspace, stream=None) -> None:
    _lib.call("lmep_frozen_set_refresh", h.ptr, _ptr(workspace), _stream(stream))


def lmep_frozen_set_step_once(h: Handle, workspace, u_in, u_out, stream=None) -> None:
    """One step of every instance of a prepared set, u_in -> u_out: CUDA tensors, or pinned host tensors."""
    _lib.call("lmep_frozen_set_step_once", h.ptr, _ptr(workspace), _state_ptr(u_in), _state_ptr(u_out),
              _stream(stream))


def lmep_adjoint_scratch_bytes(grid: Grid, precision: str = "fp64") -> int:
    out = C.c_size_t()
    _lib.call("lmep_adjoint_scratch_bytes", C.byref(grid.c()), PREC[precision], C.byref(out))
    return int(out.value)


def lmep_adjoint_step(h: Handle, grid: Grid, op: Operator, dt: float, u, lam_next, lam, dnu, scratch,
                      precision: str = "fp64", stream=None) -> None:
    _lib.call("lmep_adjoint_step", h.ptr, C.byref(grid.c()), C.byref(op.c()), dt, _ptr(u), _ptr(lam_next),
              _ptr(lam), _ptr(dnu), _ptr(scratch), scratch.numel() * scratch.element_size(), PREC[precision],
              _stream(stream))


def lmep_adjoint_step_noalloc(grid: Grid, op: Operator, dt: float, u, lam_next, lam, dnu,
                              precision: str = "fp64", stream=None) -> None:
    """lmep_adjoint_step without caller scratch or handle (library-static scratch, no allocation)."""
    _lib.call("lmep_adjoint_step_noalloc", C.byref(grid.c()), C.byref(op.c()), dt, _ptr(u), _ptr(lam_next),
              _ptr(lam), _ptr(dnu), PREC[precision], _stream(stream))


def lmep_frozen_stats(h: Handle, grid: Grid, op: Operator, dt: float, u, stats, precision: str = "fp64",
                      stream=None) -> None:
    _lib.call("lmep_frozen_stats", h.ptr, C.byref(grid.c()), C.byref(op.c()), dt, _ptr(u), _ptr(stats),
              PREC[precision], _stream(stream))


def lmep_set_expm_method(h: Handle, method: str = "auto") -> None:
    """Frozen-velocity exponential rows of handle h: "series" (finite series of the nilpotent local
    matrix, Pade scaling and squaring where its error bound is large), "auto" (the factorised row
    l(r + a)^T exp(E) first, then as "series") or "pade"."""
    _lib.call("lmep_set_expm_method", h.ptr, EXPM[method])


def lmep_set_wait_limit(h: Handle, polls: int = -1) -> None:
    """Bound (in polls) of the streaming apply's waits for its bulk copies; -1 restores the default."""
    _lib.call("lmep_set_wait_limit", h.ptr, int(polls))


def lmep_sync_status(h: Handle, stream=None) -> None:
    _lib.call("lmep_sync_status", h.ptr, _stream(stream))


def lmep_harvest_nodes(h: Handle, x, n: int, op: Operator, dt: float, scheme: str, W, precision: str = "fp64",
                       stream=None) -> None:
    """Per-node weight rows W[N][rows][n] on the non-uniform grid x (float64 CUDA tensor, Dirichlet walls)."""
    _lib.call("lmep_harvest_nodes", h.ptr, int(x.numel()), _ptr(x), n, C.byref(op.c()), dt, SCHEME[scheme], _ptr(W),
              PREC[precision], _stream(stream))


def lmep_step_nodes(h: Handle, N: int, n: int, scheme: str, nonlin: str, dt: float, bc_lo: float, bc_hi: float, W,
                    u, work, nsteps: int, precision: str = "fp64", stream=None) -> None:
    _lib.call("lmep_step_nodes", h.ptr, N, n, SCHEME[scheme], NONLIN[nonlin], dt, bc_lo, bc_hi, _ptr(W), _ptr(u),
              _ptr(work), nsteps, PREC[precision], _stream(stream))


def lmep_amplification(w, r: int, theta, G, stream=None) -> None:
    """G[q] = sum_j w_j e^{i theta_q (j - r)} (G: float64 [M, 2], real and imaginary parts)."""
    _lib.call("lmep_amplification", _ptr(w), int(w.numel()), int(r), _ptr(theta), int(theta.numel()), _ptr(G),
              _stream(stream))


def lmep_fma_peak(precision: str = "fp64") -> float:
    out = C.c_double()
    _lib.call("lmep_fma_peak", PREC[precision], C.byref(out))
    return float(out.value)
