"""Discrete adjoint of the frozen-velocity LMEP step (oracle, FP64).

The paper has no adjoint; this is the exact derivative of the forward step of
``oracle.lmep.frozen_step``.  For an updated point i with window idx_i, row r_i
and X_i = dt (nu D2 - u_i D1 + ...),

    F_i(u) = sum_j w_ij(u_i, nu) u[idx_i[j]],   w_i = row r_i of exp(X_i),

so that

    dF_i/du_k = w_i[j: idx_i[j] = k] + delta_ik (dw_i/du_i) . u[idx_i],
    dF_i/dnu  = (dw_i/dnu) . u[idx_i].

dw_i/du_i and dw_i/dnu are rows of the Frechet derivative L(X_i, E) of the
matrix exponential in the directions E = dX_i/du_i = -dt D1 and
E = dX_i/dnu = dt D2.  L(X, E) is the top-right block of
exp([[X, E], [0, X]]) (Mathias 1996; Higham, "Functions of Matrices", 2008,
Thm. 3.6).  The window shift of departure centring is piecewise constant in
u_i and contributes nothing.  Like the weights (``oracle.lmep.exp_row``), the
Frechet rows are evaluated on the re-centred matrix X + k D-hat1: row r of
exp(X(u)) equals row r - k of exp(X(u) + k D-hat1) for every u, so the same
holds for their derivatives, and the re-centred matrix has the smaller norm.
Test infrastructure only.
"""
from __future__ import annotations

import numpy as np

from workloads import Problem

from . import grid
from .expm import expm
from .lmep import exp_row, frozen_step, recentring_shift
from .operator import local_matrix, unit_D


def frechet(X: np.ndarray, E: np.ndarray) -> np.ndarray:
    n = X.shape[0]
    B = np.zeros((2 * n, 2 * n))
    B[:n, :n] = X
    B[:n, n:] = E
    B[n:, n:] = X
    return expm(B)[:n, n:]


def point_derivatives(p: Problem, u: np.ndarray, i: int, D=None):
    """Window, harvested row r, weights w, dw/du_i and dw/dnu for frozen point i."""
    if D is None:
        D = unit_D(p.n)
    k = grid.departure_shift(u[i], p.dt, p.h, p.n) if p.departure_centring else 0
    idx, r = grid.stencil(p, i, k)
    kr = recentring_shift(p, u[i], r)
    Xk = local_matrix(p, u[i], D) + kr * D[1]
    w = exp_row(p, r, u[i], D)[0]
    dX_du = -(p.dt * p.frozen_adv / p.h) * D[1]
    dX_dnu = (p.dt / p.h ** 2) * D[2]
    return idx, r, w, frechet(Xk, dX_du)[r - kr], frechet(Xk, dX_dnu)[r - kr]


def adjoint_step(p: Problem, u: np.ndarray, lam_next: np.ndarray, D=None):
    """lambda^n = (dF/du^n)^T lambda^{n+1} and the step's contribution to dJ/dnu."""
    lam = np.zeros_like(u)
    dnu = 0.0
    for i in grid.updated_points(p):
        idx, r, w, dwu, dwnu = point_derivatives(p, u, i, D)
        for j in range(p.n):
            lam[idx[j]] += lam_next[i] * w[j]
        lam[i] += lam_next[i] * (dwu @ u[idx])
        dnu += lam_next[i] * (dwnu @ u[idx])
    return lam, dnu


def misfit(p: Problem, uT: np.ndarray, target: np.ndarray) -> float:
    """J = (h/2) ||u(T) - u*||^2."""
    return 0.5 * p.h * float(np.sum((uT - target) ** 2))


def gradient(p: Problem, u0: np.ndarray, target: np.ndarray, steps: int):
    """(J, dJ/du0, dJ/dnu) by a forward sweep that stores every state and a reverse sweep."""
    D = unit_D(p.n)
    states = [np.array(u0, dtype=np.float64)]
    for _ in range(steps):
        states.append(frozen_step(p, states[-1], D))
    lam = p.h * (states[-1] - target)
    dnu = 0.0
    for t in range(steps - 1, -1, -1):
        lam, g = adjoint_step(p, states[t], lam, D)
        dnu += g
    return misfit(p, states[-1], target), lam, dnu
