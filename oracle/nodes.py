"""Non-uniform grids: weights harvested per point on the window's own nodes (oracle, FP64).

TEST INFRASTRUCTURE ONLY.  Sec. 4.3.3 runs the method on Chebyshev nodes, where the local
differentiation matrix differs from point to point: every node gets its own weights, harvested
once and stored, and a step is a banded product with those stored rows.  Written out plainly:

* window of point i: the n consecutive nodes start_i .. start_i + n - 1,
  start_i = clamp(i - (n-1)/2, 0, N - n), harvest row r_i = i - start_i (the walls are grid points
  that keep their Dirichlet values; next to them the windows are one-sided, as in Example 1);
* local matrix X_i = dt (c0 I + c1 D1 + c2 D2 + c3 D3) with D^(k) Fornberg's weights on the
  window's nodes (Sec. 2.1 step 1, ``fornberg.derivative_matrices``);
* its exponential row r_i, or the rows of dt^k phi_k from the augmented local matrix (Sec. 3.1),
  by ``expm`` (Higham 2005) -- stored as W[i][k][:];
* ETDRK4 (Sec. 3): W[i] holds six rows, exp(dt L), dt alpha, dt beta, dt gamma (from p = 3 at dt)
  and exp(dt L / 2), (dt/2) phi_1(dt L / 2) (from p = 1 at dt/2);
* the steppers of ``oracle.lmep`` with those per-point rows; N(u) is pointwise (Allen-Cahn u - u^3)
  or absent.
"""
from __future__ import annotations

import math

import numpy as np

from workloads import DIRICHLET, Problem

from . import fornberg
from .expm import expm
from .operator import augmented_row


def chebyshev_nodes(N: int, a: float = -1.0, b: float = 1.0) -> np.ndarray:
    """Chebyshev-Gauss-Lobatto points in ascending order: (a+b)/2 - (b-a)/2 cos(pi j/(N-1))."""
    j = np.arange(N, dtype=np.float64)
    return 0.5 * (a + b) - 0.5 * (b - a) * np.cos(np.pi * j / (N - 1))


def window(p: Problem, i: int):
    n, N = p.n, p.N
    start = min(max(i - (n - 1) // 2, 0), N - n)
    return np.arange(start, start + n), i - start


def local_matrix(p: Problem, x: np.ndarray, i: int, dt: float | None = None) -> np.ndarray:
    dt = p.dt if dt is None else dt
    idx, _ = window(p, i)
    D = fornberg.derivative_matrices(x[idx], 3)
    return dt * (p.c0 * np.eye(p.n) + p.c1 * D[1] + p.c2 * D[2] + p.c3 * D[3])


def point_rows(p: Problem, x: np.ndarray, i: int, n_phi: int, dt: float | None = None) -> np.ndarray:
    """Rows k = 0..n_phi of dt^k phi_k(X_i) at the harvest row of point i."""
    dt = p.dt if dt is None else dt
    idx, r = window(p, i)
    X = local_matrix(p, x, i, dt)
    if n_phi == 0:
        return expm(X)[r:r + 1, :].copy()
    E = expm(augmented_row(X, dt, r, n_phi))
    n = p.n
    return np.stack([E[r, :n]] + [E[n + k, :n] for k in range(n_phi)])


def weights(p: Problem, x: np.ndarray) -> np.ndarray:
    """W[N][R][n], R = 1, 2, 3 (linear, ETD1, ETDRK2) or 6 (ETDRK4)."""
    rows = []
    for i in range(p.N):
        if p.scheme != "etdrk4":
            rows.append(point_rows(p, x, i, p.n_phi))
            continue
        w = point_rows(p, x, i, 3)
        w1, w2, w3 = w[1], w[2] / p.dt, w[3] / p.dt ** 2
        h = point_rows(p, x, i, 1, 0.5 * p.dt)
        rows.append(np.stack([w[0], w1 - 3 * w2 + 4 * w3, 2 * w2 - 4 * w3, 4 * w3 - w2, h[0], h[1]]))
    return np.array(rows)


def _apply(p: Problem, W: np.ndarray, k: int, v: np.ndarray) -> np.ndarray:
    out = np.zeros_like(v)
    for i in range(1, p.N - 1):
        idx, _ = window(p, i)
        out[i] = W[i, k] @ v[idx]
    return out


def _walls(p: Problem, v: np.ndarray) -> np.ndarray:
    v[0], v[-1] = p.bc_lo, p.bc_hi
    return v


def _nonlinear(p: Problem, v: np.ndarray) -> np.ndarray:
    if p.nonlin == "none":
        return np.zeros_like(v)
    if p.nonlin == "allen_cahn":
        return v - v ** 3
    raise ValueError(p.nonlin)


def step(p: Problem, W: np.ndarray, u: np.ndarray) -> np.ndarray:
    if p.bc != DIRICHLET:
        raise ValueError("non-uniform grids take Dirichlet walls")
    if p.scheme == "linear":
        return _walls(p, _apply(p, W, 0, u))
    Nu = _nonlinear(p, u)
    if p.scheme == "etdrk4":
        a = _walls(p, _apply(p, W, 4, u) + _apply(p, W, 5, Nu))
        Na = _nonlinear(p, a)
        b = _walls(p, _apply(p, W, 4, u) + _apply(p, W, 5, Na))
        Nb = _nonlinear(p, b)
        c = _walls(p, _apply(p, W, 4, a) + _apply(p, W, 5, 2.0 * Nb - Nu))
        Nc = _nonlinear(p, c)
        return _walls(p, _apply(p, W, 0, u) + _apply(p, W, 1, Nu) + _apply(p, W, 2, Na + Nb) + _apply(p, W, 3, Nc))
    a = _walls(p, _apply(p, W, 0, u) + _apply(p, W, 1, Nu))
    if p.scheme == "etd1":
        return a
    Na = _nonlinear(p, a)
    return _walls(p, a + _apply(p, W, 2, Na - Nu) / p.dt)


def run(p: Problem, x: np.ndarray, u0: np.ndarray, steps: int | None = None) -> np.ndarray:
    steps = p.steps if steps is None else steps
    W = weights(p, x)
    u = np.array(u0, dtype=np.float64)
    for _ in range(steps):
        u = step(p, W, u)
    return u


def stretched_nodes(N: int, beta: float = 2.0) -> np.ndarray:
    """A smooth non-uniform grid on [-1, 1]: sinh(beta s) / sinh(beta), s uniform (nodes cluster at 0)."""
    s = np.linspace(-1.0, 1.0, N)
    return np.sinh(beta * s) / math.sinh(beta)
