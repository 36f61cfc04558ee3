"""Finite-difference weights on arbitrary nodes (oracle, FP64).

Sec. 2.1, step 1 builds the local differentiation matrix D_n with Fornberg's
recursive algorithm (Fornberg 1988).  The recursion below is derived from the
Lagrange basis: when node x_i joins nodes x_0..x_{i-1},

  l_j^{(i)}(z) = l_j^{(i-1)}(z) (z - x_i) / (x_j - x_i)            (j < i)
  l_i^{(i)}(z) = l_{i-1}^{(i-1)}(z) (z - x_{i-1}) c_{i-1} / c_i

with c_i = prod_{j<i} (x_i - x_j).  Differentiating k times (Leibniz rule)
turns each product with a linear factor into two terms, giving a recursion on
the k-th derivative weights.  Test infrastructure only.
"""
from __future__ import annotations

import numpy as np


def weights(z: float, x, kmax: int) -> np.ndarray:
    """Return C[k, j] (k = 0..kmax) with sum_j C[k, j] f(x_j) = f^(k)(z) for deg f < len(x)."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    C = np.zeros((kmax + 1, n))
    C[0, 0] = 1.0
    c_prev = 1.0                                   # c_{i-1} = prod_{j<i-1} (x_{i-1} - x_j)
    for i in range(1, n):
        old = C.copy()                             # weights using nodes 0..i-1
        c_i = 1.0
        for j in range(i):
            c_i *= x[i] - x[j]
        # existing nodes: multiply l_j by (z - x_i)/(x_j - x_i)
        for j in range(i):
            for k in range(0, min(i, kmax) + 1):
                lower = k * old[k - 1, j] if k > 0 else 0.0
                C[k, j] = ((z - x[i]) * old[k, j] + lower) / (x[j] - x[i])
        # the new node: l_i = l_{i-1} (z - x_{i-1}) c_{i-1} / c_i
        for k in range(0, min(i, kmax) + 1):
            lower = k * old[k - 1, i - 1] if k > 0 else 0.0
            C[k, i] = (c_prev / c_i) * ((z - x[i - 1]) * old[k, i - 1] + lower)
        c_prev = c_i
    return C


def derivative_matrices(x, kmax: int = 3) -> np.ndarray:
    """D[k] (n x n): row i holds the weights of d^k/dx^k at node x_i on all n nodes."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    D = np.zeros((kmax + 1, n, n))
    for i in range(n):
        D[:, i, :] = weights(x[i], x, kmax)
    return D


def unit_derivative_matrices(n: int, kmax: int = 3) -> np.ndarray:
    """D-hat[k] on the integer nodes 0..n-1: the uniform-grid D^(k) times h^k."""
    return derivative_matrices(np.arange(n, dtype=np.float64), kmax)
