"""Local operator and augmented local matrix (oracle).

* Thm. 2 (proof): L_n = c0 I + K_n, the discrete local operator with a
  reaction part c0 and a differential part K_n built from the derivative
  matrices D^(k) of the stencil.  For a frozen-velocity Burgers point the
  operator gains -u_i D^(1) (the locally frozen advection speed u_i).
* Sec. 3.1 step 1: the augmented local matrix of dimension s n.
* The row-restricted augmented matrix of dimension n + p (Sidje 1998,
  Al-Mohy & Higham 2011, both cited in Sec. 3): exponentiating

      M = [[X^T, dt e_r, 0 ],
           [0,   0,     dt],
           [0,   0,     0 ]]          (p = 2 shown)

  gives dt phi_1(X^T) e_r and dt^2 phi_2(X^T) e_r in its last columns, i.e.
  row r of dt^k phi_k(X) transposed.  The oracle builds the transpose of M,
  whose rows r, n, n+1 (first n columns) are the harvested rows.
Test infrastructure only.
"""
from __future__ import annotations

import numpy as np

from workloads import Problem

from . import fornberg


def unit_D(n: int) -> np.ndarray:
    return fornberg.unit_derivative_matrices(n, 3)


def local_matrix(p: Problem, u_i: float = 0.0, D: np.ndarray | None = None) -> np.ndarray:
    """X = dt * (c0 I + c1 D1 + c2 D2 + c3 D3 - frozen_adv u_i D1) on the uniform window.

    D^(k) = D-hat^(k) / h^k with D-hat on the integer nodes 0..n-1 (translation invariant).
    """
    n, h, dt = p.n, p.h, p.dt
    if D is None:
        D = unit_D(n)
    a1 = p.c1 - p.frozen_adv * u_i
    return (dt * p.c0 * np.eye(n) + (dt * a1 / h) * D[1] + (dt * p.c2 / h ** 2) * D[2]
            + (dt * p.c3 / h ** 3) * D[3])


def augmented_block(X: np.ndarray, dt: float, s: int) -> np.ndarray:
    """Sec. 3.1: dt * A-tilde_n, the s n x s n block matrix [[L, I, 0..], [0, 0, I..], .., 0].

    X = dt L; the identity blocks are scaled by dt because the whole generator is.
    """
    n = X.shape[0]
    A = np.zeros((s * n, s * n))
    A[:n, :n] = X
    for b in range(s - 1):
        A[b * n:(b + 1) * n, (b + 1) * n:(b + 2) * n] = dt * np.eye(n)
    return A


def augmented_row(X: np.ndarray, dt: float, r: int, p: int) -> np.ndarray:
    """Transpose of the (n+p) x (n+p) row-restricted augmented matrix for harvest row r."""
    n = X.shape[0]
    M = np.zeros((n + p, n + p))
    M[:n, :n] = X
    if p >= 1:
        M[n, r] = dt
    for j in range(1, p):
        M[n + j, n + j - 1] = dt
    return M
