"""Exact rational arithmetic for tiny stencils (oracle pin tier).

* Lagrange-basis derivative matrices: D^(k)[i, j] = l_j^(k)(x_i), the plain
  definition of the weights that are exact on polynomials of degree < n
  (Thm. 1 proof: D_n is exact on P_{n-1}).
* Nilpotency (remark after Example 1, Thm. 2 proof): a purely differential
  local operator K_n maps P_{n-1} into P_{n-2}, so K_n^n = 0 and
  exp(K_n) = sum_{k<n} K_n^k / k! exactly.  With exact rational entries this
  finite sum is the exact exponential of the FP64 input, with no rounding.
Test infrastructure only.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def _poly_mul_linear(c: list, root) -> list:
    """(sum_i c_i x^i) * (x - root)."""
    out = [Fraction(0)] * (len(c) + 1)
    for i, ci in enumerate(c):
        out[i + 1] += ci
        out[i] -= ci * root
    return out


def _poly_deriv(c: list) -> list:
    return [c[i] * i for i in range(1, len(c))] or [Fraction(0)]


def _poly_eval(c: list, x) -> Fraction:
    acc = Fraction(0)
    for ci in reversed(c):
        acc = acc * x + ci
    return acc


def lagrange_D(nodes, k: int) -> list:
    """Exact D^(k) on rational nodes as a list of lists of Fractions."""
    xs = [Fraction(v) for v in nodes]
    n = len(xs)
    rows = [[Fraction(0)] * n for _ in range(n)]
    for j in range(n):
        c = [Fraction(1)]
        den = Fraction(1)
        for m in range(n):
            if m != j:
                c = _poly_mul_linear(c, xs[m])
                den *= xs[j] - xs[m]
        c = [ci / den for ci in c]
        for _ in range(k):
            c = _poly_deriv(c)
        for i in range(n):
            rows[i][j] = _poly_eval(c, xs[i])
    return rows


def to_frac(M: np.ndarray) -> list:
    return [[Fraction(float(v)) for v in row] for row in np.asarray(M)]


def to_float(M: list) -> np.ndarray:
    return np.array([[float(v) for v in row] for row in M])


def matmul(A: list, B: list) -> list:
    n, m, p = len(A), len(B), len(B[0])
    return [[sum((A[i][k] * B[k][j] for k in range(m)), Fraction(0)) for j in range(p)]
            for i in range(n)]


def is_zero(A: list) -> bool:
    return all(v == 0 for row in A for v in row)


def expm_nilpotent(X: list) -> list:
    """sum_{k<d} X^k/k! for a nilpotent d x d rational X; raises if X^d != 0."""
    d = len(X)
    term = [[Fraction(int(i == j)) for j in range(d)] for i in range(d)]
    acc = [row[:] for row in term]
    for k in range(1, d + 1):
        term = matmul(term, X)
        if k == d:
            if not is_zero(term):
                raise ValueError("matrix is not nilpotent")
            break
        f = Fraction(1, math.factorial(k))
        acc = [[acc[i][j] + f * term[i][j] for j in range(d)] for i in range(d)]
    return acc


def local_matrix(n: int, dt: float, h: float, c1: float, c2: float, c3: float = 0.0) -> list:
    """Exact X = dt (c1 D1 + c2 D2 + c3 D3) on the window h*(0..n-1), from FP64 coefficients.

    The three FP64 products dt*c_k/h^k are rounded exactly as the oracle rounds
    them; everything after that is exact.
    """
    coef = [Fraction(dt * c1 / h), Fraction(dt * c2 / h ** 2), Fraction(dt * c3 / h ** 3)]
    nodes = list(range(n))
    Ds = [lagrange_D(nodes, k) for k in (1, 2, 3)]
    return [[sum(coef[k] * Ds[k][i][j] for k in range(3)) for j in range(n)] for i in range(n)]
