"""Matrix exponential by Pade scaling and squaring (oracle, FP64).

Sec. 2.1 step 2 computes W_n = exp(dt D_n) but does not say how (it cites
Moler & Van Loan).  Reading: the scaling-and-squaring method of N. J. Higham,
"The scaling and squaring method for the matrix exponential revisited",
SIAM J. Matrix Anal. Appl. 26(4), 2005, Algorithm 2.3:

* the diagonal Pade approximant r_m = q_m^{-1} p_m with
  p_m(x) = sum_j b_j x^j,  b_j = (2m-j)! m! / ((2m)! j! (m-j)!),  q_m(x) = p_m(-x);
* degree m in {3, 5, 7, 9} when ||A||_1 <= theta_m, else m = 13 after scaling
  A by 2^-s with s = ceil(log2(||A||_1 / theta_13));
* p_m = V + U, q_m = V - U with U the odd and V the even part, evaluated with
  the products of Higham's eqs. (2.10)-(2.11); q_m r = p_m solved by LU with
  partial pivoting; then s squarings.
theta_m are the backward-error bounds of Higham (2005), Table 2.3.
Test infrastructure only.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

THETA = {3: 1.495585217958292e-2, 5: 2.539398330063230e-1, 7: 9.504178996162932e-1,
         9: 2.097847961257068e0, 13: 5.371920351148152e0}


def pade_coefficients(m: int) -> list[float]:
    f = math.factorial
    return [float(Fraction(f(2 * m - j) * f(m), f(2 * m) * f(j) * f(m - j))) for j in range(m + 1)]


def norm1(A: np.ndarray) -> float:
    return float(np.max(np.sum(np.abs(A), axis=0)))


def pade_uv(A: np.ndarray, m: int):
    """Odd part U and even part V of p_m(A), so p_m = V + U and q_m = V - U."""
    b = pade_coefficients(m)
    I = np.eye(A.shape[0])
    A2 = A @ A
    if m < 13:
        powers = [I, A2]                          # A^0, A^2, A^4, ...
        for _ in range(2, (m - 1) // 2 + 1):
            powers.append(powers[-1] @ A2)
        odd = sum(b[2 * j + 1] * powers[j] for j in range((m - 1) // 2 + 1))
        even = sum(b[2 * j] * powers[j] for j in range((m - 1) // 2 + 1))
        return A @ odd, even
    A4 = A2 @ A2
    A6 = A4 @ A2
    U = A @ (A6 @ (b[13] * A6 + b[11] * A4 + b[9] * A2) + b[7] * A6 + b[5] * A4 + b[3] * A2 + b[1] * I)
    V = A6 @ (b[12] * A6 + b[10] * A4 + b[8] * A2) + b[6] * A6 + b[4] * A4 + b[2] * A2 + b[0] * I
    return U, V


def lu_solve(Q: np.ndarray, P: np.ndarray) -> np.ndarray:
    """Solve Q R = P by Gaussian elimination with partial pivoting (plain loops)."""
    Q = Q.copy()
    R = P.copy()
    d = Q.shape[0]
    for k in range(d):
        piv = k + int(np.argmax(np.abs(Q[k:, k])))
        if piv != k:
            Q[[k, piv]] = Q[[piv, k]]
            R[[k, piv]] = R[[piv, k]]
        for i in range(k + 1, d):
            l = Q[i, k] / Q[k, k]
            Q[i, k:] -= l * Q[k, k:]
            R[i] -= l * R[k]
    for k in range(d - 1, -1, -1):
        R[k] = (R[k] - Q[k, k + 1:] @ R[k + 1:]) / Q[k, k]
    return R


def choose(A: np.ndarray):
    """Pade degree m and scaling power s of Higham (2005) Algorithm 2.3."""
    a = norm1(A)
    for m in (3, 5, 7, 9):
        if a <= THETA[m]:
            return m, 0
    s = max(0, math.ceil(math.log2(a / THETA[13]))) if a > 0 else 0
    return 13, s


def expm(A: np.ndarray, return_ms: bool = False):
    m, s = choose(A)
    As = A / 2.0 ** s
    U, V = pade_uv(As, m)
    R = lu_solve(V - U, V + U)
    for _ in range(s):
        R = R @ R
    return (R, m, s) if return_ms else R
