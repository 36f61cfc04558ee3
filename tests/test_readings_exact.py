"""Pins, in exact rational arithmetic, of the identities behind the GPU routes for frozen-velocity rows.

The local matrix of a window is X = a D1 + b D2 + c D3 on the integer nodes 0..n-1 (a the local
Courant number, b and c the diffusion and dispersion numbers, the identity term factored out).
 * Its derivative matrices are powers of one differentiation matrix on the local polynomial space
   (D2 = D1^2, D3 = D1^3 exactly), so they commute and X is nilpotent (the General Exactness
   theorem's proof): exp(X) is a finite sum.
 * Hence row r of exp(X) equals l(r + a)^T exp(b D2 + c D3), l the Lagrange weights of the window
   at the departure point (Thm. 1 for the advection factor), and the a-derivative of that row is
   l'(r + a)^T exp(b D2 + c D3), the form the adjoint takes.
 * The finite series evaluated in floating point stays within 2 u beta of the exact row,
   beta = sum_k ||e_r^T |X|^k||_1 / k! (the bound the kernels use to choose their route).
Everything here is exact (Fractions) except the last pin, which checks a floating-point series
written in this file against exact rows.
"""
from fractions import Fraction

import numpy as np
import pytest

import workloads as wl
from oracle import exact, grid as ogrid, operator as oop


def lagrange_row(n, z):
    """Exact Lagrange weights l_j(z) of the nodes 0..n-1."""
    out = []
    for j in range(n):
        v = Fraction(1)
        for m in range(n):
            if m != j:
                v *= Fraction(z - m, j - m) if isinstance(z, int) else (z - m) / (j - m)
        out.append(v)
    return out


def lagrange_row_derivative(n, z):
    """Exact l_j'(z) = sum_q prod_{m != j, q} (z - m) / prod_{m != j} (j - m)."""
    out = []
    for j in range(n):
        den = Fraction(1)
        for m in range(n):
            if m != j:
                den *= j - m
        acc = Fraction(0)
        for q in range(n):
            if q == j:
                continue
            t = Fraction(1)
            for m in range(n):
                if m not in (j, q):
                    t *= z - m
            acc += t
        out.append(acc / den)
    return out


def lin(*terms):
    """sum of coefficient * matrix (lists of Fractions)."""
    n = len(terms[0][1])
    return [[sum(c * M[i][j] for c, M in terms) for j in range(n)] for i in range(n)]


@pytest.mark.parametrize("n", [3, 5, 7, 9])
def test_derivative_matrices_are_powers(n):
    D1, D2, D3 = (exact.lagrange_D(range(n), k) for k in (1, 2, 3))
    assert exact.matmul(D1, D1) == D2
    assert exact.matmul(D2, D1) == D3
    assert exact.matmul(D1, D2) == exact.matmul(D2, D1)


@pytest.mark.parametrize("n", [5, 7])
@pytest.mark.parametrize("a,b,c", [(Fraction(3, 7), Fraction(1, 9), Fraction(0)),
                                   (Fraction(-5, 4), Fraction(1, 50), Fraction(-1, 300)),
                                   (Fraction(2.3), Fraction(0.02), Fraction(0))])
def test_factorised_row_is_exact(n, a, b, c):
    D1, D2, D3 = (exact.lagrange_D(range(n), k) for k in (1, 2, 3))
    full = exact.expm_nilpotent(lin((a, D1), (b, D2), (c, D3)))
    expE = exact.expm_nilpotent(lin((b, D2), (c, D3)))
    for r in range(n):
        l = lagrange_row(n, r + a)
        row = [sum(l[j] * expE[j][k] for j in range(n)) for k in range(n)]
        assert row == full[r], r


@pytest.mark.parametrize("n", [5, 7])
def test_lagrange_derivative_is_the_advection_row_derivative(n):
    """d/da e_r^T exp(a D1) = e_r^T D1 exp(a D1) = l'(r + a)^T (exactly)."""
    D1 = exact.lagrange_D(range(n), 1)
    for a in (Fraction(1, 3), Fraction(-7, 5)):
        E = exact.expm_nilpotent(lin((a, D1)))
        DE = exact.matmul(D1, E)
        for r in range(n):
            assert lagrange_row_derivative(n, r + a) == DE[r]
            assert lagrange_row(n, r + a) == E[r]


@pytest.mark.parametrize("nu,n,cfl", [(1e-6, 13, 4.0), (4e-4, 13, 4.0), (1e-3, 9, 2.0)])
def test_series_error_within_two_u_beta(nu, n, cfl):
    """Reading of the finite-series route: the floating-point series (FP64 and FP32) is within
    2 u beta of the exact row, on Burgers rows whose beta spans 1 .. 1e3."""
    p = wl.burgers(N=513, n=n, cfl=cfl, nu=nu)
    u = wl.burgers_ic(513, 0)
    D = oop.unit_D(n)
    D1, D2 = exact.lagrange_D(range(n), 1), exact.lagrange_D(range(n), 2)
    rng = np.random.default_rng(n)
    for i in sorted(set(rng.integers(1, 512, 8).tolist()) | {1, 2, 510, 511}):
        idx, r = ogrid.stencil(p, i, ogrid.departure_shift(u[i], p.dt, p.h, n))
        a = -p.dt * u[i] / p.h
        bd = p.dt * p.c2 / p.h ** 2
        kr = int(np.clip(np.floor(a + 0.5), r - (n - 1), r))     # any in-range shift gives the row
        X = (a - kr) * D[1] + bd * D[2]
        hr = r - kr
        Xe = lin((Fraction(a - kr), D1), (Fraction(bd), D2))
        ex = np.array([float(v) for v in exact.expm_nilpotent(Xe)[hr]])
        A = np.abs(X)
        w = np.zeros(n)
        w[hr] = 1.0
        beta = 1.0
        for k in range(1, n):
            w = w @ A / k
            beta += w.sum()
        for dt_, unit in ((np.float64, 2.0 ** -53), (np.float32, 2.0 ** -24)):
            Xt = X.astype(dt_)
            v = np.zeros(n, dt_)
            v[hr] = 1
            acc = v.copy()
            for k in range(1, n):
                v = (v @ Xt) / dt_(k)
                acc = acc + v
            err = np.max(np.abs(acc.astype(np.float64) - ex)) / np.sum(np.abs(ex))
            assert err <= 2.0 * unit * beta + 4 * unit, (i, dt_, err, beta)


# ------------------------------------------------------------------ wide stencils (n = 17 .. 25)
def row_series(n, X, v):
    """v^T exp(X) for a nilpotent X, by the finite series of row-vector products."""
    acc, t = v[:], v[:]
    for k in range(1, n + 1):
        t = [sum((t[i] * X[i][j] for i in range(n)), Fraction(0)) / k for j in range(n)]
        if k == n:
            assert all(x == 0 for x in t)
            break
        acc = [acc[j] + t[j] for j in range(n)]
    return acc


@pytest.mark.parametrize("n", [17, 25])
def test_wide_derivative_matrices_are_powers(n):
    """The wide rows take D2 = D1^2 and D3 = D1^3: exact on the window's polynomial space at these widths too."""
    D1, D2, D3 = (exact.lagrange_D(range(n), k) for k in (1, 2, 3))
    assert exact.matmul(D1, D1) == D2
    assert exact.matmul(D2, D1) == D3


@pytest.mark.parametrize("n", [17, 25])
def test_wide_factorised_row_is_exact(n):
    """Row r of exp(a D1 + b D2 + c D3) equals l(r + a)^T exp(b D2 + c D3) at the wide widths, for the
    classes a one-sided (r = n - 1) and a centred (r = (n - 1) / 2) window take."""
    D1, D2, D3 = (exact.lagrange_D(range(n), k) for k in (1, 2, 3))
    a, b, c = Fraction(-n, 2), Fraction(1, 40), Fraction(-1, 900)
    X = lin((a, D1), (b, D2), (c, D3))
    E = lin((b, D2), (c, D3))
    for r in (n - 1, (n - 1) // 2):
        e_r = [Fraction(int(j == r)) for j in range(n)]
        assert row_series(n, E, lagrange_row(n, r + a)) == row_series(n, X, e_r), r


def test_oracle_pade_rows_are_themselves_off_at_wide_n():
    """Why exact rows decide the GPU's wide rows: the oracle's Pade of the rounded local matrix of a
    diffusive, dispersive n = 25 operator is off its exact row by more than 1e-10 of the row's l1 norm."""
    from oracle import lmep as olmep
    N = 3001
    h = 2.0 / N
    p = wl.Problem("adv", N, -1.0, 1.0, wl.PERIODIC, 25, 0.0, c0=-0.3, c1=-1.0, c2=0.0625 * h, c3=1e-3 * h * h,
                   steps=1).with_(dt=0.8 * 2.0 / N)
    r = 12
    X = exact.local_matrix(p.n, p.dt, p.h, p.c1, p.c2, p.c3)
    want = np.exp(p.c0 * p.dt) * np.array([float(x) for x in
                                           row_series(p.n, X, [Fraction(int(j == r)) for j in range(p.n)])])
    got = olmep.constant_weights(p)[r, 0]
    assert np.max(np.abs(got - want)) > 1e-10 * np.sum(np.abs(want))
