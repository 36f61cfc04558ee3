"""Pins of the oracle's frozen-velocity harvest and adjoint.

* Exact rows: with exact rational D-hat and the FP64 coefficients, the local
  operator is nilpotent, so row r of exp(X) is the finite sum
  sum_{k<n} e_r^T X^k / k!  (nilpotency remark after Example 1), evaluated
  here in 60-digit arithmetic.
* Adjoint: central finite differences of the oracle's own forward map (the
  definition of a derivative), the Frechet derivative against finite
  differences of expm, and the dot-product identity <lambda, du> = <dF du, mu>.
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import adjoint, exact, expm as ox, lmep, operator

mp = pytest.importorskip("mpmath")


def exact_row(n, a_hat, mu_hat, r, dps=60):
    """Row r of exp(a_hat D-hat1 + mu_hat D-hat2) from the finite Taylor series."""
    mp.mp.dps = dps
    D1 = exact.lagrange_D(range(n), 1)
    D2 = exact.lagrange_D(range(n), 2)
    q = lambda f: mp.mpf(f.numerator) / f.denominator
    X = [[mp.mpf(a_hat) * q(D1[i][j]) + mp.mpf(mu_hat) * q(D2[i][j]) for j in range(n)] for i in range(n)]
    v = [mp.mpf(int(j == r)) for j in range(n)]
    acc = v[:]
    for k in range(1, n + 1):
        v = [sum(v[i] * X[i][j] for i in range(n)) / k for j in range(n)]
        acc = [acc[j] + v[j] for j in range(n)]
    assert max(abs(x) for x in v) < mp.mpf(10) ** (-40)      # the series has terminated
    return np.array([float(x) for x in acc])


@pytest.mark.parametrize("n", [7, 9, 13])
@pytest.mark.parametrize("cfl", [1.0, 2.0, 4.0])
def test_frozen_rows_match_exact_series(n, cfl):
    """Burgers-shaped rows (departure-centred, stable-variant nu) to 1e-13 of the exact row."""
    N = 4001
    p = wl.burgers(N=N, n=n, cfl=cfl, nu=1e-6, steps=1)
    u = wl.burgers_ic(N, seed=0)
    rng = np.random.default_rng(n)
    D = operator.unit_D(n)
    for i in list(rng.integers(1, N - 1, 6)) + [1, 2, N - 2, N - 3]:
        idx, r, w = lmep.point_weights(p, u, int(i), D)
        a_hat = -p.dt * p.frozen_adv * u[i] / p.h
        mu_hat = p.dt * p.c2 / p.h ** 2
        want = exact_row(n, a_hat, mu_hat, r)
        err = np.max(np.abs(w[0] - want)) / np.sum(np.abs(want))
        assert err < 1e-13, (i, r, err)
        # the plain (un-recentred) evaluation agrees to its own, larger, FP64 error
        _, _, w_plain = lmep.point_weights(p, u, int(i), D, recentre=False)
        assert np.max(np.abs(w_plain[0] - want)) / np.sum(np.abs(want)) < 2e-9


def test_frechet_matches_finite_differences():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((7, 7)) * 0.6
    E = rng.standard_normal((7, 7))
    L = adjoint.frechet(X, E)
    eps = 1e-5
    fd = (ox.expm(X + eps * E) - ox.expm(X - eps * E)) / (2 * eps)
    assert np.max(np.abs(L - fd)) < 1e-8 * np.max(np.abs(L))


def small_burgers(departure_centring=True):
    N = 48
    p = wl.burgers(N=N, n=7, cfl=1.6, nu=2e-4, steps=6, departure_centring=departure_centring)
    return p, wl.burgers_ic(N, seed=3), wl.burgers_ic(N, seed=1003)


@pytest.mark.parametrize("centring", [False, True])
def test_adjoint_gradient_matches_central_differences(centring):
    p, u0, target = small_burgers(centring)
    steps = 6
    J, g_u, g_nu = adjoint.gradient(p, u0, target, steps)

    def J_of(u_init, nu):
        q = p.with_(c2=nu)
        return adjoint.misfit(q, lmep.run(q, u_init, steps), target)

    rng = np.random.default_rng(0)
    for i in rng.choice(np.arange(1, p.N - 1), 8, replace=False):
        eps = 1e-6
        up, um = u0.copy(), u0.copy()
        up[i] += eps
        um[i] -= eps
        fd = (J_of(up, p.c2) - J_of(um, p.c2)) / (2 * eps)
        assert abs(fd - g_u[i]) < 1e-6 * max(abs(fd), 1e-3 * np.max(np.abs(g_u))), (i, fd, g_u[i])
    eps = 1e-7 * p.c2 * 10
    fd_nu = (J_of(u0, p.c2 + eps) - J_of(u0, p.c2 - eps)) / (2 * eps)
    assert abs(fd_nu - g_nu) < 1e-5 * abs(fd_nu), (fd_nu, g_nu)


def test_adjoint_dot_product_identity():
    """<lambda, du> = <dF du, mu> for one step: the adjoint is the transpose of the linearisation."""
    p, u, _ = small_burgers(False)
    rng = np.random.default_rng(2)
    du = rng.standard_normal(p.N)
    mu = rng.standard_normal(p.N)
    eps = 1e-6
    Jdu = (lmep.frozen_step(p, u + eps * du) - lmep.frozen_step(p, u - eps * du)) / (2 * eps)
    lam, _ = adjoint.adjoint_step(p, u, mu)
    assert abs(lam @ du - mu @ Jdu) < 1e-7 * (abs(lam @ du) + 1.0)
