"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it follows.  None of them compares the oracle
with itself: the expected values come from closed forms printed in the
paper, exact rational arithmetic, an independent library routine, or an
identity that holds for the exact result.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

import workloads as wl
from oracle import exact, expm as ox, fornberg, grid, lmep, operator

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def poly(coefs, t):
    return sum(c * t ** k for k, c in enumerate(coefs))


def lagrange_weights(nodes, xi):
    """Plain Lagrange basis values l_j(xi) by the product formula."""
    nodes = np.asarray(nodes, dtype=np.float64)
    w = np.ones(len(nodes))
    for j in range(len(nodes)):
        for m in range(len(nodes)):
            if m != j:
                w[j] *= (xi - nodes[m]) / (nodes[j] - nodes[m])
    return w


# ------------------------------------------------------------ Fornberg (Sec. 2.1 step 1)
@pytest.mark.parametrize("kind", ["uniform", "random", "chebyshev"])
def test_fornberg_exact_on_monomials(kind):
    """D^(k) x^m equals the k-th derivative of x^m at every node for m <= n-1."""
    n = 9
    rng = np.random.default_rng(3)
    x = {"uniform": np.arange(n) * 0.25 - 1.0,
         "random": np.sort(rng.uniform(-1, 1, n)),
         "chebyshev": -np.cos(np.pi * np.arange(n) / (n - 1))}[kind]
    D = fornberg.derivative_matrices(x, 3)
    for k in range(4):
        for m in range(n):
            got = D[k] @ x ** m
            want = (math.factorial(m) / math.factorial(m - k) * x ** (m - k)) if m >= k else 0 * x
            assert np.max(np.abs(got - want)) <= 1e-9 * max(1.0, np.max(np.abs(want)))


@pytest.mark.parametrize("n", [3, 5, 7, 9, 11, 13, 15])
def test_fornberg_matches_exact_lagrange(n):
    """Integer nodes: the recursion agrees with exact rational Lagrange derivatives."""
    D = fornberg.unit_derivative_matrices(n, 3)
    for k in (1, 2, 3):
        E = exact.to_float(exact.lagrange_D(range(n), k))
        assert np.max(np.abs(D[k] - E)) <= 4e-15 * np.max(np.abs(E)) * n


def test_example1_derivative_matrix():
    """Example 1 prints h D_3^(1) on {-h, 0, h}."""
    g = golden("example1_advection_n3.json")
    D = fornberg.derivative_matrices([-1.0, 0.0, 1.0], 1)[1]
    assert np.allclose(D, np.array(g["h_D3_1"]), rtol=0, atol=1e-15)


def test_centred_five_point_rows():
    D = fornberg.unit_derivative_matrices(5, 2)
    assert np.allclose(D[1][2], [1 / 12, -2 / 3, 0, 2 / 3, -1 / 12], atol=1e-15)
    assert np.allclose(D[2][2], [-1 / 12, 4 / 3, -5 / 2, 4 / 3, -1 / 12], atol=1e-15)


# ------------------------------------------------------------ expm (Sec. 2.1 step 2)
def _rand_nilpotent(n, c1, c2, c3=0.0):
    return exact.local_matrix(n, 1.0, 1.0, c1, c2, c3)


@pytest.mark.parametrize("n,c1,c2", [(3, 0.3, 0.0), (5, -0.8, 0.33), (5, 2.5, 1.0),
                                     (7, -3.7, 0.02), (7, 0.5, 2.0), (9, 1.5, 0.1)])
def test_expm_matches_exact_finite_series(n, c1, c2):
    """Nilpotent local operator: Pade S&S equals the exact finite Taylor sum."""
    Xf = _rand_nilpotent(n, c1, c2)
    X = exact.to_float(Xf)
    want = exact.to_float(exact.expm_nilpotent(Xf))
    got, m, s = ox.expm(X, return_ms=True)
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    assert err < 1e-13 * max(1.0, ox.norm1(X)), (m, s, err)


def test_expm_all_branches_vs_scipy():
    """Random dense matrices over norms that hit every (m, s) branch vs scipy.linalg.expm."""
    rng = np.random.default_rng(7)
    seen = set()
    for scale in [1e-3, 1e-2, 0.1, 0.5, 1.5, 4.0, 20.0, 200.0]:
        for d in (4, 9, 13, 16):
            A = rng.standard_normal((d, d))
            A *= scale / ox.norm1(A)
            got, m, s = ox.expm(A, return_ms=True)
            seen.add(m if s == 0 else (m, "s>0"))
            want = scipy.linalg.expm(A)
            rel = np.max(np.abs(got - want)) / np.max(np.abs(want))
            assert rel < 1e-12 * max(1.0, scale), (d, scale, m, s, rel)
    assert {3, 5, 7, 9, 13, (13, "s>0")} <= seen


def test_expm_closed_forms():
    t = 0.7
    R = ox.expm(np.array([[0.0, t], [-t, 0.0]]))
    assert np.allclose(R, [[math.cos(t), math.sin(t)], [-math.sin(t), math.cos(t)]], atol=1e-15)
    d = np.array([-30.0, -1.0, 0.0, 2.5])
    assert np.allclose(ox.expm(np.diag(d)), np.diag(np.exp(d)), rtol=1e-14, atol=0)
    J = np.diag(np.ones(3), 1) * 5.0
    assert np.allclose(ox.expm(J), [[1, 5, 12.5, 125 / 6], [0, 1, 5, 12.5], [0, 0, 1, 5], [0, 0, 0, 1]],
                       rtol=1e-14, atol=1e-14)


def test_pade_coefficients_are_the_pade_approximant():
    """p_m(x)/p_m(-x) matches e^x to order x^(2m) (definition of the [m/m] Pade approximant)."""
    for m in (3, 5, 7, 9, 13):
        b = [Fraction(v) for v in ox.pade_coefficients(m)]
        assert b[0] == 1
        x = 1e-2
        p = sum(float(c) * x ** j for j, c in enumerate(b))
        q = sum(float(c) * (-x) ** j for j, c in enumerate(b))
        assert abs(p / q - math.exp(x)) < 1e-15
        # ratio b_{j+1}/b_j = (m-j) / ((2m-j)(j+1))
        for j in range(m):
            assert abs(float(b[j + 1] / b[j]) - (m - j) / ((2 * m - j) * (j + 1))) < 1e-15


def test_lu_solve_matches_numpy():
    rng = np.random.default_rng(1)
    Q = rng.standard_normal((11, 11))
    P = rng.standard_normal((11, 11))
    assert np.allclose(ox.lu_solve(Q, P), np.linalg.solve(Q, P), rtol=1e-11, atol=1e-12)


def test_nilpotency_remark():
    """D_n^n = 0 exactly for any combination of derivative matrices (remark after Ex. 1)."""
    for n in (3, 5, 7):
        X = _rand_nilpotent(n, 0.37, -1.3, 0.2)
        P = X
        for _ in range(n - 1):
            P = exact.matmul(P, X)
        assert exact.is_zero(P)


# ------------------------------------------------------------ Examples 1 and 2
@pytest.mark.parametrize("nu", [-0.8, -0.3, 0.25, 0.5, 1.0, 1.7])
def test_example1_lax_wendroff_beam_warming(nu):
    g = golden("example1_advection_n3.json")
    p = wl.Problem("ex1", 3, 0.0, 3.0, wl.DIRICHLET, 3, 1.0, c1=nu)   # h = 1.5
    p = p.with_(c1=nu * p.h / p.dt)                                   # dt c1 / h = nu
    W = lmep.constant_weights(p)[:, 0, :]
    centre = [poly(c, nu) for c in g["centre_row"]]
    last = [poly(c, nu) for c in g["last_row"]]
    first = [poly(c, -nu) for c in g["last_row"]][::-1]                # mirror: x -> -x, nu -> -nu
    assert np.allclose(W[1], centre, rtol=0, atol=1e-14 * (1 + nu * nu))
    assert np.allclose(W[2], last, rtol=0, atol=1e-14 * (1 + nu * nu))
    assert np.allclose(W[0], first, rtol=0, atol=1e-14 * (1 + nu * nu))


@pytest.mark.parametrize("mu", [0.05, 0.3, 0.5, 0.66])
def test_example2_diffusion_rows(mu):
    g = golden("example2_diffusion.json")
    for n, key in ((3, "n3_centre_row"), (5, "n5_centre_row")):
        p = wl.Problem("ex2", 64, 0.0, 1.0, wl.PERIODIC, n, 1.0, c2=1.0)
        p = p.with_(dt=mu * p.h ** 2)
        w = lmep.constant_weights(p)[(n - 1) // 2, 0]
        want = [poly(c, mu) for c in g[key]]
        assert np.allclose(w, want, rtol=0, atol=2e-15)
    fr = [[Fraction(c) for c in row] for row in g["n5_centre_row_exact_fractions"]]
    assert np.allclose([[float(c) for c in r] for r in fr], g["n5_centre_row"], atol=1e-16)


# ------------------------------------------------------------ Theorem 1 (Sec. 2.2)
@pytest.mark.parametrize("n", [5, 7, 9, 13])
def test_theorem1_lagrange_semi_lagrangian(n):
    """Row r of exp(-a dt D_n) = Lagrange weights at x_r - a dt, any nodes, rows and CFL."""
    rng = np.random.default_rng(n)
    x = np.arange(n) + rng.uniform(-0.3, 0.3, n)           # non-uniform, well separated
    D = fornberg.derivative_matrices(x, 1)[1]
    for shift in (0.3, -1.6, 2.45):
        W = ox.expm(-shift * D)
        for r in range(n):
            want = lagrange_weights(x, x[r] - shift)
            assert np.max(np.abs(W[r] - want)) <= 1e-12 * np.sum(np.abs(want)) * n


@pytest.mark.parametrize("n,cfl", [(5, 1.0), (7, 2.0), (9, 3.0), (13, 4.0)])
def test_theorem1_integer_cfl_is_a_shift(n, cfl):
    """Lagrangian configuration (Sec. 4.1): integer CFL gives the identity shift.

    Sec. 4.1 reports an error floor near 1e-12 for this case; the tolerance is 5x that floor.
    """
    p = wl.Problem("adv", 64, 0.0, 1.0, wl.DIRICHLET, n, 1.0, c1=-1.0)
    p = p.with_(dt=cfl * p.h)
    W = lmep.constant_weights(p)[:, 0, :]
    k = int(cfl)
    for r in range(k, n):
        e = np.zeros(n)
        e[r - k] = 1.0
        assert np.max(np.abs(W[r] - e)) < 5e-12


# ------------------------------------------------------------ Theorem 2 and weight sums
def gaussian_moments(mean, var, kmax):
    """E[(mean + sqrt(var) Z)^k], Z ~ N(0,1), by M_k = mean M_{k-1} + (k-1) var M_{k-2}."""
    M = [1.0, mean]
    for k in range(2, kmax + 1):
        M.append(mean * M[-1] + (k - 1) * var * M[-2])
    return M


@pytest.mark.parametrize("n,cfl,mu", [(5, 1.0, 0.2), (7, -2.3, 0.05), (9, 0.4, 0.6), (11, 3.1, 0.3)])
@pytest.mark.parametrize("recentre", [True, False])
def test_theorem2_coupled_exactness(n, cfl, mu, recentre):
    """w . p(x_S) = (e^{dt L} p)(x_r) = E[p(x_r - a dt + sqrt(2 nu dt) Z)] for deg p < n.

    Units with h = dt = 1, so a = cfl and nu = mu; moments of (x - x_r) keep the sums small.
    """
    p = wl.Problem("ad", 50, 0.0, 49.0, wl.DIRICHLET, n, 1.0, c1=-cfl, c2=mu)
    W = lmep.constant_weights(p, recentre=recentre)[:, 0, :]
    xs = np.arange(n, dtype=np.float64)
    for r in range(n):
        M = gaussian_moments(-cfl, 2 * mu, n - 1)
        for deg in range(n):
            got = W[r] @ (xs - r) ** deg
            tol = 1e-12 * np.sum(np.abs(W[r]) * np.abs(xs - r) ** deg) * (1 if recentre else 30)
            assert abs(got - M[deg]) <= max(tol, 1e-15), (r, deg)


def test_weight_sums_and_reaction_factor():
    """sum w_lin = e^{c0 dt} (Thm. 2 proof); sum of row dt^k phi_k = dt^k / k! (Sec. 3)."""
    p = wl.Problem("r", 40, 0.0, 1.0, wl.PERIODIC, 9, 0.0, c0=0.7, c1=-1.2, c2=0.01, scheme="etdrk2")
    p = p.with_(dt=0.6 * p.h)
    W = lmep.constant_weights(p)
    assert abs(np.sum(W[4, 0]) - math.exp(0.7 * p.dt)) < 1e-13
    p0 = p.with_(c0=0.0)
    W0 = lmep.constant_weights(p0)
    for r in range(p.n):
        assert abs(np.sum(W0[r, 0]) - 1.0) < 1e-12
        assert abs(np.sum(W0[r, 1]) - p.dt) < 1e-12 * p.dt
        assert abs(np.sum(W0[r, 2]) - p.dt ** 2 / 2) < 1e-12 * p.dt ** 2


# ------------------------------------------------------------ phi via augmented (Sec. 3.1)
@pytest.mark.parametrize("n,c1,c2,c3", [(3, -0.7, 0.2, 0.0), (5, 1.3, 0.4, 0.0), (7, 0.2, 0.0, -0.05)])
def test_phi_rows_match_taylor(n, c1, c2, c3):
    """Row r of dt^k phi_k(X) = dt^k sum_j X^j/(j+k)!, finite because X is nilpotent."""
    dt = 0.37
    Xf = exact.local_matrix(n, dt, 1.0, c1, c2, c3)
    X = exact.to_float(Xf)
    p = wl.Problem("phi", 30, 0.0, 29.0, wl.DIRICHLET, n, dt, c1=c1, c2=c2, c3=c3, scheme="etdrk2")
    # phi_k by the finite Taylor series in exact arithmetic
    phis = []
    for k in range(3):
        acc = [[Fraction(0)] * n for _ in range(n)]
        term = [[Fraction(int(i == j)) for j in range(n)] for i in range(n)]
        for j in range(n):
            f = Fraction(1, math.factorial(j + k))
            acc = [[acc[a][b] + f * term[a][b] for b in range(n)] for a in range(n)]
            term = exact.matmul(term, Xf)
        phis.append(exact.to_float(acc) * dt ** k)
    for r in range(n):
        got = lmep.harvest(p, X, r)
        for k in range(3):
            assert np.max(np.abs(got[k] - phis[k][r])) <= 1e-13 * max(dt ** k, np.max(np.abs(phis[k][r])))


def test_row_restricted_equals_paper_block_form():
    """The (n+p) row-restricted matrix and the paper's s n x s n block form give the same rows."""
    p = wl.kdv(N=128, n=11).with_(dt=0.2)
    X = operator.local_matrix(p.with_(dt=0.2))
    E = ox.expm(operator.augmented_block(X, p.dt, 3))
    for r in range(p.n):
        got = lmep.harvest(p, X, r)
        for k in range(3):
            want = E[r, k * p.n:(k + 1) * p.n]
            assert np.max(np.abs(got[k] - want)) < 1e-13 * max(1.0, np.max(np.abs(want)))


# ------------------------------------------------------------ n = N (Sec. 2 global exponential)
@pytest.mark.parametrize("N", [5, 8, 12])
def test_n_equals_N_is_the_global_exponential(N):
    """With one stencil covering the grid, the LMEP update is the dense exp(dt D) (Sec. 2)."""
    p = wl.Problem("glob", N, 0.0, 1.0, wl.DIRICHLET, N, 0.0, c1=-1.0, c2=0.02)
    p = p.with_(dt=0.5 * p.h)
    D1 = exact.to_float(exact.lagrange_D(range(N), 1)) / p.h
    D2 = exact.to_float(exact.lagrange_D(range(N), 2)) / p.h ** 2
    G = scipy.linalg.expm(p.dt * (-1.0 * D1 + 0.02 * D2))
    u = np.random.default_rng(0).standard_normal(N)
    got = lmep.step(p, lmep.constant_weights(p), u)
    assert np.max(np.abs(got[1:-1] - (G @ u)[1:-1])) < 1e-11 * np.max(np.abs(G @ u))


# ------------------------------------------------------------ periodic Fourier decay (config 1)
@pytest.mark.parametrize("k", [1, 5, 17])
def test_periodic_mode_evolves_by_symbol(k):
    """Circulant update: cos(k x) after m steps is Re(G(kh)^m e^{ikx}) exactly."""
    p = wl.advection_diffusion(N=64, n=5, steps=7)
    x = p.nodes()
    W = lmep.constant_weights(p)
    G = lmep.amplification(W[2, 0], 2, np.array([k * p.h]))[0]
    got = lmep.run(p, np.cos(k * x), 7)
    want = np.real(G ** 7 * np.exp(1j * k * x))
    assert np.max(np.abs(got - want)) < 1e-13
    # the symbol approaches the exact decay exp(-(i c k + nu k^2) dt) as kh -> 0
    if k == 1:
        assert abs(G - np.exp(-(1j * k + 0.01 * k * k) * p.dt)) < 1e-6


def config1_exact(p, t):
    """e^{-nu t} sin(x - ct) + Gaussian wrapped over periodic shifts (Sec. 4.2, K = 2)."""
    x = p.nodes()
    nu, c = p.c2, -p.c1
    u = np.exp(-nu * t) * np.sin(x - c * t)
    for s in range(-2, 3):
        z = x - math.pi - c * t - 2 * math.pi * s
        u += np.exp(-20 * z ** 2 / (1 + 80 * nu * t)) / math.sqrt(1 + 80 * nu * t)
    return u


def test_config1_converges_in_stencil_size():
    """Sec. 4.2: at fixed N and dt the error vs the wrapped exact solution falls spectrally in n."""
    errs = []
    for n in (5, 7, 9, 11):
        p = wl.advection_diffusion(N=256, n=n, steps=100)
        u = lmep.run(p, wl.advection_diffusion_ic(p))
        errs.append(np.max(np.abs(u - config1_exact(p, p.dt * p.steps))))
    assert errs[0] < 1e-4 and errs[-1] < 5e-12, errs
    assert all(errs[i + 1] < errs[i] / 25 for i in range(3)), errs


# ------------------------------------------------------------ Neumann reading
def test_neumann_equals_mirrored_periodic():
    N = 33
    p = wl.allen_cahn(N, bc=wl.NEUMANN, n=7, scheme="etdrk2", steps=3, dt=0.05, eps2=0.002)
    u0 = wl.allen_cahn_ic(N, 5)
    got = lmep.run(p, u0)
    M = 2 * (N - 1)
    q = p.with_(N=M, bc=wl.PERIODIC, b=p.a + 2 * (p.b - p.a))   # same h
    assert abs(q.h - p.h) < 1e-15
    um = np.concatenate([u0, u0[-2:0:-1]])
    want = lmep.run(q, um)[:N]
    assert np.max(np.abs(got - want)) < 1e-14


# ------------------------------------------------------------ ETD steppers (Sec. 3)
def test_etd_orders_on_pure_reaction():
    """L = 0: ETD1 is forward Euler (order 1), ETDRK2 is Heun (order 2) for u' = u - u^3."""
    u0 = np.array([0.1, -0.5, 0.9, 0.3, 0.05])
    T = 1.0

    def exact_sol(u, t):
        return u * math.exp(t) / np.sqrt(1 + u * u * (math.exp(2 * t) - 1))

    for scheme, order in (("etd1", 1.0), ("etdrk2", 2.0)):
        errs = []
        for m in (20, 40, 80):
            p = wl.Problem("rx", 5, 0.0, 1.0, wl.PERIODIC, 3, T / m, scheme=scheme,
                           nonlin="allen_cahn")
            u = lmep.run(p, u0, m)
            errs.append(np.max(np.abs(u - exact_sol(u0, T))))
        rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
        assert all(abs(r - order) < 0.15 for r in rates), (scheme, rates)


def test_etd_linear_reaction_is_exact():
    """u' = c0 u + f with constant f: ETD1 is exact (u+ = e^{c0 dt} u + dt phi_1 f)."""
    c0, dt = -3.0, 0.3
    p = wl.Problem("lin", 5, 0.0, 1.0, wl.PERIODIC, 3, dt, c0=c0, scheme="etdrk2", nonlin="allen_cahn")
    W = lmep.constant_weights(p)
    assert abs(W[1, 0, 1] - math.exp(c0 * dt)) < 1e-15
    assert abs(W[1, 1, 1] - (math.exp(c0 * dt) - 1) / c0) < 1e-15
    assert abs(W[1, 2, 1] - (math.exp(c0 * dt) - 1 - c0 * dt) / c0 ** 2) < 1e-15


# ------------------------------------------------------------ KdV (Sec. 4.3.2)
def test_kdv_single_soliton_speed():
    """2 k^2 sech^2(k (x - 4 k^2 t - x0)) solves u_t + 6 u u_x + u_xxx = 0."""
    kap, x0 = 0.6, -5.0
    p = wl.kdv(N=200, n=11, L=25.0, mu3=0.05, steps=0)
    steps = int(round(1.5 / p.dt))
    x = p.nodes()
    sol = lambda t: 2 * kap ** 2 / np.cosh(kap * (x - 4 * kap ** 2 * t - x0)) ** 2
    u = lmep.run(p, sol(0.0), steps)
    err = np.max(np.abs(u - sol(steps * p.dt)))
    moved = np.max(np.abs(sol(steps * p.dt) - sol(0.0)))
    assert err < 2e-3 and moved > 0.2, (err, moved)
    # invariants of the semi-discrete flow: mass and energy drift stay small
    u0 = sol(0.0)
    assert abs(np.sum(u) - np.sum(u0)) * p.h < 1e-8
    assert abs(np.sum(u ** 2) - np.sum(u0 ** 2)) * p.h < 1e-3


# ------------------------------------------------------------ frozen-velocity Burgers
@pytest.mark.parametrize("centring", [False, True])
def test_frozen_weights_are_departure_point_lagrange(centring):
    """nu = 0: each point's weights are the Lagrange weights at x_i - u_i dt on its window."""
    N = 41
    u = wl.burgers_ic(N, seed=2)
    p = wl.burgers(N=N, n=7, cfl=2.5, nu=0.0, departure_centring=centring, steps=1)
    x = p.nodes()
    for i in range(1, N - 1):
        idx, r, w = lmep.point_weights(p, u, i)
        want = lagrange_weights(x[idx], x[i] - u[i] * p.dt)
        assert np.max(np.abs(w[0] - want)) <= 1e-11 * np.sum(np.abs(want))
        if centring:
            lo, hi = x[idx[0]], x[idx[-1]]
            assert lo - 0.5 * p.h <= x[i] - u[i] * p.dt <= hi + 0.5 * p.h or idx[0] == 0 or idx[-1] == N - 1


def test_recentring_identity():
    """Row r of exp(X(u)) = row r-k of exp(X(u - k h/dt)): both are Thm. 2's Gaussian weights."""
    p = wl.burgers(N=1001, n=13, cfl=3.7, nu=1e-6, steps=1)
    u_i = 1.0
    D = operator.unit_D(p.n)
    X = operator.local_matrix(p, u_i, D)
    k = grid.departure_shift(u_i, p.dt, p.h, p.n)
    assert k == 3
    Xk = operator.local_matrix(p, u_i - k * p.h / p.dt, D)
    assert np.max(np.abs(Xk - (X + k * D[1]))) < 1e-13 * np.max(np.abs(X))
    E, Ek = ox.expm(X), ox.expm(Xk)
    assert ox.norm1(Xk) < ox.norm1(X) / 5
    for r in range(k, p.n):
        assert np.max(np.abs(E[r] - Ek[r - k])) < 1e-11 * np.sum(np.abs(E[r]))
        assert np.max(np.abs(lmep.exp_row(p, r, u_i, D)[0] - Ek[r - k])) < 1e-13 * np.sum(np.abs(E[r]))


def test_stability_precheck_closed_form():
    """Centred n = 5 diffusion: G(pi) = 1 - 16 mu/3 + 8 mu^2 from Example 2's row; mu* = 2/3."""
    for mu in (0.2, 0.5, 2 / 3, 0.8):
        p = wl.Problem("d", 64, 0.0, 1.0, wl.PERIODIC, 5, 0.0, c2=1.0)
        p = p.with_(dt=mu * p.h ** 2)
        w = lmep.constant_weights(p)[2, 0]
        G = lmep.amplification(w, 2, np.array([np.pi]))[0]
        assert abs(G - (1 - 16 * mu / 3 + 8 * mu * mu)) < 1e-13
    assert abs(1 - 16 * (2 / 3) / 3 + 8 * (2 / 3) ** 2 - 1.0) < 1e-15


# ------------------------------------------------------------ ETDRK4 (Sec. 3)
def _phi(k, z):
    """phi_k(z) by the paper's recursion phi_0 = e^z, phi_{j+1} = (phi_j - 1/j!) / z (z away from 0)."""
    v = math.exp(z)
    for j in range(k):
        v = (v - 1.0 / math.factorial(j)) / z
    return v


def test_etdrk4_is_classical_rk4_without_linear_part_and_order4_with_it():
    """L = 0: the stages a, b, c and the alpha, beta, gamma combination reduce to the classical
    fourth-order Runge-Kutta method (phi_k(0) = 1/k!); with L = c0 it keeps order 4.  Both against
    the closed-form solution of u' = (1 + c0) u - u^3 (a Bernoulli equation)."""
    u0 = np.array([0.1, -0.5, 0.9, 0.3, 0.05])
    T = 1.0
    for c0 in (0.0, -2.0):
        a = 1.0 + c0
        exact_sol = u0 * math.exp(a * T) / np.sqrt(1 + u0 * u0 * (math.exp(2 * a * T) - 1) / a)
        errs = []
        for m in (10, 20, 40, 80):
            p = wl.Problem("rx", 5, 0.0, 1.0, wl.PERIODIC, 3, T / m, c0=c0, scheme="etdrk4", nonlin="allen_cahn")
            errs.append(np.max(np.abs(lmep.run(p, u0, m) - exact_sol)))
        rates = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
        assert all(abs(r - 4.0) < 0.15 for r in rates), (c0, rates)
    # L = 0, one step: exactly the classical RK4 weights 1/6, 1/3, 1/3, 1/6
    dt = 0.3
    f = lambda v: v - v ** 3
    k1 = f(u0)
    k2 = f(u0 + dt / 2 * k1)
    k3 = f(u0 + dt / 2 * k2)
    k4 = f(u0 + dt * k3)
    rk4 = u0 + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    p = wl.Problem("rx", 5, 0.0, 1.0, wl.PERIODIC, 3, dt, scheme="etdrk4", nonlin="allen_cahn")
    assert np.max(np.abs(lmep.run(p, u0, 1) - rk4)) < 1e-15


def test_etdrk4_rows_closed_forms():
    """Pure reaction L = c0: the harvested rows are scalars, dt^k phi_k(dt c0) (k <= 3) at dt and
    e^{c0 dt/2}, (dt/2) phi_1(c0 dt/2) at dt/2; the rows of dt alpha, dt beta, dt gamma are
    dt (phi_1 - 3 phi_2 + 4 phi_3), dt (2 phi_2 - 4 phi_3), dt (4 phi_3 - phi_2) (Sec. 3)."""
    c0, dt = -3.0, 0.3
    z = c0 * dt
    p = wl.Problem("lin", 5, 0.0, 1.0, wl.PERIODIC, 3, dt, c0=c0, scheme="etdrk4", nonlin="allen_cahn")
    W = lmep.constant_weights(p)
    for k in range(4):
        assert abs(W[1, k, 1] - dt ** k * _phi(k, z)) < 1e-15 * max(1.0, dt ** k), k
        assert abs(W[1, k, 0]) < 1e-15 and abs(W[1, k, 2]) < 1e-15
    Wh = lmep.half_step_weights(p)
    assert abs(Wh[1, 0, 1] - math.exp(z / 2)) < 1e-15
    assert abs(Wh[1, 1, 1] - dt / 2 * _phi(1, z / 2)) < 1e-15
    al, be, ga = lmep.etdrk4_coefficient_rows(p, W)
    p1, p2, p3 = _phi(1, z), _phi(2, z), _phi(3, z)
    assert abs(al[1, 1] - dt * (p1 - 3 * p2 + 4 * p3)) < 1e-14
    assert abs(be[1, 1] - dt * (2 * p2 - 4 * p3)) < 1e-14
    assert abs(ga[1, 1] - dt * (4 * p3 - p2)) < 1e-14
    # Kassam & Trefethen's explicit forms of the same three functions
    assert abs(al[1, 1] - dt * (-4 - z + math.exp(z) * (4 - 3 * z + z * z)) / z ** 3) < 1e-13
    assert abs(be[1, 1] - dt * 2 * (2 + z + math.exp(z) * (z - 2)) / z ** 3) < 1e-13
    assert abs(ga[1, 1] - dt * (-4 - 3 * z - z * z + math.exp(z) * (4 - z)) / z ** 3) < 1e-13


def test_etdrk4_weight_sums_are_rk4_weights():
    """c0 = 0: every row of dt^k phi_k(X) sums to dt^k / k! (constants are annihilated), so the rows
    of dt alpha, dt beta, dt gamma sum to dt/6, dt/3, dt/6, the classical weights."""
    p = wl.Problem("r", 40, 0.0, 1.0, wl.DIRICHLET, 11, 0.0, c1=-0.8, c2=0.02, c3=-0.001, scheme="etdrk4",
                   nonlin="allen_cahn")
    p = p.with_(dt=0.9 * p.h)
    W = lmep.constant_weights(p)
    al, be, ga = lmep.etdrk4_coefficient_rows(p, W)
    for r in range(p.n):       # to the rounding of the sums: 1e-13 of the rows' absolute sums
        for row, want in ((W[r, 3], p.dt ** 3 / 6), (al[r], p.dt / 6), (be[r], p.dt / 3), (ga[r], p.dt / 6)):
            assert abs(np.sum(row) - want) < 1e-13 * np.sum(np.abs(row)), r


def test_etdrk4_phi3_rows_match_taylor_and_block_form():
    """Row r of dt^3 phi_3(X) = dt^3 sum_j X^j/(j+3)! (finite: X nilpotent) and equals the paper's
    s n x s n block form with s = 4 (Sec. 3.1)."""
    n, c1, c2, c3, dt = 5, 1.3, 0.4, -0.05, 0.37
    Xf = exact.local_matrix(n, dt, 1.0, c1, c2, c3)
    X = exact.to_float(Xf)
    p = wl.Problem("phi", 30, 0.0, 29.0, wl.DIRICHLET, n, dt, c1=c1, c2=c2, c3=c3, scheme="etdrk4")
    acc = [[Fraction(0)] * n for _ in range(n)]
    term = [[Fraction(int(i == j)) for j in range(n)] for i in range(n)]
    for j in range(n):
        f = Fraction(1, math.factorial(j + 3))
        acc = [[acc[a][b] + f * term[a][b] for b in range(n)] for a in range(n)]
        term = exact.matmul(term, Xf)
    phi3 = exact.to_float(acc) * dt ** 3
    E = ox.expm(operator.augmented_block(X, dt, 4))
    for r in range(n):
        got = lmep.harvest(p, X, r)
        assert np.max(np.abs(got[3] - phi3[r])) <= 1e-13 * max(dt ** 3, np.max(np.abs(phi3[r])))
        for k in range(4):
            want = E[r, k * n:(k + 1) * n]
            assert np.max(np.abs(got[k] - want)) < 1e-13 * max(1.0, np.max(np.abs(want)))


def test_etdrk4_without_nonlinearity_is_the_exponential_step():
    p = wl.allen_cahn(64, bc=wl.NEUMANN, n=9, scheme="etdrk4", steps=3, mu=0.8).with_(nonlin="none")
    u0 = np.cos(np.pi * p.nodes()) + 0.2 * np.sin(5 * p.nodes())
    lin = p.with_(scheme="linear")
    # the same exponential rows (augmented harvest vs the re-centred plain one, both FP64 Pade)
    assert np.max(np.abs(lmep.run(p, u0) - lmep.run(lin, u0))) < 1e-12


def test_burgers_etd_nonlinearity_is_minus_u_ux():
    """N(u) = -u u_x with u_x from row r of D^(1): exact for a quadratic u = x^2 (n >= 3)."""
    p = wl.burgers_etd(N=64, n=7).with_(bc=wl.DIRICHLET, a=0.0, b=1.0)
    x = p.nodes()
    got = lmep.nonlinear(p, x ** 2)
    assert np.max(np.abs(got - (-(x ** 2) * 2 * x))) < 1e-12


# ------------------------------------------------------------ high-CFL one-sided advection (Sec. 4.1)
def _lagrange(z, n):
    return np.array([np.prod([(z - m) / (j - m) for m in range(n) if m != j]) for j in range(n)])


@pytest.mark.parametrize("n", [5, 9, 13])
def test_one_sided_rows_are_departure_point_interpolation(n):
    """Thm. 1 with a fully upwind window: the harvested row (class (n-1)/2 + k, k = (n-1)/2) is the
    Lagrange interpolation at the departure point, r - nu in window coordinates."""
    for sigma in (0.0, 0.3, 0.5):
        p = wl.advection(N=64, n=n, sigma=sigma)
        W = lmep.constant_weights(p)
        r = (n - 1) // 2 + p.window_shift
        want = _lagrange(r - p.meta["nu"], n)
        assert np.max(np.abs(W[r, 0] - want)) < 1e-12 * max(1.0, np.max(np.abs(want)))


@pytest.mark.parametrize("n", [7, 11])
def test_one_sided_lagrangian_transport_is_exact(n):
    """Integer Courant numbers nu = (n+1)/2: after 100 periods the profile is back exactly (the row is a
    unit vector: a shift by nu nodes)."""
    p = wl.advection(N=96, n=n, sigma=0.0)
    u = lmep.run(p, wl.advection_ic(p))
    assert np.max(np.abs(u - wl.advection_exact(p, p.steps * p.dt))) < 1e-12


def test_one_sided_spectral_convergence_and_amplification():
    """nu = (n+1)/2 - 1/2 (non-Lagrangian): the error after 100 periods falls by at least 5x per width
    step, and no Fourier mode is amplified, max |G(theta)| <= 1 (up to rounding), |G(0)| = 1."""
    errs = []
    th = np.linspace(-np.pi, np.pi, 1001)
    for n in (7, 9, 11, 13):
        p = wl.advection(N=128, n=n, sigma=0.5)
        u = lmep.run(p, wl.advection_ic(p))
        errs.append(np.max(np.abs(u - wl.advection_exact(p, p.steps * p.dt))))
        W = lmep.constant_weights(p)
        r = (n - 1) // 2 + p.window_shift
        G = np.abs(lmep.amplification(W[r, 0], r, th))
        assert np.max(G) <= 1.0 + 1e-12 and abs(G[500] - 1.0) < 1e-13
    assert all(errs[i + 1] < errs[i] / 5 for i in range(3)), errs


# ------------------------------------------------------------ non-uniform (Chebyshev) grids (Sec. 4.3.3)
from oracle import nodes as onodes  # noqa: E402


def _cheb_matrix(x):
    """Derivative of the polynomial interpolant at Chebyshev-Gauss-Lobatto points x_0 < ... < x_{N-1}:
    barycentric weights w_j = (-1)^j (halved at both ends), D_ij = (w_j / w_i) / (x_i - x_j) for i != j,
    D_ii = -sum_{j != i} D_ij (the textbook spectral differentiation matrix)."""
    N = len(x)
    w = np.array([(-1.0) ** j * (0.5 if j in (0, N - 1) else 1.0) for j in range(N)])
    D = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            if i != j:
                D[i, j] = (w[j] / w[i]) / (x[i] - x[j])
        D[i, i] = -np.sum(D[i])
    return D


@pytest.mark.parametrize("N", [7, 11, 15])
def test_nodes_n_equals_N_is_the_global_chebyshev_exponential(N):
    """One window covering a Chebyshev grid: the harvested rows are rows of the dense exp(dt L_N)
    with L_N built from the spectral differentiation matrix (Sec. 4.3.3 avoids exactly this
    global exponential for large N)."""
    x = onodes.chebyshev_nodes(N)
    p = wl.Problem("cheb", N, -1.0, 1.0, wl.DIRICHLET, N, 0.02, c1=-0.6, c2=0.01)
    D = _cheb_matrix(x)
    G = scipy.linalg.expm(p.dt * (p.c1 * D + p.c2 * D @ D))
    W = onodes.weights(p, x)
    for i in range(1, N - 1):
        assert np.max(np.abs(W[i, 0] - G[i])) < 1e-11 * max(1.0, np.max(np.abs(G[i]))), i


def test_nodes_uniform_grid_matches_row_classes():
    """On uniform nodes the per-point weights are the uniform oracle's row classes."""
    p = wl.Problem("u", 41, -1.0, 1.0, wl.DIRICHLET, 9, 0.0, c1=-0.4, c2=3e-3, scheme="etdrk2",
                   nonlin="allen_cahn")
    p = p.with_(dt=0.7 * p.h)
    x = p.nodes()
    Wn = onodes.weights(p, x)
    Wc = lmep.constant_weights(p)
    for i in range(1, p.N - 1):
        idx, r = onodes.window(p, i)
        assert np.max(np.abs(Wn[i] - Wc[r])) < 1e-12 * max(1.0, np.max(np.abs(Wc[r]))), i


@pytest.mark.parametrize("scheme", ["linear", "etd1", "etdrk2", "etdrk4"])
def test_nodes_constants_and_steady_states(scheme):
    """Rows of exp(dt L) sum to 1 on any nodes (constants are annihilated by D^(k)); u = 1 with walls
    at 1 is a steady state of Allen-Cahn (N(1) = 0) under every scheme."""
    x = onodes.chebyshev_nodes(40)
    p = wl.Problem("c", 40, -1.0, 1.0, wl.DIRICHLET, 9, 1e-3, c2=0.01, scheme=scheme,
                   nonlin="none" if scheme == "linear" else "allen_cahn", bc_lo=1.0, bc_hi=1.0, steps=3)
    W = onodes.weights(p, x)
    assert np.max(np.abs(W[:, 0].sum(axis=1) - 1.0)) < 1e-11
    u = onodes.run(p, x, np.ones(40))
    assert np.max(np.abs(u - 1.0)) < 1e-11
