"""Wide stencils (odd n = 17 .. 25, the widths of the paper's one-sided study, Sec. 4.1) of the
constant-coefficient linear scheme, through the C ABI.

* Rows: the FP64 row of a class equals the exact rational row e_r^T exp(X) (the finite Taylor sum of
  the nilpotent local matrix of oracle.exact, no factorisation involved) within 1e-12 of its l1
  norm, the FP32 row within 1e-6.  For these widths the oracle's Pade of the rounded local matrix is
  itself off, by up to 1e-7 at n = 25 (the derivative matrices of wide windows have large norms), so
  the exact rows decide, as they do for the FP64 rows of the nine-instance benchmark set
  (tests/test_readings_exact.py pins that gap, and the factorisation, at these widths).
* One-sided advection for 100 periods (N = 256, nu = (n+1)/2 - 1/2): the GPU trajectory equals the
  oracle's banded step with the exact row within 1e-12 K (FP64) / 1e-5 K (FP32 form, 20 steps), and
  its error against the exact solution stays below 1e-7 (it grows at n = 25: the Runge onset the
  paper reports).
* The Fourier symbol of a harvested row against the oracle's.
* Several tiles with a ragged end, both signs of the window shift and a diffusive, dispersive,
  reactive operator, against the oracle's step with the exact rows.
* Configurations outside the wide path are refused before anything is launched.
"""
from fractions import Fraction
from functools import lru_cache

import numpy as np
import pytest

import workloads as wl
from oracle import exact
from oracle import lmep as olmep

from lmep_testutil import grid_of, op_of, rel_linf, tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = ["fp64", "mixed"]
WIDE = [17, 19, 21, 23, 25]


@pytest.fixture(scope="module")
def L():
    import paper_2603_15964_gb300 as L
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return L


@pytest.fixture(scope="module")
def H(L):
    return L.Handle()


def exact_row(p, r):
    """Row r of exp(X), X = dt (c1 D1 + c2 D2 + c3 D3) in exact rational arithmetic (finite series of
    the nilpotent X), times e^{c0 dt}."""
    X = exact.local_matrix(p.n, p.dt, p.h, p.c1, p.c2, p.c3)
    v = [Fraction(int(j == r)) for j in range(p.n)]
    acc = v[:]
    for k in range(1, p.n + 1):
        v = [sum((v[i] * X[i][j] for i in range(p.n)), Fraction(0)) / k for j in range(p.n)]
        if k == p.n:
            assert all(x == 0 for x in v)          # e_r^T X^n = 0 exactly
            break
        acc = [acc[j] + v[j] for j in range(p.n)]
    return np.exp(p.c0 * p.dt) * np.array([float(x) for x in acc])


def used_class(p):
    return (p.n - 1) // 2 + p.window_shift


def exact_weights(p):
    """W[n][1][n] holding only the exact row of the class every point of a periodic grid takes."""
    W = np.zeros((p.n, 1, p.n))
    W[used_class(p), 0] = exact_row(p, used_class(p))
    return W


def harvest(L, H, p, precision):
    W = torch.empty(p.n, 1, p.n, dtype=L.state_dtype(precision), device="cuda")
    L.lmep_harvest_weights(H, grid_of(p), op_of(p), p.dt, 0, None, W, precision)
    L.lmep_sync_status(H)
    return W


def run_gpu(L, H, p, W, u0, precision, steps):
    u = torch.tensor(u0, dtype=L.state_dtype(precision), device="cuda")
    L.lmep_step(H, grid_of(p), op_of(p), "linear", "none", p.dt, W, u, torch.empty_like(u), steps, precision)
    L.lmep_sync_status(H)
    return u.cpu().numpy().astype(np.float64)


def general(n, N=3001, shift=0):
    """Periodic u_t = c0 u - u_x + c2 u_xx + c3 u_xxx at CFL 0.8, diffusion number 0.05."""
    h = 2.0 / N
    p = wl.Problem("adv", N, -1.0, 1.0, wl.PERIODIC, n, 0.0, c0=-0.3, c1=-1.0, c2=0.0625 * h, c3=1e-3 * h * h,
                   window_shift=shift, steps=6)
    return p.with_(dt=0.8 * p.h)


@lru_cache(maxsize=None)
def one_sided_reference(n):
    p = wl.advection(N=256, n=n, sigma=0.5, periods=100)
    W = exact_weights(p)
    u = wl.advection_ic(p)
    for _ in range(p.steps):
        u = olmep.step(p, W, u)
    return u


# ------------------------------------------------------------------ rows
@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("n", WIDE)
@pytest.mark.parametrize("case", ["one_sided", "general"])
def test_rows_equal_the_exact_rows(L, H, precision, n, case):
    """Pure advection: every class, the extrapolating edge ones included (l1 norms up to 1e16 at
    n = 25). With diffusion and dispersion, the classes within four of the centre, which windows
    shifted by up to four points take (l1 norms below 2.4): the edge classes of such an operator are
    ill-conditioned (l1 norms of 3e4 and more at n = 25)."""
    hs = (n - 1) // 2
    if case == "one_sided":
        p = wl.advection(N=256, n=n, sigma=0.5)
        classes = sorted({used_class(p), hs, 0, n - 1})
    else:
        p = general(n)
        classes = range(hs - 4, hs + 5)
    W = harvest(L, H, p, precision).cpu().numpy().astype(np.float64)[:, 0]
    bound = 1e-12 if precision == "fp64" else 1e-6
    for r in classes:
        want = exact_row(p, r)
        assert np.max(np.abs(W[r] - want)) <= bound * np.sum(np.abs(want)), r


# ------------------------------------------------------------------ trajectories
@pytest.mark.parametrize("n", [17, 21, 25])
def test_one_sided_hundred_periods(L, H, n):
    p = wl.advection(N=256, n=n, sigma=0.5, periods=100)
    W = harvest(L, H, p, "fp64")
    u0 = wl.advection_ic(p)
    got = run_gpu(L, H, p, W, u0, "fp64", p.steps)
    assert rel_linf(got, one_sided_reference(n)) <= tol("fp64") * p.steps
    assert np.max(np.abs(got - wl.advection_exact(p, p.steps * p.dt))) <= 1e-7


@pytest.mark.parametrize("n", [17, 25])
def test_one_sided_fp32_form(L, H, n):
    p = wl.advection(N=256, n=n, sigma=0.5, periods=100)
    W = harvest(L, H, p, "mixed")
    u0 = wl.advection_ic(p).astype(np.float32).astype(np.float64)
    got = run_gpu(L, H, p, W, u0, "mixed", 20)
    u = u0
    Wx = exact_weights(p)
    for _ in range(20):
        u = olmep.step(p, Wx, u)
    assert rel_linf(got, u) <= tol("mixed") * 20


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("n,N,shift,pure", [(17, 2049, 0, False), (19, 4100, 4, False), (21, 3001, -3, False),
                                            (25, 1025, 2, False), (25, 2050, 12, True), (23, 4097, 11, True)])
def test_tiles_and_shifts(L, H, precision, n, N, shift, pure):
    """Ragged last tiles (2048 points in the FP32 form, 1024 in FP64), shifted windows of the diffusive,
    dispersive, reactive operator, and fully upwind windows of pure advection at the Courant number
    (n+1)/2 - 1/2 of Sec. 4.1, which puts the departure point mid-window."""
    p = general(n, N=N, shift=shift)
    if pure:
        p = p.with_(c0=0.0, c2=0.0, c3=0.0, dt=((n + 1) / 2 - 0.5) * p.h)
    W = harvest(L, H, p, precision)
    x = p.nodes()
    u0 = np.sin(np.pi * x) + 0.3 * np.cos(3 * np.pi * x)
    if precision == "mixed":
        u0 = u0.astype(np.float32).astype(np.float64)
    got = run_gpu(L, H, p, W, u0, precision, p.steps)
    u = u0
    Wx = exact_weights(p)
    for _ in range(p.steps):
        u = olmep.step(p, Wx, u)
    assert rel_linf(got, u) <= tol(precision) * p.steps


# ------------------------------------------------------------------ symbol
@pytest.mark.parametrize("n", [17, 25])
def test_amplification_of_a_wide_row(L, H, n):
    p = wl.advection(N=256, n=n, sigma=0.5)
    W = harvest(L, H, p, "fp64")
    r = used_class(p)
    w = W[r, 0].contiguous()
    th = np.linspace(-np.pi, np.pi, 513)
    G = torch.empty(len(th), 2, dtype=torch.float64, device="cuda")
    L.lmep_amplification(w, r, torch.tensor(th, device="cuda"), G)
    got = G.cpu().numpy()
    want = olmep.amplification(exact_row(p, r), r, th)
    assert np.max(np.abs(got[:, 0] + 1j * got[:, 1] - want)) <= 1e-12 * np.sum(np.abs(exact_row(p, r)))
    assert np.max(np.hypot(got[:, 0], got[:, 1])) <= 1.0 + 1e-12       # sigma = 1/2: stable


# ------------------------------------------------------------------ refused
def test_outside_the_wide_path_is_refused(L, H):
    p = general(17)
    W = harvest(L, H, p, "fp64")
    u = torch.ones(p.N, dtype=torch.float64, device="cuda")
    walls = p.with_(bc=wl.DIRICHLET)
    with pytest.raises(L.LmepError) as e:                   # walled grids: not built for n > 15
        L.lmep_step(H, grid_of(walls), op_of(walls), "linear", "none", p.dt, W, u, torch.empty_like(u), 1, "fp64")
    assert e.value.status == 5
    q = wl.allen_cahn(3001, n=17, scheme="etd1")
    Wq = torch.empty(17, 2, 17, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LmepError) as e:                   # phi-rows: not built for n > 15
        L.lmep_harvest_weights(H, grid_of(q), op_of(q), q.dt, 1, None, Wq, "fp64")
    assert e.value.status == 5
    b = wl.burgers(N=4001, n=17, cfl=2.0)
    v = torch.ones(b.N, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LmepError) as e:                   # frozen velocity: not built for n > 15
        L.lmep_step(H, grid_of(b), op_of(b), "linear", "none", b.dt, None, v, torch.empty_like(v), 1, "fp64")
    assert e.value.status == 5
    assert bool((v == 1).all())
    assert bool((u == 1).all())
    L.lmep_sync_status(H)
