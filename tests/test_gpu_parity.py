"""GPU parity of every hot-path step against the FP64 oracle, through the C ABI.

Tolerances (FP64 path / FP32 form): weights ||dw||_inf / ||w||_1 <= 1e-12 / 1e-5;
one step from an identical state: rel l_inf <= 1e-12 / 1e-5; trajectories of
K steps: rel l_inf <= 1e-12 * K / 1e-5 * K (rounding grows at most linearly for
these contractive or norm-preserving updates).  Integer outputs (windows, rows,
Pade degree, squarings) are bit-exact.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import adjoint as oadj, expm as oexpm, grid as ogrid, lmep as olmep, operator as oop

from lmep_testutil import grid_of, op_of, rel_linf, tol, weight_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = ["fp64", "mixed"]


@pytest.fixture(scope="module")
def L():
    import paper_2603_15964_gb300 as L
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return L


@pytest.fixture(scope="module")
def H(L):
    return L.Handle()


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


# ------------------------------------------------------------------ (a1)-(a3)
@pytest.mark.parametrize("case", ["burgers", "burgers_plain", "kdv_aug", "ac_neumann_aug", "dirichlet_adv"])
def test_build_operator(L, H, case):
    if case.startswith("burgers"):
        p = wl.burgers(N=301, n=9, cfl=2.6, nu=1e-4, departure_centring=case == "burgers")
        u = wl.burgers_ic(p.N, 4)
        n_phi = 0
    elif case == "kdv_aug":
        p = wl.kdv(N=200, n=11, L=25.0)
        u, n_phi = None, 2
    elif case == "ac_neumann_aug":
        p = wl.allen_cahn(97, bc=wl.NEUMANN, n=9, scheme="etd1")
        u, n_phi = None, 1
    else:
        p = wl.Problem("adv", 40, 0.0, 1.0, wl.DIRICHLET, 7, 0.0, c1=-1.0, c2=0.003).with_(dt=2.5 / 39)
        u, n_phi = None, 0
    d = p.n + n_phi
    M = torch.empty(p.N, d, d, dtype=torch.float64, device="cuda")
    st = torch.empty(p.N, dtype=torch.int32, device="cuda")
    rw = torch.empty(p.N, dtype=torch.int32, device="cuda")
    L.lmep_build_operator(H, grid_of(p), op_of(p), p.dt, n_phi, None if u is None else dev(u), 0, p.N, M, st, rw)
    M, st, rw = M.cpu().numpy(), st.cpu().numpy(), rw.cpu().numpy()
    D = oop.unit_D(p.n)
    for i in range(p.N):
        k = ogrid.departure_shift(u[i], p.dt, p.h, p.n) if (u is not None and p.departure_centring) else 0
        idx, r = ogrid.stencil(p, i, k)
        assert rw[i] == r
        X = oop.local_matrix(p, 0.0 if u is None else u[i], D)
        want = oop.augmented_row(X, p.dt, r, n_phi) if n_phi else X
        assert np.max(np.abs(M[i] - want)) <= 1e-14 * max(1.0, np.max(np.abs(want))), i
        if p.bc == wl.DIRICHLET:
            assert st[i] == idx[0]
        elif p.bc == wl.PERIODIC:
            assert st[i] % p.N == idx[0]


# ------------------------------------------------------------------ (a4)
@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("d", [3, 5, 7, 9, 11, 13, 15, 16])
def test_expm_batched(L, H, precision, d):
    rng = np.random.default_rng(d)
    scales = [1e-3, 0.02, 0.2, 0.8, 1.8, 4.0, 30.0, 400.0]
    A = []
    for s in scales:
        for _ in range(5):
            a = rng.standard_normal((d, d))
            A.append(a * s / oexpm.norm1(a))
    A = np.array(A)
    E = torch.empty(A.shape, dtype=torch.float64, device="cuda")
    ms = torch.empty(len(A), 2, dtype=torch.int32, device="cuda")
    L.lmep_expm(H, dev(A), d, E, precision, ms)
    E, ms = E.cpu().numpy(), ms.cpu().numpy()
    for q in range(len(A)):
        want, m, s = oexpm.expm(A[q], return_ms=True)
        # same degree rule; the GPU scales m = 13 by Al-Mohy & Higham (2009), the
        # oracle by Higham (2005), so only the degree is compared exactly
        assert ms[q, 0] == m
        err = np.max(np.abs(E[q] - want)) / np.max(np.abs(want))
        # conditioning of exp grows with the norm: allow the FP64 oracle's own growth
        assert err <= tol(precision) * max(1.0, oexpm.norm1(A[q]) / 5.0), (q, m, s, err)


# ------------------------------------------------------------------ (a1)-(a5) constant coefficients
def const_cases():
    return {
        "advdiff_n5": wl.advection_diffusion(N=256, n=5),
        "dirichlet_adv_n7": wl.Problem("adv", 64, 0.0, 1.0, wl.DIRICHLET, 7, 0.0, c1=-1.0, c2=0.002)
                             .with_(dt=2.5 / 63),
        "ac_etdrk2_n9": wl.allen_cahn(1024, n=9, scheme="etdrk2", mu=0.5),
        "ac_etd1_n13": wl.allen_cahn(500, bc=wl.NEUMANN, n=13, scheme="etd1", mu=0.9),
        "kdv_etdrk2_n11": wl.kdv(N=4096, n=11, L=50.0),
        "reaction_n9": wl.Problem("r", 64, 0.0, 1.0, wl.PERIODIC, 9, 0.05, c0=1.0, c2=0.001, scheme="etdrk2",
                                  nonlin="allen_cahn"),
    }


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("name", list(const_cases()))
def test_harvest_constant(L, H, precision, name):
    p = const_cases()[name]
    W = torch.empty(p.n, 1 + p.n_phi, p.n, dtype=L.state_dtype(precision), device="cuda")
    L.lmep_harvest_weights(H, grid_of(p), op_of(p), p.dt, p.n_phi, None, W, precision)
    want = olmep.constant_weights(p)
    got = W.cpu().numpy()
    for k in range(1 + p.n_phi):
        assert weight_err(got[:, k], want[:, k]) <= tol(precision), k


# ------------------------------------------------------------------ (a1)-(a5) frozen velocity
@pytest.mark.parametrize("method", ["auto", "series", "pade"])
@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("n,cfl", [(7, 1.0), (9, 2.0), (13, 4.0), (13, 1.0), (5, 3.0)])
@pytest.mark.parametrize("nu", [1e-6, 4e-4, 1e-3])
def test_harvest_frozen(L, H, precision, n, cfl, nu, method):
    """Every evaluation of the exponential row ("series": finite series of the nilpotent local
    matrix where its error bound is small, Pade elsewhere; "auto": in the FP32 form the factorised
    row l(r + a)^T exp(E) first, then as "series"; "pade": Pade only).  At N = 513 the viscosities
    4e-4 and 1e-3 give launches where several routes run side by side."""
    N = 513
    p = wl.burgers(N=N, n=n, cfl=cfl, nu=nu)
    u = wl.burgers_ic(N, 0)
    if precision == "mixed":
        u = u.astype(np.float32).astype(np.float64)     # both sides see the same FP32 state
    W = torch.empty(N, n, dtype=L.state_dtype(precision), device="cuda")
    L.lmep_set_expm_method(H, method)
    try:
        L.lmep_harvest_weights(H, grid_of(p), op_of(p), p.dt, 0, dev(u, L.state_dtype(precision)), W, precision)
    finally:
        L.lmep_set_expm_method(H, "auto")
    got = W.cpu().numpy()
    D = oop.unit_D(n)
    want = np.zeros((N, n))
    for i in range(1, N - 1):
        want[i] = olmep.point_weights(p, u, i, D)[2][0]
    assert np.all(got[0] == 0) and np.all(got[-1] == 0)
    if precision == "mixed":
        assert weight_err(got[1:-1], want[1:-1]) <= tol(precision)
        return
    # FP64: the exponential of the rounded local matrix -- the oracle's -- can be off by ~1e-12
    # (and by ~1e-11 at the as-written viscosity, where ||X||_1 reaches ~470 and s = 7), while
    # the factorised rows avoid that rounding.  Where the two differ by more than 1e-12 the exact
    # rows decide: the GPU must be at least as accurate as the oracle (within 2x).
    diff = np.max(np.abs(got - want), axis=1) / np.maximum(np.sum(np.abs(want), axis=1), 1e-300)
    diff[0] = diff[-1] = 0.0
    worst = [int(i) for i in np.argsort(-diff)[:12] if diff[i] > 1e-12]
    e_gpu, e_orc = [], []
    for i in worst:
        idx, r = ogrid.stencil(p, i, ogrid.departure_shift(u[i], p.dt, p.h, n))
        ex = exact_row(n, -p.dt * u[i] / p.h, p.dt * p.c2 / p.h ** 2, r)
        den = np.sum(np.abs(ex))
        e_gpu.append(np.max(np.abs(got[i] - ex)) / den)
        e_orc.append(np.max(np.abs(want[i] - ex)) / den)
    if worst:
        assert max(e_gpu) <= max(2 * max(e_orc), 1e-12), (worst, e_gpu, e_orc)


def exact_row(n, a_hat, mu_hat, r):
    """Row r of exp(a_hat D-hat1 + mu_hat D-hat2) in exact rational arithmetic: the local matrix
    is nilpotent, so the Taylor series ends after n terms (a double is a rational number)."""
    from fractions import Fraction
    from oracle import exact
    D1 = exact.lagrange_D(range(n), 1)
    D2 = exact.lagrange_D(range(n), 2)
    a, mu = Fraction(a_hat), Fraction(mu_hat)
    X = [[a * D1[i][j] + mu * D2[i][j] for j in range(n)] for i in range(n)]
    v = [Fraction(int(j == r)) for j in range(n)]
    acc = v[:]
    for k in range(1, n + 1):
        v = [sum(v[i] * X[i][j] for i in range(n)) / k for j in range(n)]
        acc = [acc[j] + v[j] for j in range(n)]
    assert all(x == 0 for x in v)            # X^n = 0 exactly
    return np.array([float(x) for x in acc])


# ------------------------------------------------------------------ (a6) stored weights
def step_cases():
    return {
        "cfg1_advdiff": (wl.advection_diffusion(N=256, n=5, steps=100), None),
        "dirichlet_advdiff_tiles": (wl.Problem("adv", 3001, 0.0, 1.0, wl.DIRICHLET, 7, 0.0, c1=-1.0, c2=1e-5,
                                               bc_lo=0.0, bc_hi=0.0, steps=12).with_(dt=2.2 / 3000), None),
        "ac_etdrk2_periodic_ragged": (wl.allen_cahn(5000, n=9, scheme="etdrk2", steps=15), 3),
        "ac_etdrk2_neumann": (wl.allen_cahn(1531, bc=wl.NEUMANN, n=9, scheme="etdrk2", steps=15), 4),
        "ac_etd1_periodic": (wl.allen_cahn(2049, n=7, scheme="etd1", steps=15), 5),
        "kdv_etdrk2": (wl.kdv(N=3000, n=11, L=30.0, steps=10), None),
        # widths of the stand-alone apply sweep: n = 5 and 13 for ETDRK2, 15 for the linear apply
        "ac_etdrk2_n5_periodic": (wl.allen_cahn(3001, n=5, scheme="etdrk2", steps=12), 6),
        "ac_etdrk2_n13_neumann": (wl.allen_cahn(2500, bc=wl.NEUMANN, n=13, scheme="etdrk2", steps=12), 7),
        "advdiff_n15_periodic": (wl.Problem("adv", 4099, -1.0, 1.0, wl.PERIODIC, 15, 0.0, c1=-1.0, c2=1e-4,
                                            steps=12).with_(dt=0.7 * 2.0 / 4099), None),
        # walled grids of several tiles (2048 points in FP32, 1024 in FP64): the tiles whose halo stays clear
        # of the walls take the interior path of the tiled kernel, the two next to the walls the per-point one
        "dirichlet_advdiff_many_tiles": (wl.Problem("adv", 9001, 0.0, 1.0, wl.DIRICHLET, 7, 0.0, c1=-1.0, c2=1e-5,
                                                    bc_lo=0.0, bc_hi=0.0, steps=12).with_(dt=2.2 / 9000), None),
        "ac_etdrk2_dirichlet_tiles": (wl.allen_cahn(7001, bc=wl.DIRICHLET, n=9, scheme="etdrk2", steps=8, mu=0.1), 8),
    }


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("name", list(step_cases()))
def test_step_stored_weights(L, H, precision, name):
    p, seed = step_cases()[name]
    if p.nonlin == "allen_cahn":
        u0 = wl.allen_cahn_ic(p.N, seed)
    elif p.nonlin == "kdv":
        u0 = wl.kdv_ic(p, 0)
    elif name == "cfg1_advdiff":
        u0 = wl.advection_diffusion_ic(p)
    else:
        u0 = np.sin(3 * np.pi * p.nodes()) * np.exp(-p.nodes())
        u0[0] = u0[-1] = 0.0
    dt_ = L.state_dtype(precision)
    if precision == "mixed":
        u0 = u0.astype(np.float32).astype(np.float64)
    W = torch.empty(p.n, 1 + p.n_phi, p.n, dtype=dt_, device="cuda")
    L.lmep_harvest_weights(H, grid_of(p), op_of(p), p.dt, p.n_phi, None, W, precision)
    u = dev(u0, dt_)
    work = torch.empty_like(u)
    # one step from an identical state
    u1 = u.clone()
    L.lmep_step(H, grid_of(p), op_of(p), p.scheme, p.nonlin, p.dt, W, u1, work, 1, precision)
    L.lmep_sync_status(H)
    want1 = olmep.step(p, olmep.constant_weights(p), u0)
    assert rel_linf(u1.cpu().numpy(), want1) <= tol(precision)
    # trajectory
    L.lmep_step(H, grid_of(p), op_of(p), p.scheme, p.nonlin, p.dt, W, u, work, p.steps, precision)
    L.lmep_sync_status(H)
    want = olmep.run(p, u0)
    assert rel_linf(u.cpu().numpy(), want) <= tol(precision) * p.steps


# ------------------------------------------------------------------ (a1)-(a6) frozen velocity fused
@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("n,cfl", [(7, 1.0), (9, 2.0), (13, 4.0)])
def test_frozen_step_trajectory(L, H, precision, n, cfl):
    N, steps = 257, 8
    p = wl.burgers(N=N, n=n, cfl=cfl, nu=1e-6, steps=steps)
    u0 = wl.burgers_ic(N, 1)
    if precision == "mixed":
        u0 = u0.astype(np.float32).astype(np.float64)
    dt_ = L.state_dtype(precision)
    u = dev(u0, dt_)
    work = torch.empty_like(u)
    u1 = u.clone()
    L.lmep_step(H, grid_of(p), op_of(p), "linear", "none", p.dt, None, u1, work, 1, precision)
    L.lmep_sync_status(H)
    assert rel_linf(u1.cpu().numpy(), olmep.frozen_step(p, u0)) <= tol(precision)
    # the K-step trajectory, FP32 form included (its state is re-read in FP32 every step)
    L.lmep_step(H, grid_of(p), op_of(p), "linear", "none", p.dt, None, u, work, steps, precision)
    L.lmep_sync_status(H)
    assert rel_linf(u.cpu().numpy(), olmep.run(p, u0)) <= tol(precision) * steps


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("n,cfl", [(7, 1.0), (9, 2.0), (13, 4.0)])
def test_frozen_step_full_size_sampled(L, H, precision, n, cfl):
    """Burgers at N = 65536 (the benchmark launch): one step, oracle on sampled points."""
    N = 65536
    p = wl.burgers(N=N, n=n, cfl=cfl, nu=1e-6)
    u0 = wl.burgers_ic(N, 0)
    if precision == "mixed":
        u0 = u0.astype(np.float32).astype(np.float64)
    dt_ = L.state_dtype(precision)
    u = dev(u0, dt_)
    work = torch.empty_like(u)
    L.lmep_step(H, grid_of(p), op_of(p), "linear", "none", p.dt, None, u, work, 1, precision)
    L.lmep_sync_status(H)
    got = u.cpu().numpy()
    rng = np.random.default_rng(n)
    pts = sorted(set(rng.integers(1, N - 1, 300).tolist()) | {0, 1, 2, 3, 7, N - 8, N - 3, N - 2, N - 1})
    D = oop.unit_D(n)
    scale = np.max(np.abs(u0))
    for i in pts:
        if i in (0, N - 1):
            assert got[i] == 0.0
            continue
        idx, r, w = olmep.point_weights(p, u0, i, D)
        if abs(got[i] - w[0] @ u0[idx]) <= tol(precision) * scale:
            continue
        # FP64: the oracle's exponential of the rounded local matrix can be off by ~2e-12 at
        # n = 13, CFL 4; the exact rational row decides
        assert precision == "fp64", i
        ex = exact_row(n, -p.dt * u0[i] / p.h, p.dt * p.c2 / p.h ** 2, r)
        assert abs(got[i] - ex @ u0[idx]) <= tol(precision) * scale, i


# ------------------------------------------------------------------ batched persistent launch
@pytest.mark.parametrize("precision", PRECS)
def test_batched_allen_cahn(L, H, precision):
    B = 24
    batch = wl.allen_cahn_batch(B=B, Nmin=64, Nmax=3000, n=9, scheme="etdrk2", steps=6, seed=3)
    hs = [batch.problem(b).h for b in range(B)]
    dt_ = L.state_dtype(precision)
    u0s = [wl.allen_cahn_ic(int(batch.Ns[b]), b) for b in range(B)]
    if precision == "mixed":
        u0s = [x.astype(np.float32).astype(np.float64) for x in u0s]
    op = op_of(batch.problem(0))
    nbytes = L.lmep_batch_workspace_bytes(batch.Ns, hs, batch.bcs, 9, "etdrk2", "allen_cahn", batch.dt, op,
                                          precision, tile=512)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    L.lmep_batch_prepare(H, batch.Ns, hs, batch.bcs, 9, "etdrk2", "allen_cahn", batch.dt, op, ws, precision,
                         tile=512)
    from paper_2603_15964_gb300.batch import pack, unpack
    u = pack(u0s, dt_)
    work = torch.empty_like(u)
    L.lmep_step_batched(H, ws, u, work, batch.steps)
    L.lmep_sync_status(H)
    got = unpack(u, batch.Ns)
    for b in range(B):
        want = olmep.run(batch.problem(b), u0s[b], batch.steps)
        assert rel_linf(got[b], want) <= tol(precision) * batch.steps, b


# ------------------------------------------------------------------ (a7) adjoint
@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("centring", [False, True])
@pytest.mark.parametrize("method", ["auto", "pade"])
@pytest.mark.parametrize("nu", [2e-4, 1e-2])
def test_adjoint_step(L, H, precision, centring, nu, method):
    """One reverse step against the oracle.  "auto" takes the closed-form derivatives of the
    factorised rows, l'(z)^T exp(E) and l(z)^T Dh2 exp(E); at nu = 1e-2 the points next to the walls
    exceed the factorised bound and take the Pade derivatives in the same step (2 points with
    departure centring, 22 without); "pade" takes the Pade derivatives everywhere."""
    N = 96
    p = wl.burgers(N=N, n=7, cfl=1.6, nu=nu, departure_centring=centring)
    u = wl.burgers_ic(N, 3)
    lam_next = np.random.default_rng(1).standard_normal(N)
    if precision == "mixed":
        u = u.astype(np.float32).astype(np.float64)
        lam_next = lam_next.astype(np.float32).astype(np.float64)
    dt_ = L.state_dtype(precision)
    g = grid_of(p)
    scratch = torch.empty(L.lmep_adjoint_scratch_bytes(g, precision), dtype=torch.uint8, device="cuda")
    lam = torch.empty(N, dtype=dt_, device="cuda")
    dnu = torch.zeros(1, dtype=torch.float64, device="cuda")
    L.lmep_set_expm_method(H, method)
    try:
        L.lmep_adjoint_step(H, g, op_of(p), p.dt, dev(u, dt_), dev(lam_next, dt_), lam, dnu, scratch, precision)
        L.lmep_sync_status(H)
    finally:
        L.lmep_set_expm_method(H, "auto")
    want_lam, want_dnu = oadj.adjoint_step(p, u, lam_next)
    assert rel_linf(lam.cpu().numpy(), want_lam) <= 10 * tol(precision)
    # dJ/dnu is a sum with cancellation: bound its error by the sum of |terms|
    D = oop.unit_D(p.n)
    terms = []
    for i in ogrid.updated_points(p):
        idx, r, w, dwu, dwnu = oadj.point_derivatives(p, u, i, D)
        terms.append(lam_next[i] * (dwnu @ u[idx]))
    assert abs(dnu.item() - want_dnu) <= 10 * tol(precision) * np.sum(np.abs(terms))


# ------------------------------------------------------------------ status flags
def test_nonfinite_is_reported(L, H):
    """The as-written viscosity blows up; the overflow surfaces as LMEP_ERR_NONFINITE."""
    p = wl.burgers(N=65536, n=7, cfl=4.0, nu=1e-3)      # mu = nu dt / h^2 ~ 130
    u = dev(wl.burgers_ic(p.N, 0))
    work = torch.empty_like(u)
    with pytest.raises(L.LmepError) as e:
        L.lmep_step(H, grid_of(p), op_of(p), "linear", "none", p.dt, None, u, work, 300, "fp64")
        L.lmep_sync_status(H)
    assert e.value.status == 3
    L.lmep_sync_status(H)          # flags were cleared


def test_invalid_arguments_launch_nothing(L, H):
    p = wl.burgers(N=257, n=7, cfl=1.0)
    g = grid_of(p)
    u = dev(wl.burgers_ic(257, 0))
    with pytest.raises(L.LmepError) as e:
        L.lmep_step(H, g, op_of(p), "linear", "none", p.dt, None, u, u, 1, "fp64")
    assert e.value.status == 1
    bad = L.Grid(N=257, h=p.h, bc="dirichlet", n=8)
    with pytest.raises(L.LmepError):
        L.lmep_step(H, bad, op_of(p), "linear", "none", p.dt, None, u, torch.empty_like(u), 1, "fp64")


def test_fma_peaks_positive(L):
    f64 = L.lmep_fma_peak("fp64")
    f32 = L.lmep_fma_peak("mixed")
    assert f64 > 1e11 and f32 > 1e12
