"""The evaluations of a frozen-velocity exponential row (Sec. 2.1 step 4).

Without its identity term the local matrix X = a D1 + b D2 + c D3 of a window is a polynomial
without constant term in the differentiation matrix of the window's interpolating polynomial, so
X^n = 0 and a row of exp(X) is the finite Taylor sum of n terms ("series"): the library takes
that sum when its a-posteriori bound beta = sum_k ||e_r^T |X|^k||_1 / k! is small -- the FP32 form
sums in FP32 while beta <= 16 (statistics m = 0), else in FP64 while beta <= 2^20 (m = 1); the
FP64 path sums in FP64 while beta <= 64 (m = 0) -- and Pade scaling and squaring for the rest, or
for every point ("pade").  The parts a D1 and E = b D2 + c D3 of X commute, so row r of exp(X) is
also l(r + a)^T exp(E), l the Lagrange weights of the window (Thm. 1); the FP32 form takes that
factorised row first ("auto", m = 2) where sum_j |l_j| ||row j of exp(E)||_1 <= 16.

Checked here:
 * the route a point takes follows beta, computed on the CPU from the oracle's local matrix:
   series rows (statistics m = s = a = 0) where beta is well below the threshold, Pade rows
   where it is well above (near the threshold either; the kernel forms beta in FP32);
 * "pade" never reports a series row;
 * "auto" in the FP32 form takes the factorised row where its bound is well below 16 and
   matches the oracle; its rows match the exact rational rows;
 * a frozen operator with reaction (c0, which factors out as e^{dt c0}) and dispersion (c3) on a
   periodic grid, one fused step by either route, against the oracle (tolerances as in the
   parity tests: 1e-12 FP64, 1e-5 FP32 form, relative l_inf).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import grid as ogrid, lmep as olmep, operator as oop

from lmep_testutil import grid_of, op_of, rel_linf, tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TAU = {"fp64": 64.0, "mixed": 16.0, "mixed_f64": 2.0 ** 20}


@pytest.fixture(scope="module")
def L():
    import paper_2603_15964_gb300 as L
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return L


@pytest.fixture(scope="module")
def H(L):
    return L.Handle()


def beta_of(p, u, i, D):
    """The error bound of the finite series at point i, from the oracle's local matrix."""
    k = ogrid.departure_shift(u[i], p.dt, p.h, p.n) if p.departure_centring else 0
    idx, r = ogrid.stencil(p, i, k)
    X = oop.local_matrix(p, u[i], D) - p.dt * p.c0 * np.eye(p.n)
    kr = olmep.recentring_shift(p, u[i], r)
    A = np.abs(X + kr * D[1])
    w = np.zeros(p.n)
    w[r - kr] = 1.0
    beta = 1.0
    for j in range(1, p.n):
        w = w @ A / j
        beta += w.sum()
    return beta


def sl_bound_of(p, u, i, D):
    """The factorised form's bound sum_j |l_j(r + a)| ||row j of exp(E)||_1, on the CPU."""
    from scipy.linalg import expm
    k = ogrid.departure_shift(u[i], p.dt, p.h, p.n) if p.departure_centring else 0
    idx, r = ogrid.stencil(p, i, k)
    E = expm(p.dt * p.c2 / p.h ** 2 * D[2] + p.dt * p.c3 / p.h ** 3 * D[3])
    z = r + p.dt * (p.c1 - p.frozen_adv * u[i]) / p.h
    n = p.n
    lw = np.array([np.prod([(z - m) / (j - m) for m in range(n) if m != j]) for j in range(n)])
    return float(np.abs(lw) @ np.abs(E).sum(axis=1))


def stats_of(L, H, p, u, precision, method):
    st = torch.zeros(p.N, 3, dtype=torch.int32, device="cuda")
    L.lmep_set_expm_method(H, method)
    try:
        L.lmep_frozen_stats(H, grid_of(p), op_of(p), p.dt,
                            torch.tensor(u, dtype=L.state_dtype(precision), device="cuda"), st, precision)
        L.lmep_sync_status(H)
    finally:
        L.lmep_set_expm_method(H, "auto")
    return st.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nu,n,cfl", [(1e-6, 13, 4.0), (4e-4, 13, 4.0), (1e-3, 13, 1.0), (1e-3, 13, 4.0),
                                      (1e-3, 9, 2.0), (3e-3, 7, 1.0)])
def test_route_follows_error_bound(L, H, precision, nu, n, cfl):
    N = 513
    p = wl.burgers(N=N, n=n, cfl=cfl, nu=nu)
    u = wl.burgers_ic(N, 0)
    if precision == "mixed":
        u = u.astype(np.float32).astype(np.float64)
    D = oop.unit_D(n)
    beta = np.array([beta_of(p, u, i, D) for i in range(1, N - 1)])
    st = stats_of(L, H, p, u, precision, "series")[1:-1]
    assert np.all(st[:, 1:][st[:, 0] < 3] == 0)
    m = st[:, 0]
    t64 = TAU["fp64"]
    if precision == "mixed":
        t32, t64 = TAU["mixed"], TAU["mixed_f64"]
        assert np.all(m[beta < 0.5 * t32] == 0), np.flatnonzero((m != 0) & (beta < 0.5 * t32))
        mid = (beta > 2 * t32) & (beta < 0.5 * t64)
        assert np.all(m[mid] == 1), np.flatnonzero((m != 1) & mid)
    else:
        assert np.all(m[beta < 0.5 * t64] == 0), np.flatnonzero((m != 0) & (beta < 0.5 * t64))
        assert not np.any(m == 1)
    assert np.all(m[beta > 2 * t64] >= 3), np.flatnonzero((m < 3) & (beta > 2 * t64))
    pade = stats_of(L, H, p, u, precision, "pade")[1:-1]
    assert np.all(pade[:, 0] >= 3)


def test_all_routes_in_one_launch(L, H):
    """The cases above that mix the routes do mix them, so that launches in which the routes run
    side by side are tested: FP32 and FP64 series, and FP64 series and Pade, in FP32-form
    launches; series and Pade in an FP64 launch."""
    for precision, (nu, n, cfl), want in (("mixed", (1e-3, 13, 1.0), {"f32", "f64"}),
                                          ("mixed", (1e-3, 13, 4.0), {"f64", "pade"}),
                                          ("fp64", (4e-4, 13, 4.0), {"f64", "pade"})):
        p = wl.burgers(N=513, n=n, cfl=cfl, nu=nu)
        u = wl.burgers_ic(513, 0)
        if precision == "mixed":
            u = u.astype(np.float32).astype(np.float64)
        m = stats_of(L, H, p, u, precision, "series")[1:-1, 0]
        name = {0: "f32" if precision == "mixed" else "f64", 1: "f64"}
        got = {name.get(int(v), "pade") for v in np.unique(m)}
        assert want <= got, (precision, nu, n, cfl, got)


def reaction_dispersion(n):
    N = 1021
    p = wl.Problem("frozen_rd", N, -1.0, 1.0, wl.PERIODIC, n, 0.0, c0=-0.7, c2=2e-5, c3=-1e-9,
                   frozen_adv=1.0, departure_centring=True)
    u0 = 0.8 * np.sin(np.pi * p.nodes()) + 0.3 * np.cos(3 * np.pi * p.nodes())
    return p.with_(dt=2.5 * p.h / np.max(np.abs(u0))), u0


@pytest.mark.parametrize("method", ["auto", "series", "pade"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [5, 9, 13])
def test_reaction_dispersion_periodic_step(L, H, precision, n, method):
    p, u0 = reaction_dispersion(n)
    if precision == "mixed":
        u0 = u0.astype(np.float32).astype(np.float64)
    dt_ = L.state_dtype(precision)
    u = torch.tensor(u0, dtype=dt_, device="cuda")
    work = torch.empty_like(u)
    L.lmep_set_expm_method(H, method)
    try:
        L.lmep_step(H, grid_of(p), op_of(p), "linear", "none", p.dt, None, u, work, 1, precision)
        L.lmep_sync_status(H)
    finally:
        L.lmep_set_expm_method(H, "auto")
    assert rel_linf(u.cpu().numpy(), olmep.frozen_step(p, u0)) <= tol(precision)
    if method != "pade":
        st = stats_of(L, H, p, u0, precision, method)
        want = 2 if method == "auto" else 0
        assert np.mean(st[:, 0] == want) > 0.9       # this operator takes the cheap route


def test_invalid_method_is_rejected(L, H):
    from paper_2603_15964_gb300 import _lib
    with pytest.raises(_lib.LmepError):
        _lib.call("lmep_set_expm_method", H.ptr, 7)
    with pytest.raises(KeyError):
        L.lmep_set_expm_method(H, "taylor")


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_matches_eager_steps(L, precision, fused):
    """FrozenSet: K steps replayed from captured CUDA graphs equal K eager steps bit for bit (three
    instances of different n and dt, one with Pade rows), as one launch per step (fused) and as one
    library call per instance."""
    from paper_2603_15964_gb300.frozen import FrozenInstance, FrozenSet
    probs = [wl.burgers(N=4099, n=7, cfl=2.0, nu=1e-6), wl.burgers(N=2048, n=13, cfl=4.0, nu=4e-4),
             wl.burgers(N=3001, n=9, cfl=1.0, nu=1e-6)]
    insts = [FrozenInstance(grid_of(p), op_of(p), p.dt) for p in probs]
    u0 = [wl.burgers_ic(p.N, s) for s, p in enumerate(probs)]
    K = 5
    eager = FrozenSet(insts, precision=precision, fused=fused)
    eager.load(u0)
    eager.step(K)
    graph = FrozenSet(insts, precision=precision, fused=fused)
    graph.load(u0)
    graph.capture()               # eager warm-up: two steps (fused, one per direction) or one
    graph.replay(K - (2 if fused else 1))
    torch.cuda.synchronize()
    for a, b in zip(eager.states, graph.states):
        assert torch.equal(a, b)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nu,n,cfl,N", [(1e-6, 13, 4.0, 513), (1e-6, 7, 1.0, 513), (4e-4, 13, 4.0, 513),
                                        (1e-3, 13, 1.0, 513), (1e-3, 9, 2.0, 513), (3e-3, 7, 1.0, 513),
                                        (1e-6, 13, 4.0, 65536)])
def test_factorised_rows(L, H, precision, nu, n, cfl, N):
    """"auto": the factorised route is taken where its bound is well below 16 and not where it is
    well above; its rows match the exact rational rows (<= 2e-6 FP32 form, <= 1e-14 FP64) and the
    oracle (FP32 form: within its tolerance; FP64: within 1e-12 except where the oracle's
    exponential of the rounded local matrix is itself off, ~2e-12 at N = 65536, n = 13, CFL 4 --
    there the exact row decides)."""
    from test_gpu_parity import exact_row
    from lmep_testutil import weight_err
    p = wl.burgers(N=N, n=n, cfl=cfl, nu=nu)
    u = wl.burgers_ic(N, 0)
    if precision == "mixed":
        u = u.astype(np.float32).astype(np.float64)
    D = oop.unit_D(n)
    rng = np.random.default_rng(7)
    pts = np.arange(1, N - 1) if N <= 1024 else np.unique(np.concatenate(
        [rng.integers(1, N - 1, 400), [1, 2, 3, N - 4, N - 3, N - 2]]))
    bound = np.array([sl_bound_of(p, u, int(i), D) for i in pts])
    m = stats_of(L, H, p, u, precision, "auto")[pts, 0]
    assert np.all(m[bound < 8.0] == 2), pts[(m != 2) & (bound < 8.0)]
    assert not np.any(m[bound > 32.0] == 2), pts[(m == 2) & (bound > 32.0)]
    dt_ = L.state_dtype(precision)
    W = torch.empty(N, n, dtype=dt_, device="cuda")
    L.lmep_set_expm_method(H, "auto")
    L.lmep_harvest_weights(H, grid_of(p), op_of(p), p.dt, 0, torch.tensor(u, dtype=dt_, device="cuda"), W,
                           precision)
    got = W.cpu().numpy().astype(np.float64)[pts]
    want = np.array([olmep.point_weights(p, u, int(i), D)[2][0] for i in pts])
    diff = np.max(np.abs(got - want), axis=1) / np.sum(np.abs(want), axis=1)
    if precision == "mixed":
        assert weight_err(got, want) <= tol("mixed")
    sl = np.flatnonzero(m == 2)
    check = set(sl[:: max(1, len(sl) // 6)][:6].tolist())
    if precision == "fp64":
        check |= set(np.flatnonzero(diff > tol("fp64")).tolist())
    for q in sorted(check):
        i = int(pts[q])
        idx, r = ogrid.stencil(p, i, ogrid.departure_shift(u[i], p.dt, p.h, n))
        ex = exact_row(n, -p.dt * u[i] / p.h, p.dt * p.c2 / p.h ** 2, r)
        e_gpu = np.max(np.abs(got[q] - ex)) / np.sum(np.abs(ex))
        if m[q] == 2:
            assert e_gpu <= (2e-6 if precision == "mixed" else 1e-14), (i, e_gpu)
        else:
            assert e_gpu <= max(2 * np.max(np.abs(want[q] - ex)) / np.sum(np.abs(ex)), tol(precision)), i
