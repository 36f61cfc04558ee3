"""Edge and degenerate cases of the hot path on the GPU, through the C ABI, against the FP64 oracle.

* Zero steps leave the state untouched, bit for bit (stored weights and frozen velocity).
* Windows that span the whole grid (Dirichlet, N = n and N = n + 1): every point takes a one-sided
  row of the same local matrix (Sec. 2.1 step 1 at the walls).
* A last tile of one or two points (stored-weight steps on walled grids; tiles of 2048 points in
  the FP32 form, 1024 in FP64).
* Equilibria: the zero state of the frozen-velocity Burgers step and of Allen-Cahn stays exactly
  zero; constants are kept to rounding (the rows of exp(dt L) sum to one), and u = 1 is a fixed
  point of Allen-Cahn (N(1) = 0).
* Pure advection (c2 = 0): exp(E) = I, the row is the Lagrange interpolant at the departure point
  (Thm. 1), against the oracle's exponential of the local matrix.
* Grids too small for the tiled kernels' halo are refused before anything is launched.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import lmep as olmep

from lmep_testutil import grid_of, op_of, rel_linf, tol

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


def dev(a, dtype):
    return torch.tensor(np.asarray(a, dtype=np.float64), dtype=dtype, device="cuda")


def rounded(u0, precision):
    return u0.astype(np.float32).astype(np.float64) if precision == "mixed" else u0


def same_bits(a, b) -> bool:
    it = torch.int32 if a.dtype == torch.float32 else torch.int64
    return torch.equal(a.contiguous().view(it), b.contiguous().view(it))


def stored_step(L, H, p, u0, precision, steps):
    dt_ = L.state_dtype(precision)
    W = torch.empty(p.n, 1 + p.n_phi, p.n, dtype=dt_, device="cuda")
    L.lmep_harvest_weights(H, grid_of(p), op_of(p), p.dt, p.n_phi, None, W, precision)
    u = dev(u0, dt_)
    L.lmep_step(H, grid_of(p), op_of(p), p.scheme, p.nonlin, p.dt, W, u, torch.empty_like(u), steps, precision)
    L.lmep_sync_status(H)
    return u


def frozen_step(L, H, p, u0, precision, steps):
    u = dev(u0, L.state_dtype(precision))
    L.lmep_step(H, grid_of(p), op_of(p), "linear", "none", p.dt, None, u, torch.empty_like(u), steps, precision)
    L.lmep_sync_status(H)
    return u


def walled_advdiff(N, n=7, steps=5):
    """u_t = u_x + c2 u_xx on [0, 1] with zero walls at CFL 0.8; c2 = 0.06 h keeps the diffusion number
    (0.048) and so the local matrices, and the l1 norms of the one-sided rows, the same at every N."""
    h = 1.0 / (N - 1)
    p = wl.Problem("adv", N, 0.0, 1.0, wl.DIRICHLET, n, 0.0, c1=-1.0, c2=0.06 * h, bc_lo=0.0, bc_hi=0.0,
                   steps=steps)
    return p.with_(dt=0.8 * p.h)


def walled_ic(p):
    u = np.sin(3 * np.pi * p.nodes()) * np.exp(-p.nodes())
    u[0] = u[-1] = 0.0
    return u


# ------------------------------------------------------------------ zero steps
@pytest.mark.parametrize("precision", PRECS)
def test_zero_steps_leave_the_state(L, H, precision):
    dt_ = L.state_dtype(precision)
    p = walled_advdiff(3001)
    u0 = rounded(walled_ic(p), precision)
    W = torch.empty(p.n, 1, p.n, dtype=dt_, device="cuda")
    L.lmep_harvest_weights(H, grid_of(p), op_of(p), p.dt, 0, None, W, precision)
    u = dev(u0, dt_)
    ref = u.clone()
    L.lmep_step(H, grid_of(p), op_of(p), "linear", "none", p.dt, W, u, torch.empty_like(u), 0, precision)
    q = wl.burgers(N=2049, n=9, cfl=2.0, nu=1e-6)
    v = dev(rounded(wl.burgers_ic(q.N, 1), precision), dt_)
    vref = v.clone()
    L.lmep_step(H, grid_of(q), op_of(q), "linear", "none", q.dt, None, v, torch.empty_like(v), 0, precision)
    L.lmep_sync_status(H)
    assert same_bits(u, ref) and same_bits(v, vref)


# ------------------------------------------------------------------ windows spanning the grid
@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("n,extra", [(7, 0), (7, 1), (9, 0), (13, 1)])
def test_stored_step_window_spans_the_grid(L, H, precision, n, extra):
    p = walled_advdiff(n + extra, n=n, steps=4)
    u0 = rounded(walled_ic(p), precision)
    got = stored_step(L, H, p, u0, precision, p.steps).cpu().numpy()
    assert rel_linf(got, olmep.run(p, u0)) <= tol(precision) * p.steps


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("n,extra", [(5, 0), (7, 0), (9, 2)])
def test_frozen_step_window_spans_the_grid(L, H, precision, n, extra):
    # (at N = n = 13 the equispaced one-sided interpolants amplify the state a thousandfold in three
    # steps, a property of the method on so coarse a grid, so the widest case here is n = 9)
    p = wl.burgers(N=n + extra, n=n, cfl=1.0, nu=1e-6, steps=3)
    u0 = rounded(wl.burgers_ic(p.N, 2), precision)
    got = frozen_step(L, H, p, u0, precision, p.steps).cpu().numpy()
    assert rel_linf(got, olmep.run(p, u0)) <= tol(precision) * p.steps


# ------------------------------------------------------------------ ragged last tile
@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("N", [1025, 1026, 2049, 2050])
def test_last_tile_of_one_or_two_points(L, H, precision, N):
    p = walled_advdiff(N, steps=6)
    u0 = rounded(walled_ic(p), precision)
    got = stored_step(L, H, p, u0, precision, p.steps).cpu().numpy()
    assert rel_linf(got, olmep.run(p, u0)) <= tol(precision) * p.steps


# ------------------------------------------------------------------ equilibria
@pytest.mark.parametrize("precision", PRECS)
def test_zero_state_stays_zero(L, H, precision):
    p = wl.burgers(N=4099, n=13, cfl=4.0, nu=1e-6)
    got = frozen_step(L, H, p, np.zeros(p.N), precision, 5)
    assert bool((got == 0).all())
    q = wl.allen_cahn(3001, n=9, scheme="etdrk2")
    got = stored_step(L, H, q, np.zeros(q.N), precision, 5)
    assert bool((got == 0).all())


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("case", ["advdiff_periodic", "ac_neumann", "ac_periodic_etd1"])
def test_constants_are_kept(L, H, precision, case):
    # (the periodic linear case at the configuration-1 shape: diffusion number 0.33, so the rows' sums
    # are one to a few units of rounding)
    p = {"advdiff_periodic": wl.advection_diffusion(N=256, n=9, steps=10),
         "ac_neumann": wl.allen_cahn(2500, bc=wl.NEUMANN, n=9, scheme="etdrk2", steps=10),
         "ac_periodic_etd1": wl.allen_cahn(3001, n=7, scheme="etd1", steps=10)}[case]
    got = stored_step(L, H, p, np.ones(p.N), precision, p.steps).cpu().numpy()
    assert np.max(np.abs(got - 1.0)) <= tol(precision) * p.steps


# ------------------------------------------------------------------ pure advection
@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("n,cfl", [(7, 1.0), (9, 2.5), (13, 4.0)])
def test_pure_advection_is_the_lagrange_interpolant(L, H, precision, n, cfl):
    p = wl.burgers(N=3001, n=n, cfl=cfl, nu=0.0, steps=4)
    u0 = rounded(wl.burgers_ic(p.N, 3), precision)
    one = frozen_step(L, H, p, u0, precision, 1).cpu().numpy()
    assert rel_linf(one, olmep.frozen_step(p, u0)) <= tol(precision)
    got = frozen_step(L, H, p, u0, precision, p.steps).cpu().numpy()
    assert rel_linf(got, olmep.run(p, u0)) <= tol(precision) * p.steps


# ------------------------------------------------------------------ refused sizes
def test_grids_too_small_for_the_halo_are_refused(L, H):
    # n <= N (the harvest's own bound) but N below the halo of an ETDRK2 tile at n = 13
    for bc, N in ((wl.PERIODIC, 14), (wl.NEUMANN, 26)):
        p = wl.allen_cahn(N, bc=bc, n=13, scheme="etdrk2")
        W = torch.empty(p.n, 1 + p.n_phi, p.n, dtype=torch.float64, device="cuda")
        L.lmep_harvest_weights(H, grid_of(p), op_of(p), p.dt, p.n_phi, None, W, "fp64")
        u = dev(np.ones(p.N), torch.float64)
        with pytest.raises(L.LmepError) as e:
            L.lmep_step(H, grid_of(p), op_of(p), p.scheme, p.nonlin, p.dt, W, u, torch.empty_like(u), 1, "fp64")
        assert e.value.status == 5
        assert bool((u == 1).all())
    L.lmep_sync_status(H)
