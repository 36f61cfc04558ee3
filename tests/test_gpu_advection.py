"""High-CFL one-sided advection (Sec. 4.1) on the GPU, through the C ABI.

* Fully upwind windows (lmep_grid.window_shift = (n-1)/2) at the paper's Courant numbers
  nu = (n+1)/2 - sigma: 100 periods of u_t + u_x = 0 against the oracle (1e-12 K / 1e-5 K) and,
  for integer nu, against the exact solution: the row is a unit vector, an exact shift (Thm. 1).
* Shifted windows on Dirichlet and Neumann grids against the oracle over a few steps.
* lmep_amplification against the oracle's symbol G(theta) of the harvested row.
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


def run_gpu(L, H, p, u0, precision, steps):
    dt_ = L.state_dtype(precision)
    W = torch.empty(p.n, 1, p.n, dtype=dt_, device="cuda")
    L.lmep_harvest_weights(H, grid_of(p), op_of(p), p.dt, 0, None, W, precision)
    u = torch.tensor(u0, dtype=dt_, device="cuda")
    L.lmep_step(H, grid_of(p), op_of(p), "linear", "none", p.dt, W, u, torch.empty_like(u), steps, precision)
    L.lmep_sync_status(H)
    return u.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("n", [5, 9, 13, 15])
@pytest.mark.parametrize("sigma", [0.0, 0.5])
def test_one_sided_hundred_periods(L, H, precision, n, sigma):
    p = wl.advection(N=250, n=n, sigma=sigma, periods=100)
    u0 = wl.advection_ic(p)
    if precision == "mixed":
        u0 = u0.astype(np.float32).astype(np.float64)
    got = run_gpu(L, H, p, u0, precision, p.steps)
    if sigma == 0.0:
        # integer Courant number: every step shifts the profile by nu nodes exactly
        shift = int(round(p.meta["nu"])) * p.steps
        assert np.array_equal(got, np.roll(u0, shift))
        return
    want = olmep.run(p, u0)
    assert rel_linf(got, want) <= tol(precision) * p.steps, p.steps


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("bc,shift,cfl", [(wl.DIRICHLET, 3, 0.8), (wl.DIRICHLET, 1, 0.8), (wl.NEUMANN, 2, 2.4),
                                          (wl.PERIODIC, 2, 2.4), (wl.PERIODIC, 1, 1.4)])
def test_shifted_windows_other_boundaries(L, H, precision, bc, shift, cfl):
    """Upstream shifts (the speed is +0.7); next to a Dirichlet inflow wall a departure point beyond
    the wall would be an extrapolation, so the walled grids run below CFL 1."""
    p = wl.Problem("adv", 1001, -1.0, 1.0, bc, 7, 0.0, c1=-0.7, c2=1e-4, window_shift=shift, steps=6)
    p = p.with_(dt=cfl * p.h / 0.7)
    u0 = np.sin(np.pi * p.nodes()) * np.exp(-p.nodes() ** 2)
    if bc == wl.DIRICHLET:
        u0[0] = u0[-1] = 0.0
    if precision == "mixed":
        u0 = u0.astype(np.float32).astype(np.float64)
    got = run_gpu(L, H, p, u0, precision, p.steps)
    assert rel_linf(got, olmep.run(p, u0)) <= tol(precision) * p.steps


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("bc,shift,cfl", [(wl.DIRICHLET, 3, 0.8), (wl.PERIODIC, 2, 2.4)])
def test_shifted_windows_many_tiles(L, H, precision, bc, shift, cfl):
    """As above on 9001 points: several tiles of the tiled kernel, interior ones included.  The
    diffusion coefficient shrinks with h, so the local matrices (and the rows' l1 norms, which
    bound the rounding the rows pass on) are those of the 1001-point grid."""
    p = wl.Problem("adv", 9001, -1.0, 1.0, bc, 7, 0.0, c1=-0.7, c2=1e-4 / 9, window_shift=shift, steps=6)
    p = p.with_(dt=cfl * p.h / 0.7)
    u0 = np.sin(np.pi * p.nodes()) * np.exp(-p.nodes() ** 2)
    if bc == wl.DIRICHLET:
        u0[0] = u0[-1] = 0.0
    if precision == "mixed":
        u0 = u0.astype(np.float32).astype(np.float64)
    got = run_gpu(L, H, p, u0, precision, p.steps)
    assert rel_linf(got, olmep.run(p, u0)) <= tol(precision) * p.steps


@pytest.mark.parametrize("one_sided", [True, False])
def test_amplification_matches_oracle(L, H, one_sided):
    th = np.linspace(-np.pi, np.pi, 1001)
    for n in (5, 9, 15):
        p = wl.advection(N=128, n=n, sigma=0.5, one_sided=one_sided)
        W = torch.empty(p.n, 1, p.n, dtype=torch.float64, device="cuda")
        L.lmep_harvest_weights(H, grid_of(p), op_of(p), p.dt, 0, None, W, "fp64")
        r = (n - 1) // 2 + p.window_shift
        w = W[r, 0].contiguous()
        G = torch.empty(len(th), 2, dtype=torch.float64, device="cuda")
        L.lmep_amplification(w, r, torch.tensor(th, device="cuda"), G)
        got = G.cpu().numpy()
        want = olmep.amplification(w.cpu().numpy(), r, th)
        assert np.max(np.abs(got[:, 0] + 1j * got[:, 1] - want)) <= 1e-13 * np.sum(np.abs(w.cpu().numpy()))
        assert np.max(np.hypot(got[:, 0], got[:, 1])) <= 1.0 + 1e-12


def test_window_shift_rejections(L, H):
    p = wl.burgers(N=257, n=7, cfl=1.0).with_(window_shift=1)
    u = torch.tensor(wl.burgers_ic(257, 0), device="cuda")
    with pytest.raises(L.LmepError) as e:                                 # frozen velocity
        L.lmep_step(H, grid_of(p), op_of(p), "linear", "none", p.dt, None, u, torch.empty_like(u), 1, "fp64")
    assert e.value.status == 5
    q = wl.allen_cahn(256, n=9, scheme="etdrk2").with_(window_shift=2)
    W = torch.zeros(9, 3, 9, dtype=torch.float64, device="cuda")
    v = torch.zeros(256, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LmepError) as e:                                 # ETD schemes
        L.lmep_step(H, grid_of(q), op_of(q), "etdrk2", "allen_cahn", q.dt, W, v, torch.empty_like(v), 1, "fp64")
    assert e.value.status == 5
    with pytest.raises(L.LmepError) as e:                                 # |k| > (n-1)/2
        L.lmep_step(H, grid_of(q.with_(window_shift=5, scheme="linear", nonlin="none")), op_of(q), "linear", "none",
                    q.dt, W[:, :1].contiguous(), v, torch.empty_like(v), 1, "fp64")
    assert e.value.status == 1
