"""ETDRK4 (Sec. 3) and the Burgers term N(u) = -u u_x (Sec. 4.3.1) on the GPU, through the C ABI.

* lmep_harvest_scheme_weights: the six rows per row class (exp(dt L), dt alpha, dt beta, dt gamma,
  exp(dt L / 2), (dt/2) phi_1(dt L / 2)) against the oracle's rows (augmented local matrices with
  p = 3 at dt and p = 1 at dt/2, alpha/beta/gamma combined as in the paper), every row class;
  lmep_harvest_weights with n_phi = 3 against the raw rows of dt^k phi_k.
* lmep_step with LMEP_SCHEME_ETDRK4: one step and K-step trajectories against the oracle's ETDRK4
  (Allen-Cahn periodic / Neumann / Dirichlet with walls at -1 and 1, KdV, the paper's viscous Burgers
  benchmark and a Dirichlet Burgers case), at 1e-12 K (FP64) / 1e-5 K (FP32 form), ragged sizes.
* ETD1 and ETDRK2 with the Burgers term on periodic grids.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import lmep as olmep

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


def cases():
    return {
        "ac_periodic_n9": (wl.allen_cahn(3001, n=9, scheme="etdrk4", steps=5, mu=0.6), 1),
        "ac_neumann_n7": (wl.allen_cahn(1531, bc=wl.NEUMANN, n=7, scheme="etdrk4", steps=5, mu=0.8), 2),
        "ac_dirichlet_n9": (wl.allen_cahn(2049, bc=wl.DIRICHLET, n=9, scheme="etdrk4", steps=5, mu=0.5)
                            .with_(bc_lo=-1.0, bc_hi=1.0), 3),
        "kdv_n11": (wl.kdv(N=3000, n=11, L=30.0, scheme="etdrk4", steps=4), None),
        "burgers_paper_n13": (wl.burgers_etd(N=256, n=13, nu=0.03, dt=0.01, steps=6), None),
        "burgers_dirichlet_n9": (wl.burgers_etd(N=1201, n=9, nu=1e-3, dt=2e-3, steps=4)
                                 .with_(bc=wl.DIRICHLET, a=-1.0, b=1.0), None),
        "ac_reaction_c0_n5": (wl.Problem("r", 777, 0.0, 1.0, wl.PERIODIC, 5, 0.02, c0=-1.5, c2=2e-6,
                                         scheme="etdrk4", nonlin="allen_cahn", steps=5), 4),
    }


def ic_of(name, p, seed):
    if p.nonlin == "allen_cahn":
        u = wl.allen_cahn_ic(p.N, seed)
        if p.bc == wl.DIRICHLET:
            u = 0.53 * p.nodes() + 0.47 * np.sin(-1.5 * np.pi * p.nodes())    # Sec. 4.3.3's profile
        return u
    if p.nonlin == "kdv":
        return wl.kdv_ic(p, 0)
    if p.bc == wl.DIRICHLET:
        x = p.nodes()
        return np.sin(np.pi * x) * np.exp(-x * x)
    return wl.burgers_etd_ic(p)


def oracle_rows(p):
    W = olmep.constant_weights(p)
    al, be, ga = olmep.etdrk4_coefficient_rows(p, W)
    Wh = olmep.half_step_weights(p)
    return np.stack([W[:, 0], al, be, ga, Wh[:, 0], Wh[:, 1]], axis=1)          # [n][6][n]


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("name", list(cases()))
def test_harvest_scheme_weights_etdrk4(L, H, precision, name):
    p, _ = cases()[name]
    W = torch.empty(p.n, 6, p.n, dtype=L.state_dtype(precision), device="cuda")
    L.lmep_harvest_scheme_weights(H, grid_of(p), op_of(p), p.dt, "etdrk4", W, precision)
    got = W.cpu().numpy()
    want = oracle_rows(p)
    for k in range(6):
        assert weight_err(got[:, k], want[:, k]) <= tol(precision), k
    raw = torch.empty(p.n, 4, p.n, dtype=L.state_dtype(precision), device="cuda")
    L.lmep_harvest_weights(H, grid_of(p), op_of(p), p.dt, 3, None, raw, precision)
    wraw = olmep.constant_weights(p)
    for k in range(4):
        assert weight_err(raw.cpu().numpy()[:, k], wraw[:, k]) <= tol(precision), k


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("name", list(cases()))
def test_etdrk4_step_and_trajectory(L, H, precision, name):
    p, seed = cases()[name]
    u0 = ic_of(name, p, seed)
    if p.bc == wl.DIRICHLET:
        u0[0], u0[-1] = p.bc_lo, p.bc_hi
    if precision == "mixed":
        u0 = u0.astype(np.float32).astype(np.float64)
    dt_ = L.state_dtype(precision)
    W = torch.empty(p.n, 6, p.n, dtype=dt_, device="cuda")
    L.lmep_harvest_scheme_weights(H, grid_of(p), op_of(p), p.dt, "etdrk4", W, precision)
    u = torch.tensor(u0, dtype=dt_, device="cuda")
    work = torch.empty_like(u)
    u1 = u.clone()
    L.lmep_step(H, grid_of(p), op_of(p), "etdrk4", p.nonlin, p.dt, W, u1, work, 1, precision)
    L.lmep_sync_status(H)
    assert rel_linf(u1.cpu().numpy(), olmep.run(p, u0, 1)) <= tol(precision)
    L.lmep_step(H, grid_of(p), op_of(p), "etdrk4", p.nonlin, p.dt, W, u, work, p.steps, precision)
    L.lmep_sync_status(H)
    # K-step bound: K x the one-step tolerance, times (FP32 form) the largest l1 norm kappa of an updated
    # row of exp(dt L): next to a Dirichlet wall the one-sided rows (kappa = 48 at n = 9, mu = 0.5)
    # multiply the FP32 rounding of the state at every step; kappa = 1 on periodic and Neumann grids
    kappa = 1.0
    if precision == "mixed" and p.bc == wl.DIRICHLET:
        W0 = olmep.constant_weights(p)[:, 0]
        kappa = max(float(np.sum(np.abs(W0[r]))) for r in range(1, p.n - 1))
    assert rel_linf(u.cpu().numpy(), olmep.run(p, u0)) <= tol(precision) * p.steps * kappa


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("scheme", ["etd1", "etdrk2"])
def test_burgers_term_with_etd1_and_etdrk2(L, H, precision, scheme):
    # CFL 0.16 for the explicit N(u): ETD1 treats the advection like forward Euler, stable only briefly
    p = wl.burgers_etd(N=256, n=11, nu=0.03, dt=0.004, scheme=scheme, steps=5)
    u0 = wl.burgers_etd_ic(p)
    if precision == "mixed":
        u0 = u0.astype(np.float32).astype(np.float64)
    dt_ = L.state_dtype(precision)
    W = torch.empty(p.n, 1 + p.n_phi, p.n, dtype=dt_, device="cuda")
    L.lmep_harvest_scheme_weights(H, grid_of(p), op_of(p), p.dt, scheme, W, precision)
    u = torch.tensor(u0, dtype=dt_, device="cuda")
    L.lmep_step(H, grid_of(p), op_of(p), scheme, "burgers", p.dt, W, u, torch.empty_like(u), p.steps, precision)
    L.lmep_sync_status(H)
    assert rel_linf(u.cpu().numpy(), olmep.run(p, u0)) <= tol(precision) * p.steps


def test_etdrk4_rejections(L, H):
    p = wl.allen_cahn(512, n=15, scheme="etdrk4")
    W = torch.empty(15, 6, 15, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LmepError) as e:                       # n + 3 > 16
        L.lmep_harvest_scheme_weights(H, grid_of(p), op_of(p), p.dt, "etdrk4", W, "fp64")
    assert e.value.status == 5
    q = wl.allen_cahn(64, n=13, scheme="etd1").with_(nonlin="burgers")
    u = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LmepError):                            # ETD1 with N(u) = -u u_x on Neumann
        L.lmep_step(H, grid_of(q.with_(bc=wl.NEUMANN)), op_of(q), "etd1", "burgers", q.dt,
                    torch.zeros(13, 2, 13, dtype=torch.float64, device="cuda"), u, torch.empty_like(u), 1, "fp64")
