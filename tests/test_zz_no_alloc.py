"""lmep_adjoint_step_noalloc: the allocation-free adjoint step agrees with lmep_adjoint_step.

Callers that cannot allocate device memory (their host application's
allocator owns the device, or their loop must not enter the driver's
allocator) use the entry point whose scratch is a static array inside the
library.  Two calls in a row -- the second reusing the static scratch the
first left behind -- must each match the allocating entry point (on the same
route: Pade derivatives) within the parity tolerance used by the other GPU
tests.  This file is collected last
and also runs alone in a fresh process.
"""
import numpy as np
import pytest

import workloads as wl

from lmep_testutil import grid_of, op_of, rel_linf, tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import paper_2603_15964_gb300 as L
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return L


def reference(L, h, p, u, lam_next, precision):
    """The allocating entry point on the route the allocation-free one takes: without a handle
    there is no exp(E) table, so both take the Pade derivatives of every point."""
    L.lmep_set_expm_method(h, "pade")
    dt_ = L.state_dtype(precision)
    g = grid_of(p)
    scratch = torch.empty(L.lmep_adjoint_scratch_bytes(g, precision), dtype=torch.uint8, device="cuda")
    lam = torch.empty(p.N, dtype=dt_, device="cuda")
    dnu = torch.zeros(1, dtype=torch.float64, device="cuda")
    L.lmep_adjoint_step(h, g, op_of(p), p.dt, u, lam_next, lam, dnu, scratch, precision)
    L.lmep_sync_status(h)
    return lam.cpu().numpy(), dnu.item()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_allocating_entry_point_twice(L, precision):
    h = L.Handle()
    dt_ = L.state_dtype(precision)
    cases = [wl.burgers(N=4099, n=9, cfl=2.0, nu=1e-6, seed=3),      # first call
             wl.burgers(N=257, n=13, cfl=4.0, nu=1e-5, seed=5)]      # second call, smaller grid
    for k, p in enumerate(cases):
        u = torch.tensor(wl.burgers_ic(p.N, 10 + k), dtype=dt_, device="cuda")
        lam_next = torch.tensor(np.random.default_rng(k).standard_normal(p.N), dtype=dt_, device="cuda")
        want_lam, want_dnu = reference(L, h, p, u, lam_next, precision)
        lam = torch.full((p.N,), float("nan"), dtype=dt_, device="cuda")
        dnu = torch.zeros(1, dtype=torch.float64, device="cuda")
        L.lmep_adjoint_step_noalloc(grid_of(p), op_of(p), p.dt, u, lam_next, lam, dnu, precision)
        torch.cuda.synchronize()
        assert rel_linf(lam.cpu().numpy(), want_lam) <= tol(precision)
        assert abs(dnu.item() - want_dnu) <= tol(precision) * max(abs(want_dnu), 1e-300)
    h.close()


def test_noalloc_rejects_grids_beyond_the_static_scratch(L):
    p = wl.burgers(N=1 << 20, n=15, cfl=1.0, nu=1e-6)
    u = torch.zeros(p.N, dtype=torch.float64, device="cuda")
    lam = torch.zeros_like(u)
    dnu = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LmepError) as e:
        L.lmep_adjoint_step_noalloc(grid_of(p), op_of(p), p.dt, u, u.clone(), lam, dnu, "fp64")
    assert e.value.status == 1 and "static scratch" in str(e.value)
