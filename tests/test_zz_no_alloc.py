"""lmep_adjoint_step_noalloc: the allocation-free adjoint step.

Some callers cannot allocate device memory: a plug-in whose host application's allocator owns the
device, or a loop that must never enter the driver's allocator.  They call the entry point whose
scratch is a static array inside the library.  Checked here:

* calls in a row -- a larger grid after a smaller one, then the same grid with other data, so that
  anything read from an earlier call's scratch would show -- each equal to the allocating entry
  point on the same route (the Pade Frechet derivatives: without a handle there is no exp(E)
  table), lam bit for bit (the same kernels run on the same layout), dJ/dnu within the rounding of
  its order-dependent atomic sum;
* one call against the FP64 oracle's adjoint step (10x the parity tolerance, as the other adjoint
  tests);
* the first call of a fresh process, before any handle exists;
* the size limit: N = 63548 at n = 15 in FP64 fits the 8 MiB scratch, N = 63549 is rejected.

This file is collected last, so a run that stops at its first failure has run every other test.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads as wl
from oracle import adjoint as oadj, grid as ogrid, operator as oop

from lmep_testutil import grid_of, op_of, rel_linf, tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    import paper_2603_15964_gb300 as L
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return L


def reference(L, h, p, u, lam_next, precision):
    """The allocating entry point on the route the allocation-free one takes."""
    L.lmep_set_expm_method(h, "pade")
    dt_ = L.state_dtype(precision)
    g = grid_of(p)
    scratch = torch.empty(L.lmep_adjoint_scratch_bytes(g, precision), dtype=torch.uint8, device="cuda")
    lam = torch.empty(p.N, dtype=dt_, device="cuda")
    dnu = torch.zeros(1, dtype=torch.float64, device="cuda")
    L.lmep_adjoint_step(h, g, op_of(p), p.dt, u, lam_next, lam, dnu, scratch, precision)
    L.lmep_sync_status(h)
    return lam.cpu().numpy(), dnu.item()


def noalloc(L, p, u, lam_next, precision):
    dt_ = L.state_dtype(precision)
    lam = torch.full((p.N,), float("nan"), dtype=dt_, device="cuda")
    dnu = torch.zeros(1, dtype=torch.float64, device="cuda")
    L.lmep_adjoint_step_noalloc(grid_of(p), op_of(p), p.dt, u, lam_next, lam, dnu, precision)
    torch.cuda.synchronize()
    return lam.cpu().numpy(), dnu.item()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_allocating_entry_point_in_a_row(L, precision):
    h = L.Handle()
    dt_ = L.state_dtype(precision)
    cases = [(wl.burgers(N=257, n=13, cfl=4.0, nu=1e-5, seed=5), 10),       # small grid first
             (wl.burgers(N=4099, n=9, cfl=2.0, nu=1e-6, seed=3), 11),       # then a larger one
             (wl.burgers(N=4099, n=9, cfl=2.0, nu=1e-6, seed=3), 12)]       # same grid, other data
    for k, (p, seed) in enumerate(cases):
        u = torch.tensor(wl.burgers_ic(p.N, seed), dtype=dt_, device="cuda")
        lam_next = torch.tensor(np.random.default_rng(k).standard_normal(p.N), dtype=dt_, device="cuda")
        want_lam, want_dnu = reference(L, h, p, u, lam_next, precision)
        got_lam, got_dnu = noalloc(L, p, u, lam_next, precision)
        assert np.array_equal(got_lam, want_lam), k
        assert abs(got_dnu - want_dnu) <= 1e-9 * max(abs(want_dnu), 1e-300), k
    h.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_oracle(L, precision):
    p = wl.burgers(N=160, n=7, cfl=1.6, nu=2e-4)
    u = wl.burgers_ic(p.N, 3)
    lam_next = np.random.default_rng(1).standard_normal(p.N)
    if precision == "mixed":
        u = u.astype(np.float32).astype(np.float64)
        lam_next = lam_next.astype(np.float32).astype(np.float64)
    dt_ = L.state_dtype(precision)
    got_lam, got_dnu = noalloc(L, p, torch.tensor(u, dtype=dt_, device="cuda"),
                               torch.tensor(lam_next, dtype=dt_, device="cuda"), precision)
    want_lam, want_dnu = oadj.adjoint_step(p, u, lam_next)
    assert rel_linf(got_lam, want_lam) <= 10 * tol(precision)
    D = oop.unit_D(p.n)
    terms = []
    for i in ogrid.updated_points(p):
        idx, r, w, dwu, dwnu = oadj.point_derivatives(p, u, i, D)
        terms.append(lam_next[i] * (dwnu @ u[idx]))
    assert abs(got_dnu - want_dnu) <= 10 * tol(precision) * np.sum(np.abs(terms))


FRESH = r"""
import sys
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + "/tests")
import numpy as np, torch
import paper_2603_15964_gb300 as L
import workloads as wl
from lmep_testutil import grid_of, op_of
p = wl.burgers(N=1025, n=9, cfl=2.0, nu=1e-6)
u = torch.tensor(wl.burgers_ic(p.N, 4), dtype=torch.float64, device="cuda")
ln = torch.tensor(np.random.default_rng(2).standard_normal(p.N), device="cuda")
lam = torch.full((p.N,), float("nan"), dtype=torch.float64, device="cuda")
dnu = torch.zeros(1, dtype=torch.float64, device="cuda")
L.lmep_adjoint_step_noalloc(grid_of(p), op_of(p), p.dt, u, ln, lam, dnu, "fp64")   # before any handle
torch.cuda.synchronize()
h = L.Handle()
L.lmep_set_expm_method(h, "pade")
g = grid_of(p)
s = torch.empty(L.lmep_adjoint_scratch_bytes(g, "fp64"), dtype=torch.uint8, device="cuda")
lam2 = torch.empty_like(lam)
dnu2 = torch.zeros(1, dtype=torch.float64, device="cuda")
L.lmep_adjoint_step(h, g, op_of(p), p.dt, u, ln, lam2, dnu2, s, "fp64")
L.lmep_sync_status(h)
assert torch.equal(lam, lam2)
assert abs(dnu.item() - dnu2.item()) <= 1e-9 * abs(dnu2.item())
print("fresh ok")
"""


def test_noalloc_first_call_of_a_fresh_process(L):
    code = "ROOT = " + repr(ROOT) + "\n" + FRESH
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "fresh ok" in r.stdout, r.stdout + r.stderr


def test_noalloc_size_limit(L):
    """N (n + 1) 8 + 4 N + 256 <= 8 MiB: N = 63548 fits at n = 15 in FP64, N = 63549 does not."""
    for N, fits in ((63548, True), (63549, False)):
        p = wl.burgers(N=N, n=15, cfl=1.0, nu=1e-6)
        u = torch.tensor(wl.burgers_ic(N, 0), dtype=torch.float64, device="cuda")
        lam = torch.zeros_like(u)
        dnu = torch.zeros(1, dtype=torch.float64, device="cuda")
        if fits:
            L.lmep_adjoint_step_noalloc(grid_of(p), op_of(p), p.dt, u, torch.ones_like(u), lam, dnu, "fp64")
            torch.cuda.synchronize()
            assert np.all(np.isfinite(lam.cpu().numpy()))
        else:
            with pytest.raises(L.LmepError) as e:
                L.lmep_adjoint_step_noalloc(grid_of(p), op_of(p), p.dt, u, torch.ones_like(u), lam, dnu, "fp64")
            assert e.value.status == 1 and "static scratch" in str(e.value)
