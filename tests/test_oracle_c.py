"""Pins of the C build of the frozen-velocity oracle step (oracle/c/lmep_oracle.c).

* Thm. 1: without diffusion the harvested row is the Lagrange interpolation at the departure point
  x_i - u_i dt, so the step equals that interpolant of the window data (written out here from the
  Lagrange formula, independently of any exponential), at integer and fractional Courant numbers,
  with and without departure centring, next to the walls too.
* Weights sum to e^{dt c0} (Sec. 2.1: the local operator annihilates constants): a constant state
  stays constant (times e^{dt c0}).
* The numpy oracle (pinned on its own in test_oracle_pins.py): every point of small grids of every
  boundary condition, width and viscosity agrees within 1e-12.
* Dirichlet walls keep their values; a subset of points equals the same points of a full step.
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import cpu, grid as ogrid, lmep as olmep


@pytest.fixture(scope="module", autouse=True)
def built():
    cpu.build()


def lagrange_at(z, n):
    """l_j(z) on the integer nodes 0..n-1."""
    out = np.empty(n)
    for j in range(n):
        v = 1.0
        for m in range(n):
            if m != j:
                v *= (z - m) / (j - m)
        out[j] = v
    return out


@pytest.mark.parametrize("n,cfl,dep", [(7, 1.0, True), (9, 2.5, True), (13, 3.7, True), (5, 0.6, False),
                                       (11, 1.3, False)])
def test_pure_advection_is_lagrange_interpolation(n, cfl, dep):
    p = wl.burgers(N=301, n=n, cfl=cfl, nu=0.0, departure_centring=dep)
    u = wl.burgers_ic(301, 5)
    got = cpu.frozen_step(p, u)
    for i in range(1, p.N - 1):
        k = ogrid.departure_shift(u[i], p.dt, p.h, n) if dep else 0
        idx, r = ogrid.stencil(p, i, k)
        z = r - u[i] * p.dt / p.h                   # departure point in window coordinates
        want = lagrange_at(z, n) @ u[idx]
        assert abs(got[i] - want) <= 1e-12 * max(1.0, np.max(np.abs(lagrange_at(z, n)))), (i, got[i], want)


@pytest.mark.parametrize("bc", ["dirichlet", "periodic", "neumann"])
@pytest.mark.parametrize("c0", [0.0, -0.7])
def test_constants_are_preserved(bc, c0):
    p = wl.burgers(N=200, n=9, cfl=2.0, nu=1e-4).with_(bc=bc, c0=c0, bc_lo=1.0, bc_hi=1.0)
    u = np.ones(p.N)
    # the frozen speed is u_i = 1 everywhere; the step maps constants to e^{dt c0} constants
    got = cpu.frozen_step(p, u)
    want = math.exp(p.dt * c0)
    inner = got[1:-1] if bc == "dirichlet" else got
    assert np.max(np.abs(inner - want)) <= 1e-12


@pytest.mark.parametrize("bc", ["dirichlet", "periodic", "neumann"])
@pytest.mark.parametrize("n,cfl,nu", [(13, 4.0, 1e-6), (7, 1.0, 1e-3), (9, 2.0, 1e-5), (11, 2.5, 3e-4),
                                      (5, 3.0, 4e-4), (15, 1.5, 1e-6), (3, 0.8, 1e-6)])
def test_matches_numpy_oracle(bc, n, cfl, nu):
    p = wl.burgers(N=257, n=n, cfl=cfl, nu=nu).with_(bc=bc)
    u = wl.burgers_ic(257, 3) + (0.05 * np.cos(np.pi * p.nodes()) if bc != "dirichlet" else 0.0)
    got = cpu.frozen_step(p, u)
    want = olmep.frozen_step(p, u)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_walls_and_point_subsets():
    p = wl.burgers(N=1000, n=13, cfl=4.0, nu=1e-6).with_(bc_lo=0.25, bc_hi=-0.5)
    u = wl.burgers_ic(1000, 2)
    full = cpu.frozen_step(p, u, threads=2)
    assert full[0] == 0.25 and full[-1] == -0.5
    pts = np.array([0, 1, 2, 500, 997, 998, 999])
    part = cpu.frozen_step(p, u, pts, threads=1)
    assert np.array_equal(part, full[pts])
