"""Seeded synthetic workloads for the LMEP hot path.

This module is shared by the FP64 oracle, the GPU parity tests and the
benchmark.  It holds only problem definitions (domains, grid sizes, time
steps, coefficients) and seeded initial conditions.  It contains none of the
method's arithmetic: no stencils, no derivative weights, no exponentials.

The workloads follow the paper's test problems (Section 4): periodic
advection-diffusion (Sec. 4.2), viscous Burgers (Sec. 4.3.1), KdV
(Sec. 4.3.2) and Allen-Cahn (Sec. 4.3.3), in the sizes used for the
GB300 measurements.  Every random draw comes from
``numpy.random.default_rng(seed)`` so both sides see identical inputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

PERIODIC, DIRICHLET, NEUMANN = "periodic", "dirichlet", "neumann"
BC_CODE = {PERIODIC: 0, DIRICHLET: 1, NEUMANN: 2}
SCHEME_CODE = {"linear": 0, "etd1": 1, "etdrk2": 2, "etdrk4": 3}
NONLIN_CODE = {"none": 0, "allen_cahn": 1, "kdv": 2, "burgers": 3}


@dataclass(frozen=True)
class Problem:
    """One 1-D LMEP problem on a uniform grid.

    The linear operator is L = c0 + c1 d/dx + c2 d^2/dx^2 + c3 d^3/dx^3; with
    ``frozen_adv`` != 0 each point i adds -frozen_adv*u_i*d/dx with its own
    current value u_i frozen (locally linearised Burgers).
    """

    name: str
    N: int
    a: float
    b: float
    bc: str
    n: int
    dt: float
    c0: float = 0.0
    c1: float = 0.0
    c2: float = 0.0
    c3: float = 0.0
    frozen_adv: float = 0.0
    scheme: str = "linear"
    nonlin: str = "none"
    departure_centring: bool = False
    steps: int = 1
    bc_lo: float = 0.0
    bc_hi: float = 0.0
    window_shift: int = 0       # constant coefficients: every window shifted upstream by this many nodes
    meta: dict = field(default_factory=dict, compare=False, hash=False)

    @property
    def h(self) -> float:
        # periodic: N points on [a, b) ; walls: N points on [a, b] incl. both walls
        return (self.b - self.a) / (self.N if self.bc == PERIODIC else self.N - 1)

    @property
    def n_phi(self) -> int:
        return {"linear": 0, "etd1": 1, "etdrk2": 2, "etdrk4": 3}[self.scheme]

    def nodes(self) -> np.ndarray:
        return self.a + self.h * np.arange(self.N, dtype=np.float64)

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)


# ---------------------------------------------------------------- config 1
def advection_diffusion(N: int = 256, n: int = 5, cfl: float = 0.8, c: float = 1.0,
                        nu: float = 0.01, steps: int = 100) -> Problem:
    """Periodic u_t + c u_x = nu u_xx on [0, 2 pi) (paper Sec. 4.2 family)."""
    p = Problem("advection_diffusion", N, 0.0, 2 * math.pi, PERIODIC, n, 0.0,
                c1=-c, c2=nu, scheme="linear", steps=steps)
    return p.with_(dt=cfl * p.h / abs(c))


def advection_diffusion_ic(p: Problem) -> np.ndarray:
    x = p.nodes()
    return np.sin(x) + np.exp(-20.0 * (x - math.pi) ** 2)


# ---------------------------------------------------------------- config 2
def burgers_ic(N: int, seed: int = 0, bumps: int = 8) -> np.ndarray:
    """-sin(pi x) plus seeded Gaussian bumps of amplitude 0.1 on [-1, 1], zero walls."""
    rng = np.random.default_rng(seed)
    xb = rng.uniform(-0.9, 0.9, bumps)
    sb = rng.uniform(0.01, 0.05, bumps)
    x = -1.0 + (2.0 / (N - 1)) * np.arange(N, dtype=np.float64)
    u = -np.sin(np.pi * x)
    for k in range(bumps):
        u += 0.1 * np.exp(-(((x - xb[k]) / sb[k]) ** 2))
    u[0] = 0.0
    u[-1] = 0.0
    return u


def burgers(N: int = 65536, n: int = 13, cfl: float = 4.0, nu: float = 1e-6,
            steps: int = 1000, seed: int = 0, departure_centring: bool = True) -> Problem:
    """Viscous Burgers on [-1, 1], u = 0 at both walls, velocity frozen per point.

    ``dt = cfl * h / max|u0|``.  nu = 1e-3 is the size as first stated
    (unstable for these stencils); nu = 1e-6 is the stable variant.
    """
    u0 = burgers_ic(N, seed)
    p = Problem("burgers", N, -1.0, 1.0, DIRICHLET, n, 0.0, c2=nu, frozen_adv=1.0,
                scheme="linear", departure_centring=departure_centring, steps=steps,
                meta={"cfl": cfl, "seed": seed})
    return p.with_(dt=cfl * p.h / float(np.max(np.abs(u0))))


# ---------------------------------------------------------------- config 3
@dataclass(frozen=True)
class AllenCahnBatch:
    """Many independent Allen-Cahn instances u_t = eps2 u_xx + u - u^3 on [-1, 1]."""

    Ns: np.ndarray          # int64 [B]
    bcs: list               # PERIODIC or NEUMANN per instance
    eps2: float
    n: int
    dt: float
    scheme: str
    steps: int
    seed: int

    def problem(self, b: int) -> Problem:
        return Problem(f"allen_cahn[{b}]", int(self.Ns[b]), -1.0, 1.0, self.bcs[b], self.n,
                       self.dt, c2=self.eps2, scheme=self.scheme, nonlin="allen_cahn",
                       steps=self.steps)


def allen_cahn_batch(B: int = 4096, Nmin: int = 1024, Nmax: int = 65536, n: int = 9,
                     eps2: float = 1e-4, scheme: str = "etdrk2", steps: int = 1000,
                     seed: int = 0, mu_max: float = 0.5) -> AllenCahnBatch:
    rng = np.random.default_rng(seed)
    Ns = np.rint(np.exp(rng.uniform(math.log(Nmin), math.log(Nmax), B))).astype(np.int64)
    bcs = [PERIODIC if flip else NEUMANN for flip in rng.random(B) < 0.5]
    hmin = min((2.0 / N if bc == PERIODIC else 2.0 / (N - 1)) for N, bc in zip(Ns, bcs))
    dt = mu_max * hmin * hmin / eps2
    return AllenCahnBatch(Ns, bcs, eps2, n, dt, scheme, steps, seed)


def allen_cahn_ic(N: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return 0.1 * np.tanh(rng.uniform(-1.0, 1.0, N))


def allen_cahn(N: int, bc: str = PERIODIC, n: int = 9, eps2: float = 1e-4, dt: float | None = None,
               scheme: str = "etdrk2", steps: int = 10, mu: float = 0.5) -> Problem:
    p = Problem("allen_cahn", N, -1.0, 1.0, bc, n, 0.0, c2=eps2, scheme=scheme,
                nonlin="allen_cahn", steps=steps)
    return p.with_(dt=dt if dt is not None else mu * p.h * p.h / eps2)


# ---------------------------------------------------------------- config 4
def kdv(N: int = 1 << 20, n: int = 11, L: float = 50.0, mu3: float = 0.05,
        scheme: str = "etdrk2", steps: int = 2000) -> Problem:
    """KdV u_t + 6 u u_x + u_xxx = 0, periodic on [-L, L): L = -d^3/dx^3, N(u) = -6 u u_x."""
    p = Problem("kdv", N, -L, L, PERIODIC, n, 0.0, c3=-1.0, scheme=scheme, nonlin="kdv",
                steps=steps)
    return p.with_(dt=mu3 * p.h ** 3)


def kdv_ic(p: Problem, seed: int = 0) -> np.ndarray:
    """Two-soliton sum 2 k_j^2 sech^2(k_j (x - x_j)), seeded k_j and x_j."""
    rng = np.random.default_rng(seed)
    kap = rng.uniform(0.4, 0.9, 2)
    xs = np.array([rng.uniform(-30.0, -10.0), rng.uniform(0.0, 20.0)])
    scale = (p.b - p.a) / 100.0          # keep the solitons inside smaller test domains
    x = p.nodes()
    u = np.zeros_like(x)
    for k, x0 in zip(kap, xs * scale):
        u += 2.0 * k * k / np.cosh(k * (x - x0)) ** 2
    return u


# ---------------------------------------------------------------- high-CFL advection (Sec. 4.1)
def advection(N: int = 256, n: int = 9, sigma: float = 0.5, one_sided: bool = True, a: float = 1.0,
              periods: float = 100.0) -> Problem:
    """u_t + a u_x = 0, periodic on [-1, 1), IC exp(-40 x^2) (Sec. 4.1).  Courant number
    nu = (n + 1)/2 - sigma with fully upwind (one-sided) windows, nu = 1 - sigma with centred ones;
    dt = nu h / a; `steps` covers `periods` periods (rounded to whole steps)."""
    p = Problem("advection", N, -1.0, 1.0, PERIODIC, n, 0.0, c1=-a, scheme="linear",
                window_shift=(n - 1) // 2 if one_sided else 0)
    nu = (n + 1) / 2.0 - sigma if one_sided else 1.0 - sigma
    dt = nu * p.h / abs(a)
    steps = int(round(periods * (p.b - p.a) / abs(a) / dt))
    return p.with_(dt=dt, steps=steps, meta={"nu": nu, "sigma": sigma, "one_sided": one_sided})


def advection_ic(p: Problem) -> np.ndarray:
    return np.exp(-40.0 * p.nodes() ** 2)


def advection_exact(p: Problem, t: float) -> np.ndarray:
    """The initial profile carried by a t, wrapped periodically (the exact solution)."""
    L = p.b - p.a
    x = p.nodes()
    xi = (x + p.c1 * t - p.a) % L + p.a          # departure point x - a t, c1 = -a
    return np.exp(-40.0 * xi ** 2)


# ---------------------------------------------------------------- Burgers with ETD (Sec. 4.3.1)
def burgers_etd(N: int = 128, n: int = 13, nu: float = 0.03, dt: float = 1e-2, scheme: str = "etdrk4",
                steps: int = 100) -> Problem:
    """Viscous Burgers u_t + u u_x = nu u_xx, periodic on [-pi, pi): L = nu d^2/dx^2 (exponentiated),
    N(u) = -u u_x (the paper's Sec. 4.3.1 benchmark, nu = 0.03)."""
    return Problem("burgers_etd", N, -math.pi, math.pi, PERIODIC, n, dt, c2=nu, scheme=scheme,
                   nonlin="burgers", steps=steps)


def burgers_etd_ic(p: Problem) -> np.ndarray:
    """exp(-10 sin^2(x / 2)) (Sec. 4.3.1)."""
    return np.exp(-10.0 * np.sin(p.nodes() / 2.0) ** 2)


# ---------------------------------------------------------------- config 5
def burgers_batch_ic(N: int, batch: int, seed0: int = 0) -> np.ndarray:
    return np.stack([burgers_ic(N, seed0 + b) for b in range(batch)])


def burgers_target(N: int, batch: int) -> np.ndarray:
    return burgers_batch_ic(N, batch, seed0=1000)
