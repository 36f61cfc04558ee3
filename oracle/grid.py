"""Stencil selection per grid point (oracle).

Sec. 2.1 steps 1 and 3: each point x_i is updated from a local stencil S_n of
n nodes; interior points use the centre row, points near a non-periodic
boundary use an edge row (Example 1 harvests the first and last rows).

Readings (the paper does not define the window placement):
* periodic: centred window, indices taken mod N, harvested row (n-1)/2;
* Dirichlet: window start clamp(i - hs - k, 0, N - n), row i - start, so the
  window slides inside the domain and becomes one-sided near a wall; wall
  values are data but are never updated;
* Neumann (homogeneous): centred window with even reflection about the wall
  node (index q -> -q below 0, q -> 2(N-1) - q above N-1), i.e. the periodic
  problem on the mirrored grid of 2(N-1) points;
* departure centring: the window is shifted upstream by
  k_i = clamp(floor(u_i dt / h + 1/2), -hs, hs) so that the semi-Lagrangian
  departure point x_i - u_i dt (Thm. 1) sits near the window centre.
Test infrastructure only.
"""
from __future__ import annotations

import math

import numpy as np

from workloads import DIRICHLET, NEUMANN, PERIODIC, Problem


def half_width(n: int) -> int:
    return (n - 1) // 2


def departure_shift(u_i: float, dt: float, h: float, n: int) -> int:
    hs = half_width(n)
    k = math.floor(u_i * dt / h + 0.5)
    return max(-hs, min(hs, k))


def reflect(q: int, N: int) -> int:
    if q < 0:
        return -q
    if q > N - 1:
        return 2 * (N - 1) - q
    return q


def stencil(p: Problem, i: int, k: int = 0):
    """Global indices of the n window nodes of point i and the row harvested for it."""
    n, N, hs = p.n, p.N, half_width(p.n)
    if p.bc == PERIODIC:
        start = i - hs - k
        return np.array([(start + j) % N for j in range(n)]), hs + k
    if p.bc == DIRICHLET:
        start = min(max(i - hs - k, 0), N - n)
        return np.arange(start, start + n), i - start
    if p.bc == NEUMANN:
        start = i - hs - k
        return np.array([reflect(start + j, N) for j in range(n)]), hs + k
    raise ValueError(p.bc)


def updated_points(p: Problem) -> range:
    """Dirichlet walls keep their boundary values; every other point is updated."""
    return range(1, p.N - 1) if p.bc == DIRICHLET else range(p.N)
