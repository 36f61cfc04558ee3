"""KdV at the full size of the KdV configuration (Sec. 4.3.2): N = 2^20 periodic points on
[-50, 50), n = 11, ETDRK2, dt = 0.05 h^3, two-soliton initial state.

Parity at full size on sampled windows: one ETDRK2 step at point i reads the state within
4 h_s of i (first stage, its N(.), the second stage), so K steps of the full problem agree
at the interior points of any 4096-point window with K steps of the oracle run on that
window as a periodic problem of the same h and dt (the artificial wrap reaches only the
outer 4 h_s K points).  The windows include one across the periodic seam and the two
solitons.  Tolerances: K x 1e-12 (FP64) and K x 1e-5 (FP32 form) relative to max |u|.

Long horizon (2000 steps, the configuration's length): the mass h sum u is an invariant of
the discrete scheme (stored rows sum to one; sum_i u_i (D1 u)_i = 0 for the centred,
antisymmetric periodic D1), and the energy h sum u^2 of the PDE moves by O(T) with
T = 2000 dt; the FP32-form trajectory stays within the FP32 rounding walk of the FP64 one.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import lmep as olmep

from lmep_testutil import grid_of, op_of, tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_FULL = 1 << 20


@pytest.fixture(scope="module")
def L():
    import paper_2603_15964_gb300 as L
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return L


@pytest.fixture(scope="module")
def H(L):
    return L.Handle()


def full_problem():
    return wl.kdv(N=N_FULL, n=11, L=50.0)


def run_gpu(L, H, p, u0, steps, precision):
    dt_ = L.state_dtype(precision)
    W = torch.empty(p.n, 1 + p.n_phi, p.n, dtype=dt_, device="cuda")
    L.lmep_harvest_weights(H, grid_of(p), op_of(p), p.dt, p.n_phi, None, W, precision)
    u = torch.tensor(u0, dtype=dt_, device="cuda")
    work = torch.empty_like(u)
    if steps:
        L.lmep_step(H, grid_of(p), op_of(p), p.scheme, p.nonlin, p.dt, W, u, work, steps, precision)
    L.lmep_sync_status(H)
    return u.double().cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_windows_match_oracle(L, H, precision):
    p = full_problem()
    u0 = wl.kdv_ic(p, 0)
    if precision == "mixed":
        u0 = u0.astype(np.float32).astype(np.float64)
    K = 3
    got = run_gpu(L, H, p, u0, K, precision)
    M = 4096
    margin = 4 * ((p.n - 1) // 2) * K + 8
    sub = p.with_(N=M, a=0.0, b=M * p.h)
    assert abs(sub.h - p.h) <= 1e-15 * p.h
    scale = np.max(np.abs(u0))
    half = N_FULL // 2
    peak1 = int(np.argmax(u0[:half]))
    peak2 = half + int(np.argmax(u0[half:]))
    starts = [N_FULL - M // 2, 123457, peak1 - M // 2, peak2 - M // 2]
    for s in starts:
        idx = (s + np.arange(M)) % N_FULL
        want = olmep.run(sub, u0[idx], K)
        inner = slice(margin, M - margin)
        err = np.max(np.abs(got[idx][inner] - want[inner])) / scale
        assert err <= tol(precision) * K, (s, err)


def test_long_horizon_invariants_and_precisions(L, H):
    p = full_problem()
    u0 = wl.kdv_ic(p, 0)
    steps = 2000
    u64 = run_gpu(L, H, p, u0, steps, "fp64")
    u32 = run_gpu(L, H, p, u0.astype(np.float32).astype(np.float64), steps, "mixed")
    m0, e0 = p.h * np.sum(u0), p.h * np.sum(u0 ** 2)
    assert np.all(np.isfinite(u64)) and np.all(np.isfinite(u32))
    assert abs(p.h * np.sum(u64) - m0) <= 1e-11 * abs(m0)
    assert abs(p.h * np.sum(u64 ** 2) - e0) <= 1e-9 * e0
    assert abs(p.h * np.sum(u32) - m0) <= 1e-4 * abs(m0)
    assert abs(p.h * np.sum(u32 ** 2) - e0) <= 1e-4 * e0
    scale = np.max(np.abs(u0))
    assert np.max(np.abs(u32 - u64)) / scale <= tol("mixed") * steps
