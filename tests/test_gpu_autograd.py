"""Adjoint through torch.autograd with step checkpointing (frozen-velocity Burgers).

J = (h/2) sum_b ||u_b(T) - u*_b||^2.  The gradient with respect to the
initial states and nu is checked against the FP64 oracle's reverse sweep
(oracle.adjoint.gradient, one instance at a time), against central
differences of the GPU forward pass, and for independence of the checkpoint
interval.  Tolerances: FP64 path 1e-9 relative (a gradient through T steps of
Frechet derivatives), FP32 form 1e-4.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import adjoint as oadj

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import paper_2603_15964_gb300 as L
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return L


def problem(steps=7):
    return wl.burgers(N=64, n=7, cfl=1.5, nu=3e-4, steps=steps, departure_centring=True)


def solver_for(p, precision, K):
    from paper_2603_15964_gb300.autograd import FrozenVelocitySolver
    return FrozenVelocitySolver(N=p.N, h=p.h, n=p.n, dt=p.dt, steps=p.steps, precision=precision,
                                checkpoint_every=K)


def loss_and_grads(L, p, precision, K, u0, target):
    dt_ = L.state_dtype(precision)
    x = torch.tensor(u0, dtype=dt_, device="cuda", requires_grad=True)
    nu = torch.tensor(p.c2, dtype=torch.float64, requires_grad=True)
    uT = solver_for(p, precision, K)(x, nu)
    J = 0.5 * p.h * ((uT.double() - torch.tensor(target, device="cuda")) ** 2).sum()
    J.backward()
    return float(J), x.grad.double().cpu().numpy(), float(nu.grad)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gradient_matches_oracle(L, precision):
    p = problem()
    B = 2
    u0 = np.stack([wl.burgers_ic(p.N, 3 + b) for b in range(B)])
    target = np.stack([wl.burgers_ic(p.N, 1003 + b) for b in range(B)])
    if precision == "mixed":
        u0 = u0.astype(np.float32).astype(np.float64)
    J, gu, gnu = loss_and_grads(L, p, precision, 3, u0, target)
    want_J, want_nu = 0.0, 0.0
    want_u = np.zeros_like(u0)
    for b in range(B):
        Jb, gb, nb = oadj.gradient(p, u0[b], target[b], p.steps)
        want_J += Jb
        want_u[b] = gb
        want_nu += nb
    tol = 1e-9 if precision == "fp64" else 1e-4
    assert abs(J - want_J) <= tol * abs(want_J) + (0 if precision == "fp64" else 1e-6)
    assert np.max(np.abs(gu - want_u)) <= tol * np.max(np.abs(want_u))
    assert abs(gnu - want_nu) <= tol * abs(want_nu)


def test_checkpoint_interval_does_not_change_the_gradient(L):
    p = problem(steps=9)
    u0 = np.stack([wl.burgers_ic(p.N, 8)])
    target = np.stack([wl.burgers_ic(p.N, 1008)])
    a = loss_and_grads(L, p, "fp64", 2, u0, target)
    b = loss_and_grads(L, p, "fp64", 100, u0, target)
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1])
    # dJ/dnu is summed with FP64 atomics across CTAs: same value up to summation order
    assert abs(a[2] - b[2]) <= 1e-13 * abs(a[2])


def test_gradient_matches_central_differences_of_the_gpu_forward(L):
    p = problem(steps=5)
    u0 = np.stack([wl.burgers_ic(p.N, 11)])
    target = np.stack([wl.burgers_ic(p.N, 1011)])
    J, gu, gnu = loss_and_grads(L, p, "fp64", 2, u0, target)
    s = solver_for(p, "fp64", 2)

    def J_of(u_init, nu):
        x = torch.tensor(u_init, dtype=torch.float64, device="cuda")
        uT = s(x, torch.tensor(nu, dtype=torch.float64))
        return 0.5 * p.h * float(((uT - torch.tensor(target, device="cuda")) ** 2).sum())

    for i in (5, 20, 33, 58):
        e = 1e-6
        up, um = u0.copy(), u0.copy()
        up[0, i] += e
        um[0, i] -= e
        fd = (J_of(up, p.c2) - J_of(um, p.c2)) / (2 * e)
        assert abs(fd - gu[0, i]) <= 1e-6 * max(abs(fd), 1e-3 * np.max(np.abs(gu)))
    e = 1e-3 * p.c2
    fd_nu = (J_of(u0, p.c2 + e) - J_of(u0, p.c2 - e)) / (2 * e)
    assert abs(fd_nu - gnu) <= 1e-5 * abs(fd_nu)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n,cfl,nu,N,steps", [(9, 2.0, 1e-6, 512, 2), (13, 4.0, 1e-6, 300, 1), (7, 1.0, 1e-3, 257, 3)])
def test_gradient_matches_oracle_across_configs(L, precision, n, cfl, nu, N, steps):
    p = wl.burgers(N=N, n=n, cfl=cfl, nu=nu, steps=steps, departure_centring=True)
    B = 3
    u0 = np.stack([wl.burgers_ic(p.N, 20 + b) for b in range(B)])
    target = np.stack([wl.burgers_ic(p.N, 1020 + b) for b in range(B)])
    if precision == "mixed":
        u0 = u0.astype(np.float32).astype(np.float64)
    J, gu, gnu = loss_and_grads(L, p, precision, 2, u0, target)
    want_u = np.zeros_like(u0)
    want_nu = 0.0
    for b in range(B):
        _, gb, nb = oadj.gradient(p, u0[b], target[b], p.steps)
        want_u[b] = gb
        want_nu += nb
    # Sizes above 2 x 152 points make the adjoint kernel's warps loop over several points.
    # dJ/dnu: the nu direction E = dt/h^2 Dh2 is about 1e3 times X in norm at n = 13, CFL 4;
    # the GPU's differentiated Pade and the oracle's Frechet evaluation round differently at
    # ~1e-9 relative per term there (the sum itself cancels only by a factor ~2), hence 1e-8.
    tol = 1e-9 if precision == "fp64" else 1e-4
    tol_nu = 1e-8 if precision == "fp64" else 1e-4
    err_u = np.max(np.abs(gu - want_u)) / np.max(np.abs(want_u))
    err_nu = abs(gnu - want_nu) / abs(want_nu)
    assert err_u <= tol and err_nu <= tol_nu, (err_u, err_nu, int(np.argmax(np.max(np.abs(gu - want_u), axis=0))))


def test_fp32_form_gradient_on_a_fine_grid(L):
    """Configuration 5's grid (N = 262144, n = 9, CFL 2, nu = 1e-6): the FP32 form's gradient against the
    FP64 path's over 16 steps from the same FP32 initial state.  On this grid dw/du and dw/dnu applied to
    the window are first and second differences some 1e-5 and 1e-9 of the values they difference, so an
    FP32 evaluation that rounded the values themselves would lose them; the gradients must agree to the
    FP32 forward's own precision (1e-3 relative, the two trajectories differ by FP32 rounding)."""
    p = wl.burgers(N=262144, n=9, cfl=2.0, nu=1e-6, steps=16, departure_centring=True)
    u0 = wl.burgers_ic(p.N, 0)[None, :].astype(np.float32).astype(np.float64)
    target = wl.burgers_ic(p.N, 1000)[None, :]
    _, g32, n32 = loss_and_grads(L, p, "mixed", 4, u0, target)
    _, g64, n64 = loss_and_grads(L, p, "fp64", 4, u0, target)
    v = np.random.default_rng(5).standard_normal(u0.shape)
    d32, d64 = float(np.sum(g32 * v)), float(np.sum(g64 * v))
    assert abs(d32 - d64) <= 1e-3 * abs(d64), (d32, d64)
    assert np.max(np.abs(g32 - g64)) <= 1e-3 * np.max(np.abs(g64))
    assert abs(n32 - n64) <= 1e-3 * abs(n64), (n32, n64)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_set_forward_equals_batched_step(L, precision):
    """The solver steps a batch as a frozen set (one launch per step over all states) or through lmep_step
    on the batched grid: the same final states and gradients in u0, bit for bit (dJ/dnu to its
    summation order)."""
    from paper_2603_15964_gb300.autograd import FrozenVelocitySolver
    p = wl.burgers(N=4096, n=9, cfl=2.0, nu=1e-5, steps=9, departure_centring=True)
    dt_ = L.state_dtype(precision)
    u0 = torch.tensor(np.stack([wl.burgers_ic(p.N, 20 + b) for b in range(3)]), dtype=dt_, device="cuda")
    target = torch.tensor(np.stack([wl.burgers_ic(p.N, 40 + b) for b in range(3)]), device="cuda")
    out = []
    for use_set in (True, False):
        solver = FrozenVelocitySolver(N=p.N, h=p.h, n=p.n, dt=p.dt, steps=p.steps, precision=precision,
                                      checkpoint_every=4, use_set=use_set)
        x = u0.clone().requires_grad_(True)
        nu = torch.tensor(p.c2, dtype=torch.float64, requires_grad=True)
        uT = solver(x, nu)
        (0.5 * p.h * ((uT.double() - target) ** 2).sum()).backward()
        out.append((uT.detach().clone(), x.grad.clone(), float(nu.grad)))
    (a, ga, na), (b, gb, nb) = out
    assert torch.equal(a, b) and torch.equal(ga, gb)
    assert abs(na - nb) <= 1e-12 * abs(nb)      # dJ/dnu is summed with atomic adds: the order varies
