"""Frozen-velocity sets: several instances (own N, width, boundary, dt, viscosity) advanced by one
persistent launch per step (lmep_frozen_set_*), through the C ABI.

* Bit for bit equal to lmep_step on each instance (same arithmetic in both paths: the factorised
  rows of the lean kernel and the finite-series / Pade stages of the fallback launch), over several
  steps, with every route and boundary; at nu = 4e-4 and 1e-3 the lean kernel rejects points
  (mixed routes in one step) and the fallback's counters must be cleared between steps.
* Against the FP64 oracle (Sec. 2.1 steps 1-3, Sec. 3.1 step 3): K-step trajectories at 1e-12 K
  (FP64) and 1e-5 K (FP32 form); one step of the nine-instance benchmark set at N = 65536 on sampled
  points, the exact rational row deciding where the FP64 oracle's exponential of the rounded
  local matrix is itself off.
* Graph replay equals eager steps; invalid descriptors launch nothing.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import lmep as olmep, operator as oop

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


def mixed_probs():
    """Instances of every width, both wall types, periodic, ragged sizes and three viscosities."""
    out = [wl.burgers(N=4099, n=7, cfl=2.0, nu=1e-6, seed=1),
           wl.burgers(N=2048, n=13, cfl=4.0, nu=4e-4, seed=2),                 # factorised + fallback
           wl.burgers(N=3001, n=9, cfl=1.0, nu=1e-6, seed=3),
           wl.burgers(N=515, n=5, cfl=3.0, nu=3e-4, seed=4),                   # mostly fallback
           wl.burgers(N=130, n=15, cfl=1.5, nu=1e-6, seed=5),
           wl.burgers(N=1000, n=11, cfl=2.5, nu=1e-5, seed=6).with_(bc=wl.NEUMANN),
           wl.burgers(N=777, n=3, cfl=0.8, nu=1e-6, seed=7).with_(bc=wl.PERIODIC)]
    return out


def ic_of(p, seed):
    u = wl.burgers_ic(p.N, seed)
    if p.bc != wl.DIRICHLET:
        u = u + 0.05 * np.cos(np.pi * p.nodes())
    return u


def same_bits(a, b) -> bool:
    """Bitwise equality of two float tensors (NaN payloads included)."""
    it = torch.int32 if a.dtype == torch.float32 else torch.int64
    return a.shape == b.shape and torch.equal(a.contiguous().view(it), b.contiguous().view(it))


def make_set(L, probs, precision, method="auto", block=0, ppt=0, handle=None):
    from paper_2603_15964_gb300.frozen import FrozenInstance, FrozenSet
    insts = [FrozenInstance(grid_of(p), op_of(p), p.dt) for p in probs]
    return FrozenSet(insts, precision=precision, method=method, handle=handle, block=block, points_per_thread=ppt)


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("method", ["auto", "series", "pade"])
@pytest.mark.parametrize("block,ppt", [(0, 0), (64, 1), (512, 1), (128, 2), (64, 4), (128, 8)])
def test_set_equals_single_instance_steps(L, precision, method, block, ppt):
    if method == "pade" and (block, ppt) != (0, 0):
        pytest.skip("the Pade route does not depend on the launch shape of the lean kernel")
    probs = mixed_probs()
    u0 = [ic_of(p, s) for s, p in enumerate(probs)]
    K = 4
    fs = make_set(L, probs, precision, method, block, ppt)
    fs.load(u0)
    fs.step(K)
    L.lmep_sync_status(fs.handle)
    h = L.Handle()
    L.lmep_set_expm_method(h, method)
    dt_ = L.state_dtype(precision)
    for b, (p, u) in enumerate(zip(probs, u0)):
        v = torch.tensor(u, dtype=dt_, device="cuda")
        L.lmep_step(h, grid_of(p), op_of(p), "linear", "none", p.dt, None, v, torch.empty_like(v), K, precision)
        L.lmep_sync_status(h)
        assert same_bits(fs.states[b], v), (b, p.n, p.bc)
    h.close()


@pytest.mark.parametrize("precision", PRECS)
def test_set_trajectory_matches_oracle(L, precision):
    """K-step trajectories of the mixed set against the oracle, element by element."""
    probs = [p for p in mixed_probs() if p.c2 <= 1e-5]          # the stable instances
    u0 = [ic_of(p, s) for s, p in enumerate(probs)]
    if precision == "mixed":
        u0 = [u.astype(np.float32).astype(np.float64) for u in u0]
    K = 6
    fs = make_set(L, probs, precision)
    fs.load(u0)
    fs.step(K)
    L.lmep_sync_status(fs.handle)
    for b, (p, u) in enumerate(zip(probs, u0)):
        want = olmep.run(p, u, K)
        assert rel_linf(fs.states[b].cpu().numpy(), want) <= tol(precision) * K, (b, p.n, p.bc)


@pytest.mark.parametrize("precision", PRECS)
def test_bench_set_full_size_sampled(L, precision):
    """The nine-instance benchmark set (N = 65536, n in {7, 9, 13} x CFL in {1, 2, 4}, nu = 1e-6), one
    step in one launch, against the oracle at sampled points (walls and their neighbours included)."""
    from test_gpu_parity import exact_row
    N = 65536
    probs = [wl.burgers(N=N, n=n, cfl=c, nu=1e-6) for n in (7, 9, 13) for c in (1.0, 2.0, 4.0)]
    u0 = wl.burgers_ic(N, 0)
    if precision == "mixed":
        u0 = u0.astype(np.float32).astype(np.float64)
    fs = make_set(L, probs, precision)
    fs.load([u0] * len(probs))
    fs.step(1)
    L.lmep_sync_status(fs.handle)
    scale = np.max(np.abs(u0))
    rng = np.random.default_rng(11)
    decided = 0
    for b, p in enumerate(probs):
        got = fs.states[b].cpu().numpy()
        assert got[0] == 0.0 and got[-1] == 0.0
        D = oop.unit_D(p.n)
        pts = sorted(set(rng.integers(1, N - 1, 120).tolist()) | {1, 2, 3, 7, N - 8, N - 3, N - 2})
        for i in pts:
            idx, r, w = olmep.point_weights(p, u0, i, D)
            if abs(got[i] - w[0] @ u0[idx]) <= tol(precision) * scale:
                continue
            assert precision == "fp64", (b, i)
            ex = exact_row(p.n, -p.dt * u0[i] / p.h, p.dt * p.c2 / p.h ** 2, r)
            assert abs(got[i] - ex @ u0[idx]) <= tol(precision) * scale, (b, i)
            decided += 1
    assert decided <= 40


@pytest.mark.parametrize("precision", PRECS)
def test_set_graph_replay_matches_eager(L, precision):
    probs = mixed_probs()
    u0 = [ic_of(p, s) for s, p in enumerate(probs)]
    K = 7
    eager = make_set(L, probs, precision)
    eager.load(u0)
    eager.step(K)
    graph = make_set(L, probs, precision)
    graph.load(u0)
    graph.capture()                 # two eager steps, one per direction of the ping-pong
    graph.replay(K - 2)
    torch.cuda.synchronize()
    for a, b in zip(eager.states, graph.states):
        assert same_bits(a, b)


@pytest.mark.parametrize("precision", PRECS)
def test_set_graph_replay_without_rejections(L, precision):
    # nu = 1e-6: every point takes the factorised row, so every fallback launch leaves at once; the
    # replayed states equal eager steps bit for bit and the counters (per-instance counts, the fallback's
    # arrival counter, the total) stay clear
    probs = [wl.burgers(N=5000, n=13, cfl=4.0, nu=1e-6, seed=11), wl.burgers(N=3333, n=7, cfl=1.0, nu=1e-6, seed=12)]
    u0 = [ic_of(p, s) for s, p in enumerate(probs)]
    eager = make_set(L, probs, precision)
    eager.load(u0)
    eager.step(6)
    graph = make_set(L, probs, precision)
    graph.load(u0)
    graph.capture()
    graph.replay(4)
    torch.cuda.synchronize()
    for a, b in zip(eager.states, graph.states):
        assert same_bits(a, b)
    ctl = graph.workspace[:4 * (len(probs) + 2)].view(torch.int32).cpu().tolist()
    assert ctl == [0] * (len(probs) + 2), ctl


@pytest.mark.parametrize("precision", PRECS)
def test_set_step_with_pinned_host_buffers(L, precision):
    # the step reads its input from, and writes its output to, page-locked host memory directly: the same
    # bits as the step between device buffers (rejected points included: the fallback reads the host input)
    probs = mixed_probs()
    u0 = [ic_of(p, s) for s, p in enumerate(probs)]
    fs = make_set(L, probs, precision)
    fs.load(u0)
    dev_in = fs.current().clone()
    dev_out = torch.empty_like(dev_in)
    L.lmep_frozen_set_step_once(fs.handle, fs.workspace, dev_in, dev_out)
    host_in = dev_in.cpu().pin_memory()
    host_out = torch.full_like(host_in, float("nan")).pin_memory()
    L.lmep_frozen_set_step_once(fs.handle, fs.workspace, host_in, host_out)
    torch.cuda.synchronize()
    L.lmep_sync_status(fs.handle)
    ref = dev_out.cpu()
    offs = L.frozen_set_offsets([p.N for p in probs])
    for o, p in zip(offs, probs):           # the padding between instances is neither read nor written
        assert same_bits(host_out[o:o + p.N], ref[o:o + p.N])


def test_set_refresh_is_idempotent(L):
    """Recomputing the exp(E) tables on the device gives the same steps."""
    probs = mixed_probs()[:3]
    u0 = [ic_of(p, s) for s, p in enumerate(probs)]
    a = make_set(L, probs, "mixed")
    a.load(u0)
    a.refresh()
    a.step(3)
    b = make_set(L, probs, "mixed")
    b.load(u0)
    b.step(3)
    for x, y in zip(a.states, b.states):
        assert same_bits(x, y)


def test_set_nonfinite_is_reported(L):
    """The as-written viscosity blows up inside a set, too."""
    p = wl.burgers(N=65536, n=7, cfl=4.0, nu=1e-3)      # mu = nu dt / h^2 ~ 130
    fs = make_set(L, [p, wl.burgers(N=1000, n=9, cfl=1.0, nu=1e-6)], "fp64")
    fs.load([wl.burgers_ic(p.N, 0), wl.burgers_ic(1000, 1)])
    with pytest.raises(L.LmepError) as e:
        fs.step(300)
        L.lmep_sync_status(fs.handle)
    assert e.value.status == 3
    L.lmep_sync_status(fs.handle)


def test_set_invalid_descriptors(L):
    h = L.Handle()
    p = wl.burgers(N=257, n=7, cfl=1.0)
    g, o = grid_of(p), op_of(p)
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    bad = [([g], [L.Operator(c2=1e-6)], [p.dt], 0, 0),              # not a frozen operator
           ([g], [o], [0.0], 0, 0),                                # dt <= 0
           ([g], [o], [p.dt], 96, 0),                              # block
           ([g], [o], [p.dt], 0, 3),                               # points per thread
           ([L.Grid(N=257, h=p.h, bc="dirichlet", n=8)], [o], [p.dt], 0, 0)]
    for gs, os_, ts, blk, ppt in bad:
        with pytest.raises(L.LmepError) as e:
            L.lmep_frozen_set_prepare(h, gs, os_, ts, ws, "mixed", blk, ppt)
        assert e.value.status in (1, 5)
    nbytes = L.lmep_frozen_set_workspace_bytes([g], [o], [p.dt], "mixed")
    with pytest.raises(L.LmepError) as e:
        L.lmep_frozen_set_prepare(h, [g], [o], [p.dt], ws[: nbytes - 256], "mixed")
    assert e.value.status == 6
    u = torch.zeros(260, dtype=torch.float32, device="cuda")
    with pytest.raises(L.LmepError) as e:                           # workspace not prepared
        L.lmep_frozen_set_step_once(h, ws, u, torch.empty_like(u))
    assert e.value.status == 1
    L.lmep_frozen_set_prepare(h, [g], [o], [p.dt], ws, "mixed")
    with pytest.raises(L.LmepError) as e:                           # in place
        L.lmep_frozen_set_step_once(h, ws, u, u)
    assert e.value.status == 1
    h.close()
