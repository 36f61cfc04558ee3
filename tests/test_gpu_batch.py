"""Batched persistent launch: CUDA-graph replay, ping-pong entry point, autotuner.

Graph replay and eager stepping run the same kernel on the same data, so
their results must be identical; against the oracle the usual trajectory
tolerance holds (K steps: K x 1e-12 FP64, K x 1e-5 FP32 form).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import lmep as olmep

from lmep_testutil import rel_linf, tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import paper_2603_15964_gb300 as L
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return L


def small_batch(seed=7, B=12):
    return wl.allen_cahn_batch(B=B, Nmin=80, Nmax=5000, n=9, scheme="etdrk2", steps=5, seed=seed)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_matches_eager_and_oracle(L, precision):
    from paper_2603_15964_gb300.batch import BatchedProblem, LaunchShape
    batch = small_batch()
    hs = [batch.problem(b).h for b in range(len(batch.Ns))]
    op = L.Operator(c2=batch.eps2)
    prob = BatchedProblem(list(batch.Ns), hs, batch.bcs, batch.n, "etdrk2", "allen_cahn", batch.dt, op, precision,
                          LaunchShape(tile=1024, block=256))
    from paper_2603_15964_gb300.batch import pack, unpack
    u0s = [wl.allen_cahn_ic(int(N), b) for b, N in enumerate(batch.Ns)]
    if precision == "mixed":
        u0s = [x.astype(np.float32).astype(np.float64) for x in u0s]
    dt_ = L.state_dtype(precision)
    ue = pack(u0s, dt_)
    we = torch.empty_like(ue)
    prob.step(ue, we, batch.steps)                      # eager, result in ue
    ug = pack(u0s, dt_)
    wg = torch.empty_like(ug)
    prob.capture(ug, wg)                                # capture warms up with 2 steps: restart
    ug.copy_(pack(u0s, dt_))
    prob.replay(batch.steps)
    torch.cuda.synchronize()
    L.lmep_sync_status(prob.handle)
    got = unpack(prob.current(ug, wg), batch.Ns)
    eager = unpack(ue, batch.Ns)
    for b in range(len(batch.Ns)):
        assert np.array_equal(got[b], eager[b])
    for b in (0, 3, len(batch.Ns) - 1):
        want = olmep.run(batch.problem(b), u0s[b], batch.steps)
        assert rel_linf(got[b], want) <= tol(precision) * batch.steps


def test_step_batched_once_rejects_aliasing(L):
    from paper_2603_15964_gb300.batch import BatchedProblem
    batch = small_batch(B=3)
    hs = [batch.problem(b).h for b in range(3)]
    prob = BatchedProblem(list(batch.Ns), hs, batch.bcs, 9, "etdrk2", "allen_cahn", batch.dt,
                          L.Operator(c2=batch.eps2), "mixed")
    u = prob.empty_state()
    with pytest.raises(L.LmepError):
        L.lmep_step_batched_once(prob.handle, prob.workspace, u, u)


def test_autotune_picks_a_candidate(L, tmp_path, monkeypatch):
    from paper_2603_15964_gb300.batch import LaunchShape, autotune
    monkeypatch.setenv("LMEP_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    batch = small_batch(B=40)
    hs = [batch.problem(b).h for b in range(40)]
    cands = [LaunchShape(512, 256, 0), LaunchShape(1024, 128, 0), LaunchShape(256, 64, 2)]
    best, timings = autotune(batch.Ns, hs, batch.bcs, 9, "etdrk2", "allen_cahn", batch.dt,
                             L.Operator(c2=batch.eps2), "mixed", candidates=cands)
    assert best in cands and len(timings) == 3 and all(v > 0 for v in timings.values())
    again, t2 = autotune(batch.Ns, hs, batch.bcs, 9, "etdrk2", "allen_cahn", batch.dt,
                         L.Operator(c2=batch.eps2), "mixed", candidates=cands)
    assert again == best and t2 == timings                       # served from the cache


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_launch_shapes_agree_bit_for_bit(L, precision):
    """Every output is the same sequence of operations whatever the tile size,
    block size or pipeline depth, so all launch shapes give identical states."""
    from paper_2603_15964_gb300.batch import BatchedProblem, LaunchShape, pack, unpack
    batch = wl.allen_cahn_batch(B=9, Nmin=60, Nmax=9000, n=9, scheme="etdrk2", steps=3, seed=11)
    hs = [batch.problem(b).h for b in range(len(batch.Ns))]
    u0s = [wl.allen_cahn_ic(int(N), 50 + b) for b, N in enumerate(batch.Ns)]
    results = []
    for tile, block in ((256, 64), (512, 128), (1024, 256), (2048, 128), (128, 512)):
        prob = BatchedProblem(list(batch.Ns), hs, batch.bcs, batch.n, "etdrk2", "allen_cahn", batch.dt,
                              L.Operator(c2=batch.eps2), precision, LaunchShape(tile, block))
        u = pack(u0s, L.state_dtype(precision))
        prob.step(u, torch.empty_like(u), batch.steps)
        L.lmep_sync_status(prob.handle)
        results.append(unpack(u, batch.Ns))
    for r in results[1:]:
        for b in range(len(batch.Ns)):
            assert np.array_equal(r[b], results[0][b])
    for b in (0, len(batch.Ns) - 1):
        want = olmep.run(batch.problem(b), u0s[b] if precision == "fp64" else
                         u0s[b].astype(np.float32).astype(np.float64), batch.steps)
        assert rel_linf(results[0][b], want) <= tol(precision) * batch.steps
