"""Device status reporting: the bounded waits of the streaming apply, through the C ABI.

A warp of the streaming apply waits for the bulk copies of its next tile with a bounded number of
polls.  With the bound set to 0 every such wait gives up at once: the kernel sets the timeout flag,
waits (with the default bound) for the copies it still has in flight, and returns.  No GPU fault and
no hang: lmep_sync_status reports LMEP_ERR_TIMEOUT, and the next steps of the same context are
correct again (against the oracle) once the default bound is restored.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import lmep as olmep

from lmep_testutil import grid_of, op_of, rel_linf, tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIMEOUT = 4


@pytest.fixture(scope="module")
def L():
    import paper_2603_15964_gb300 as L
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return L


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_wait_timeout_is_reported_and_the_context_survives(L, precision):
    from paper_2603_15964_gb300.batch import pack, unpack
    H = L.Handle()
    batch = wl.allen_cahn_batch(B=16, Nmin=600, Nmax=3000, n=9, scheme="etdrk2", steps=1, seed=9)
    B = len(batch.Ns)
    hs = [batch.problem(b).h for b in range(B)]
    op = op_of(batch.problem(0))
    kw = dict(tile=128, block=64, ctas_per_sm=1)
    nbytes = L.lmep_batch_workspace_bytes(batch.Ns, hs, batch.bcs, 9, "etdrk2", "allen_cahn", batch.dt, op,
                                          precision, **kw)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    L.lmep_batch_prepare(H, batch.Ns, hs, batch.bcs, 9, "etdrk2", "allen_cahn", batch.dt, op, ws, precision, **kw)
    dt_ = L.state_dtype(precision)
    u0s = [wl.allen_cahn_ic(int(batch.Ns[b]), b) for b in range(B)]
    if precision == "mixed":
        u0s = [x.astype(np.float32).astype(np.float64) for x in u0s]
    u = pack(u0s, dt_)
    out = torch.empty_like(u)
    L.lmep_set_wait_limit(H, 0)
    try:
        L.lmep_step_batched_once(H, ws, u, out)
        with pytest.raises(L.LmepError) as e:
            L.lmep_sync_status(H)
        assert e.value.status == TIMEOUT
    finally:
        L.lmep_set_wait_limit(H, -1)
    L.lmep_sync_status(H)                       # the flag was cleared; nothing else pending
    L.lmep_step_batched_once(H, ws, u, out)     # the same context, default bound
    L.lmep_sync_status(H)
    got = unpack(out, batch.Ns)
    for b in range(B):
        want = olmep.run(batch.problem(b), u0s[b], 1)
        assert rel_linf(got[b], want) <= tol(precision), b
    H.close()


def test_single_instance_wait_timeout_is_reported(L):
    H = L.Handle()
    p = wl.allen_cahn(20000, n=9, scheme="etdrk2", steps=1)
    W = torch.empty(p.n, 3, p.n, dtype=torch.float32, device="cuda")
    L.lmep_harvest_weights(H, grid_of(p), op_of(p), p.dt, 2, None, W, "mixed")
    u0 = wl.allen_cahn_ic(p.N, 3).astype(np.float32).astype(np.float64)
    u = torch.tensor(u0, dtype=torch.float32, device="cuda")
    work = torch.empty_like(u)
    L.lmep_set_wait_limit(H, 0)
    try:
        L.lmep_step(H, grid_of(p), op_of(p), "etdrk2", "allen_cahn", p.dt, W, u.clone(), work, 1, "mixed")
        with pytest.raises(L.LmepError) as e:
            L.lmep_sync_status(H)
        assert e.value.status == TIMEOUT
    finally:
        L.lmep_set_wait_limit(H, -1)
    L.lmep_step(H, grid_of(p), op_of(p), "etdrk2", "allen_cahn", p.dt, W, u, work, 1, "mixed")
    L.lmep_sync_status(H)
    assert rel_linf(u.cpu().numpy(), olmep.run(p, u0, 1)) <= tol("mixed")
    H.close()


def test_wait_limit_arguments(L):
    H = L.Handle()
    with pytest.raises(L.LmepError) as e:
        L.lmep_set_wait_limit(H, 1 << 31)
    assert e.value.status == 1
    L.lmep_set_wait_limit(H, 1000)
    L.lmep_set_wait_limit(H, -1)
    H.close()
