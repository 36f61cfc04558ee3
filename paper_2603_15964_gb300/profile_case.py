"""Small profiling cases.

`python -m paper_2603_15964_gb300.profile_case [n cfl]`: warm-up, then one
fused frozen-velocity Burgers step (N = 65536, n = 13, CFL = 4, nu = 1e-6,
departure-centred) in the FP32 form and one in FP64.  Used with
`ncu -k regex:k_warp -s 4 -c 2` (the two launches after four warm-up launches).

`python -m paper_2603_15964_gb300.profile_case adj [auto|pade]`: one reverse
step of the frozen-velocity Burgers adjoint (N = 262144, one instance, n = 9,
CFL = 2, FP32 state, FP64 derivatives: closed form of the factorised rows
with "auto", Pade Frechet derivatives with "pade") after one warm-up step.
Used with `ncu -k regex:k_adjoint_fact -s 1 -c 1` ("auto") or
`ncu -k regex:k_adjoint_points -s 1 -c 1` ("pade").

`python -m paper_2603_15964_gb300.profile_case ac [tile block]`: the batched
Allen-Cahn ETDRK2 step (4096 instances, N log-uniform in [1024, 65536],
n = 9, FP32 state, 254 MB): three warm-up steps, then one step.  Used with
`ncu -k regex:k_apply -s 3 -c 1`.
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main(n: int = 13, cfl: float = 4.0) -> None:
    import torch

    import paper_2603_15964_gb300 as L
    import workloads as wl

    p = wl.burgers(N=65536, n=n, cfl=cfl, nu=1e-6)
    g = L.Grid(N=p.N, h=p.h, bc=p.bc, n=p.n, departure_centring=True)
    op = L.Operator(c2=p.c2, frozen_adv=1.0)
    h = L.Handle()
    bufs = {}
    for prec in ("mixed", "fp64"):
        u = torch.tensor(wl.burgers_ic(p.N, 0), dtype=L.state_dtype(prec), device="cuda")
        bufs[prec] = (u, torch.empty_like(u))
    for prec in ("mixed", "fp64"):                        # 4 warm-up launches
        L.lmep_step(h, g, op, "linear", "none", p.dt, None, *bufs[prec], 2, prec)
    for prec in ("mixed", "fp64"):                        # the two profiled launches
        L.lmep_step(h, g, op, "linear", "none", p.dt, None, *bufs[prec], 1, prec)
    L.lmep_sync_status(h)
    torch.cuda.synchronize()
    print("profile case ok")


def allen_cahn(tile: int = 1024, block: int = 128) -> None:
    import torch

    import paper_2603_15964_gb300 as L
    import workloads as wl
    from paper_2603_15964_gb300.batch import BatchedProblem, LaunchShape

    batch = wl.allen_cahn_batch()
    hs = [batch.problem(b).h for b in range(len(batch.Ns))]
    prob = BatchedProblem(list(batch.Ns), hs, batch.bcs, batch.n, batch.scheme, "allen_cahn", batch.dt,
                          L.Operator(c2=batch.eps2), "mixed", LaunchShape(tile, block, 0))
    u = prob.empty_state().uniform_(-0.1, 0.1)
    w = torch.empty_like(u)
    for t in range(4):                                    # three warm-up steps, then the profiled one
        L.lmep_step_batched_once(prob.handle, prob.workspace, u if t % 2 == 0 else w, w if t % 2 == 0 else u)
    L.lmep_sync_status(prob.handle)
    torch.cuda.synchronize()
    print("profile case ok")


def adjoint(method: str = "auto") -> None:
    import torch

    import paper_2603_15964_gb300 as L
    import workloads as wl

    p = wl.burgers(N=262144, n=9, cfl=2.0, nu=1e-6, steps=1)
    g = L.Grid(N=p.N, h=p.h, bc=p.bc, n=p.n, departure_centring=True)
    op = L.Operator(c2=p.c2, frozen_adv=1.0)
    h = L.Handle()
    L.lmep_set_expm_method(h, method)
    u = torch.tensor(wl.burgers_ic(p.N, 0), dtype=torch.float32, device="cuda")
    lam_next = torch.ones_like(u)
    lam = torch.empty_like(u)
    dnu = torch.zeros(1, dtype=torch.float64, device="cuda")
    scratch = torch.empty(L.lmep_adjoint_scratch_bytes(g, "mixed"), dtype=torch.uint8, device="cuda")
    for _ in range(2):                                    # one warm-up step, then the profiled one
        L.lmep_adjoint_step(h, g, op, p.dt, u, lam_next, lam, dnu, scratch, "mixed")
    L.lmep_sync_status(h)
    torch.cuda.synchronize()
    print("profile case ok")


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "adj":
        adjoint(*sys.argv[2:3])
    elif len(sys.argv) > 1 and sys.argv[1] == "ac":
        allen_cahn(*(int(a) for a in sys.argv[2:]))
    else:
        main(*(float(a) if i else int(a) for i, a in enumerate(sys.argv[1:])))
