"""Small profiling case: warm-up, then one fused frozen-velocity Burgers step
(N = 65536, n = 13, CFL = 4, nu = 1e-6, departure-centred) in the FP32 form
and one in FP64.  Used with `ncu -k regex:k_warp -s 4 -c 2` (the two launches
after four warm-up launches)."""
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


if __name__ == "__main__":
    main(*(float(a) if i else int(a) for i, a in enumerate(sys.argv[1:])))
