"""Differentiable frozen-velocity LMEP solves with step checkpointing.

``FrozenVelocitySolver(...)(u0, nu)`` advances a batch of initial states by
`steps` frozen-velocity LMEP steps (every point rebuilds and exponentiates its
local operator -u_i D1 + nu D2 each step) and returns the final states; it is
differentiable with respect to u0 and nu through a torch.autograd.Function
whose backward pass runs the library's hand-written adjoint kernel
(``lmep_adjoint_step``: transposed banded apply plus the Frechet derivative
of each local exponential).  The forward pass keeps one checkpoint every
`checkpoint_every` steps; the backward pass recomputes the states of one
segment at a time from its checkpoint and walks it in reverse, so memory is
O(steps / K + K) states instead of O(steps).  dJ/dnu is accumulated in FP64
on the device.  The paper has no adjoint; this is the derivative of the
discrete forward step.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import (Grid, Handle, Operator, lmep_adjoint_scratch_bytes, lmep_adjoint_step, lmep_frozen_set_prepare,
               lmep_frozen_set_step_once, lmep_frozen_set_workspace_bytes, lmep_step, state_dtype)


@dataclass
class FrozenVelocitySolver:
    N: int
    h: float
    n: int
    dt: float
    steps: int
    bc: str = "dirichlet"
    departure_centring: bool = True
    frozen_adv: float = 1.0
    precision: str = "mixed"
    checkpoint_every: int = 64
    bc_lo: float = 0.0
    bc_hi: float = 0.0
    handle: Handle | None = None
    # step a batch as a frozen set (one persistent launch per step over all states; the same bits as
    # lmep_step on the batched grid), prepared at first use for each (batch, nu) with the handle's expm
    # route at that time; needs N % 4 == 0 (the set's packed layout is then the (batch, N) tensor)
    use_set: bool = True

    def __post_init__(self):
        self.handle = self.handle or Handle()
        self._sets = {}

    def grid(self, batch: int) -> Grid:
        return Grid(N=self.N, h=self.h, bc=self.bc, n=self.n, departure_centring=self.departure_centring,
                    bc_lo=self.bc_lo, bc_hi=self.bc_hi, batch=batch)

    def op(self, nu: float) -> Operator:
        return Operator(c2=nu, frozen_adv=self.frozen_adv)

    def _set_workspace(self, batch: int, nu: float) -> torch.Tensor:
        key = (batch, nu)
        if key not in self._sets:
            if len(self._sets) >= 4:
                self._sets.pop(next(iter(self._sets)))
            g = [self.grid(1)] * batch
            o = [self.op(nu)] * batch
            t = [self.dt] * batch
            ws = torch.empty(lmep_frozen_set_workspace_bytes(g, o, t, self.precision), dtype=torch.uint8,
                             device="cuda")
            lmep_frozen_set_prepare(self.handle, g, o, t, ws, self.precision)
            self._sets[key] = ws
        return self._sets[key]

    def advance(self, u: torch.Tensor, work: torch.Tensor, nu: float, nsteps: int) -> None:
        """nsteps forward steps of the whole batch in place (no autograd)."""
        if nsteps <= 0:
            return
        if not (self.use_set and self.N % 4 == 0 and self.frozen_adv != 0.0):
            lmep_step(self.handle, self.grid(u.shape[0]), self.op(nu), "linear", "none", self.dt, None, u, work,
                      nsteps, self.precision)
            return
        ws = self._set_workspace(u.shape[0], nu)
        src, dst = u, work
        for _ in range(nsteps):
            lmep_frozen_set_step_once(self.handle, ws, src, dst)
            src, dst = dst, src
        if src is not u:
            u.copy_(src)

    def step_into(self, src: torch.Tensor, dst: torch.Tensor, work: torch.Tensor, nu: float) -> None:
        """One forward step of the whole batch from src into dst (src unchanged)."""
        if self.use_set and self.N % 4 == 0 and self.frozen_adv != 0.0:
            lmep_frozen_set_step_once(self.handle, self._set_workspace(src.shape[0], nu), src, dst)
        else:
            dst.copy_(src)
            self.advance(dst, work, nu, 1)

    def __call__(self, u0: torch.Tensor, nu: torch.Tensor) -> torch.Tensor:
        return FrozenVelocitySolve.apply(u0, nu, self)


class FrozenVelocitySolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, nu, solver: FrozenVelocitySolver):
        dt_ = state_dtype(solver.precision)
        if u0.dim() != 2 or u0.shape[1] != solver.N or u0.dtype != dt_ or not u0.is_cuda:
            raise ValueError(f"u0 must be a CUDA tensor of shape (batch, {solver.N}) and dtype {dt_}")
        nu_v = float(nu)
        u = u0.detach().clone().contiguous()
        work = torch.empty_like(u)
        K = max(1, int(solver.checkpoint_every))
        checkpoints = [u.clone()]
        done = 0
        while done < solver.steps:
            k = min(K, solver.steps - done)
            solver.advance(u, work, nu_v, k)
            done += k
            if done < solver.steps:
                checkpoints.append(u.clone())
        ctx.solver = solver
        ctx.nu_v = nu_v
        ctx.nu_meta = (nu.dtype, nu.device) if torch.is_tensor(nu) else (torch.float64, u.device)
        ctx.checkpoints = checkpoints
        return u

    @staticmethod
    def backward(ctx, grad_uT):
        solver: FrozenVelocitySolver = ctx.solver
        nu_v = ctx.nu_v
        B = grad_uT.shape[0]
        grid = solver.grid(B)
        op = solver.op(nu_v)
        dt_ = state_dtype(solver.precision)
        lam = grad_uT.detach().to(dt_).contiguous().clone()
        lam_new = torch.empty_like(lam)
        dnu = torch.zeros(1, dtype=torch.float64, device=lam.device)
        scratch = torch.empty(lmep_adjoint_scratch_bytes(grid, solver.precision), dtype=torch.uint8,
                              device=lam.device)
        K = max(1, int(solver.checkpoint_every))
        work = torch.empty_like(lam)
        for seg in range(len(ctx.checkpoints) - 1, -1, -1):
            length = min(K, solver.steps - seg * K)
            states = [ctx.checkpoints[seg]]
            for _ in range(length - 1):
                nxt = torch.empty_like(states[-1])
                solver.step_into(states[-1], nxt, work, nu_v)
                states.append(nxt)
            for t in range(length - 1, -1, -1):
                lmep_adjoint_step(solver.handle, grid, op, solver.dt, states[t], lam, lam_new, dnu, scratch,
                                  solver.precision)
                lam, lam_new = lam_new, lam
        nu_dtype, nu_device = ctx.nu_meta
        grad_nu = dnu.reshape(()).to(dtype=nu_dtype, device=nu_device)
        return lam, grad_nu, None
