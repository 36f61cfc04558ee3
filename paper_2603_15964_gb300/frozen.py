"""A set of frozen-velocity instances advanced together, one step per CUDA graph replay.

Each instance (its own grid, operator, dt and stencil width) advances by ``lmep_step`` with a
NULL weight array: the library rebuilds and exponentiates every point's local operator and
applies the row in one launch (Sec. 2.1 steps 1-6), then copies the result back into the state.
With launches of a few tens of microseconds the host's submission of one call per instance is
slower than the GPU; ``capture`` records one step of every instance into a CUDA graph so that a
step is one host call.  All compute runs in the library; this module owns buffers and graphs.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from . import Grid, Handle, Operator, lmep_set_expm_method, lmep_step, state_dtype  # noqa: F401


@dataclass
class FrozenInstance:
    grid: Grid
    op: Operator
    dt: float


@dataclass
class FrozenSet:
    instances: list
    precision: str = "mixed"
    method: str = "auto"
    handle: Handle | None = None
    states: list = field(default_factory=list)

    def __post_init__(self):
        self.handle = self.handle or Handle()
        lmep_set_expm_method(self.handle, self.method)
        self._work = []
        self._graph = None

    def load(self, arrays) -> None:
        """Device states from host arrays (one per instance); drops a captured graph."""
        dt = state_dtype(self.precision)
        self.states = [torch.as_tensor(a, dtype=dt).to("cuda") for a in arrays]
        self._work = [torch.empty_like(u) for u in self.states]
        self._graph = None

    def step(self, nsteps: int = 1) -> None:
        """nsteps eager steps of every instance (one library call per instance)."""
        lmep_set_expm_method(self.handle, self.method)      # the handle may be shared
        for inst, u, w in zip(self.instances, self.states, self._work):
            lmep_step(self.handle, inst.grid, inst.op, "linear", "none", inst.dt, None, u, w, nsteps,
                      self.precision)

    def capture(self, nsteps: int = 1) -> None:
        """Record nsteps steps of every instance into a CUDA graph (after nsteps eager warm-up steps
        on a side stream, which advance the states).  An even nsteps leaves the result in the state
        buffer without the copy-back of an odd count."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.step(nsteps)
        torch.cuda.current_stream().wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="relaxed"):
            self.step(nsteps)
        self._graph = g

    def replay(self, nsteps: int = 1) -> None:
        """nsteps graph launches (each the captured number of steps) on the current stream."""
        if self._graph is None:
            raise RuntimeError("FrozenSet.replay needs capture() first")
        for _ in range(nsteps):
            self._graph.replay()
