"""A set of frozen-velocity instances advanced together.

Each instance (its own grid, operator, dt and stencil width) rebuilds and exponentiates every
point's local operator at every step and applies the harvested row (Sec. 2.1 steps 1-6).

* ``fused=True`` (default): the whole set is one library workspace (``lmep_frozen_set_*``): one
  persistent launch per step covers every instance, whatever its width, plus a launch that finishes
  the rare points the first one hands over; the state lives in two packed buffers (instance b at
  ``frozen_set_offsets(Ns)[b]``) that the steps alternate, so a step copies nothing.
* ``fused=False``: one ``lmep_step`` call per instance (each a launch and a copy back into the
  state), the form used before the set existed; kept for comparison.

``capture`` records one step per direction of the ping-pong into CUDA graphs (or, unfused, one
step of every instance into one graph), so that a step is one host call.  ``tune`` picks the launch
shape of the fused step on this GPU.  All compute runs in the library; this module owns buffers,
graphs and the tuning cache.
"""
from __future__ import annotations

import json
import os
import time
from dataclasses import dataclass, field

import torch

from . import (Grid, Handle, LmepError, Operator, frozen_set_offsets, lmep_frozen_set_prepare,  # noqa: F401
               lmep_frozen_set_refresh, lmep_frozen_set_step_once, lmep_frozen_set_workspace_bytes,
               lmep_set_expm_method, lmep_step, state_dtype)

SHAPES = [(64, 1), (64, 2), (128, 1), (128, 2), (256, 1), (256, 2), (512, 1), (64, 4), (128, 4), (256, 4), (64, 8),
          (128, 8)]


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
    fused: bool = True
    block: int = 0
    points_per_thread: int = 0
    states: list = field(default_factory=list)

    def __post_init__(self):
        self.handle = self.handle or Handle()
        self._work = []
        self._graph = None
        self._graphs = None
        self._cur = 0
        self.Ns = [inst.grid.N for inst in self.instances]
        self.offsets = frozen_set_offsets(self.Ns)
        if self.fused:
            self._prepare()

    # ------------------------------------------------------------------ fused workspace
    def _prepare(self):
        lmep_set_expm_method(self.handle, self.method)        # the route is fixed at prepare time
        g = [i.grid for i in self.instances]
        o = [i.op for i in self.instances]
        t = [i.dt for i in self.instances]
        nbytes = lmep_frozen_set_workspace_bytes(g, o, t, self.precision, self.block, self.points_per_thread)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        lmep_frozen_set_prepare(self.handle, g, o, t, self.workspace, self.precision, self.block,
                                self.points_per_thread)

    def refresh(self) -> None:
        """Recompute every instance's exp(E) table on the device (the set's setup work)."""
        lmep_frozen_set_refresh(self.handle, self.workspace)

    def _views(self, buf):
        return [buf[o:o + n] for o, n in zip(self.offsets, self.Ns)]

    @property
    def buffers(self):
        return self._bufs

    def current(self) -> torch.Tensor:
        """The packed buffer that holds the state (fused mode)."""
        return self._bufs[self._cur]

    # ------------------------------------------------------------------ both modes
    def load(self, arrays) -> None:
        """Device states from host arrays (one per instance); drops captured graphs."""
        dt = state_dtype(self.precision)
        if self.fused:
            import numpy as np
            buf = np.zeros(self.offsets[-1], dtype=np.float64)
            for a, o in zip(arrays, self.offsets):
                buf[o:o + len(a)] = a
            u = torch.tensor(buf, dtype=dt, device="cuda")
            self._bufs = (u, torch.zeros_like(u))
            self._cur = 0
            self.states = self._views(u)
        else:
            self.states = [torch.as_tensor(a, dtype=dt).to("cuda") for a in arrays]
            self._work = [torch.empty_like(u) for u in self.states]
        self._graph = None
        self._graphs = None

    def _step_once(self, src: int) -> None:
        lmep_frozen_set_step_once(self.handle, self.workspace, self._bufs[src], self._bufs[1 - src])

    def step(self, nsteps: int = 1) -> None:
        """nsteps eager steps of every instance."""
        if self.fused:
            for _ in range(nsteps):
                self._step_once(self._cur)
                self._cur ^= 1
            self.states = self._views(self._bufs[self._cur])
            return
        lmep_set_expm_method(self.handle, self.method)      # the handle may be shared
        for inst, u, w in zip(self.instances, self.states, self._work):
            lmep_step(self.handle, inst.grid, inst.op, "linear", "none", inst.dt, None, u, w, nsteps,
                      self.precision)

    def capture(self, nsteps: int = 1) -> None:
        """Fused: record one step per ping-pong direction into two CUDA graphs (after one eager step
        in each direction on a side stream, which leaves the state where it was -- two steps
        further).  Unfused: record nsteps steps of every instance into one graph (after nsteps
        eager warm-up steps, which advance the states)."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        if self.fused:
            with torch.cuda.stream(side):
                self.step(2)
            torch.cuda.current_stream().wait_stream(side)
            graphs = []
            for src in (0, 1):
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, capture_error_mode="relaxed"):
                    self._step_once(src)
                graphs.append(g)
            self._graphs = graphs
            return
        with torch.cuda.stream(side):
            self.step(nsteps)
        torch.cuda.current_stream().wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="relaxed"):
            self.step(nsteps)
        self._graph = g

    def replay(self, nsteps: int = 1) -> None:
        """nsteps graph launches on the current stream (fused: one step each, alternating the
        buffers; unfused: the captured number of steps each)."""
        if self.fused:
            if self._graphs is None:
                raise RuntimeError("FrozenSet.replay needs capture() first")
            for _ in range(nsteps):
                self._graphs[self._cur].replay()
                self._cur ^= 1
            self.states = self._views(self._bufs[self._cur])
            return
        if self._graph is None:
            raise RuntimeError("FrozenSet.replay needs capture() first")
        for _ in range(nsteps):
            self._graph.replay()


def _cache_path() -> str:
    return os.environ.get("LMEP_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "lmep", "autotune.json"))


def tune(instances, arrays, precision: str = "mixed", method: str = "auto", steps: int = 10,
         shapes=None, use_cache: bool = True, handle: Handle | None = None, cold: bool = False):
    """Time the fused step's launch shapes (threads per CTA, points per thread) on this GPU and return
    ((block, points_per_thread), {shape: ms per step}).  Each shape prepares its own workspace and is
    timed with CUDA events after two warm-up steps: over `steps` eager steps back to back, or with
    cold=True as the mean of `steps` lone steps, each after a 256 MiB write that evicts the L2 (a
    step of a caller that does other work between steps).  The winner is cached per (GPU, instance
    widths and sizes, precision, route, timing) in $LMEP_AUTOTUNE_CACHE."""
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    key = (f"{props.name}|frozen_set|" + ",".join(f"{i.grid.n}:{i.grid.N}" for i in instances) +
           f"|{precision}|{method}" + ("|cold" if cold else ""))
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return tuple(cache[key]["shape"]), cache[key]["timings"]
    handle = handle or Handle()
    timings = {}
    best, best_ms = None, float("inf")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda") if cold else None
    for block, ppt in shapes or SHAPES:
        fs = FrozenSet(instances, precision, method, handle, True, block, ppt)
        fs.load(arrays)
        fs.step(2)
        if cold:
            lone = []
            for _ in range(steps):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                fs.step(1)
                b.record()
                b.synchronize()
                lone.append(a.elapsed_time(b))
            ms = sum(lone) / len(lone)  # the mean: event times come in steps of about 1 us
        else:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fs.step(steps)
            b.record()
            b.synchronize()
            ms = a.elapsed_time(b) / steps
        timings[f"{block}/{ppt}"] = ms
        if ms < best_ms:
            best, best_ms = (block, ppt), ms
        del fs
    if use_cache:
        cache[key] = {"shape": list(best), "timings": timings, "when": time.time()}
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    return best, timings
