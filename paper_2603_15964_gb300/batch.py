"""Batched constant-coefficient instances: one persistent launch per step,
replayed from CUDA graphs, with launch shapes picked by an autotuner.

Every instance has its own N_b, h_b and boundary condition (periodic or
Neumann) and shares the stencil width, scheme, nonlinearity, dt and operator.
All compute runs in the library (``lmep_batch_prepare`` harvests every
instance's weights on the device; ``lmep_step_batched_once`` advances the
whole batch by one step in one launch).  This module only owns buffers,
graphs and the tuning cache.
"""
from __future__ import annotations

import json
import os
import time
from dataclasses import dataclass, field

import torch

from . import (Handle, LmepError, Operator, lmep_batch_prepare, lmep_batch_workspace_bytes, lmep_step_batched,
               lmep_step_batched_once, state_dtype)

TILES = (256, 512, 1024, 2048)
BLOCKS = (64, 128, 256)
CTAS = (0,)


def batch_offsets(Ns) -> list:
    """Start of every instance in the batched state: prefix sums of N_b rounded up to 4 (16-byte aligned)."""
    offs = [0]
    for v in Ns:
        offs.append(offs[-1] + (int(v) + 3) // 4 * 4)
    return offs


def pack(arrays, dtype=None) -> "torch.Tensor":
    """Concatenate per-instance host arrays into one batched state (zero padding), on the GPU."""
    import numpy as np
    offs = batch_offsets([len(a) for a in arrays])
    buf = np.zeros(offs[-1], dtype=np.float64)
    for a, o in zip(arrays, offs):
        buf[o:o + len(a)] = a
    return torch.tensor(buf, dtype=dtype or torch.float32, device="cuda")


def unpack(u: torch.Tensor, Ns) -> list:
    """Per-instance views of a batched state (host numpy arrays)."""
    offs = batch_offsets(Ns)
    h = u.detach().cpu().numpy()
    return [h[offs[b]:offs[b] + int(N)] for b, N in enumerate(Ns)]


@dataclass
class LaunchShape:
    tile: int = 0
    block: int = 0
    ctas_per_sm: int = 0


@dataclass
class BatchedProblem:
    Ns: list
    hs: list
    bcs: list
    n: int
    scheme: str
    nonlin: str
    dt: float
    op: Operator
    precision: str = "mixed"
    shape: LaunchShape = field(default_factory=LaunchShape)
    handle: Handle | None = None

    def __post_init__(self):
        self.handle = self.handle or Handle()
        self.offsets = batch_offsets(self.Ns)
        self.total = self.offsets[-1]                 # state length incl. alignment padding
        self.points = int(sum(int(v) for v in self.Ns))
        self._prepare()
        self._graphs = None

    def _prepare(self):
        sh = self.shape
        nbytes = lmep_batch_workspace_bytes(self.Ns, self.hs, self.bcs, self.n, self.scheme, self.nonlin, self.dt,
                                            self.op, self.precision, sh.tile, sh.block, sh.ctas_per_sm)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        lmep_batch_prepare(self.handle, self.Ns, self.hs, self.bcs, self.n, self.scheme, self.nonlin, self.dt,
                           self.op, self.workspace, self.precision, sh.tile, sh.block, sh.ctas_per_sm)

    def empty_state(self) -> torch.Tensor:
        return torch.empty(self.total, dtype=state_dtype(self.precision), device="cuda")

    def step(self, u: torch.Tensor, work: torch.Tensor, nsteps: int = 1) -> None:
        """nsteps steps in place (u holds the result), eager launches."""
        lmep_step_batched(self.handle, self.workspace, u, work, nsteps)

    def capture(self, u: torch.Tensor, work: torch.Tensor) -> None:
        """Capture one graph per direction: A (u -> work) and B (work -> u)."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):                         # warm-up outside the capture
            lmep_step_batched_once(self.handle, self.workspace, u, work)
            lmep_step_batched_once(self.handle, self.workspace, work, u)
        torch.cuda.current_stream().wait_stream(side)
        ga, gb = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(ga, capture_error_mode="relaxed"):
            lmep_step_batched_once(self.handle, self.workspace, u, work)
        with torch.cuda.graph(gb, capture_error_mode="relaxed"):
            lmep_step_batched_once(self.handle, self.workspace, work, u)
        self._graphs = (ga, gb, u.data_ptr(), work.data_ptr())

    def replay(self, nsteps: int) -> None:
        """nsteps graph launches alternating the captured buffers (one launch per step).

        With an odd nsteps the result is in the captured `work` buffer; `current`
        tells which one holds it.
        """
        ga, gb, _, _ = self._graphs
        for t in range(nsteps):
            (ga if t % 2 == 0 else gb).replay()
        self._parity = nsteps % 2

    def current(self, u: torch.Tensor, work: torch.Tensor) -> torch.Tensor:
        return work if getattr(self, "_parity", 0) else u


def _cache_path() -> str:
    return os.environ.get("LMEP_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "lmep", "autotune.json"))


def _key(Ns, n, scheme, nonlin, precision) -> str:
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{props.name}|B={len(Ns)}|sumN={int(sum(int(v) for v in Ns))}|n={n}|{scheme}|{nonlin}|{precision}"


def autotune(Ns, hs, bcs, n, scheme, nonlin, dt, op: Operator, precision: str = "mixed", steps: int = 6,
             candidates=None, use_cache: bool = True, handle: Handle | None = None):
    """Time the launch shapes on this GPU and return (best shape, {shape: ms per step}).

    Each candidate prepares its own workspace and is timed with CUDA events over
    `steps` graph-free launches after one warm-up step.  The winner is cached
    per (GPU, batch shape, scheme, precision) in $LMEP_AUTOTUNE_CACHE.
    """
    key = _key(Ns, n, scheme, nonlin, precision)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return LaunchShape(**cache[key]["shape"]), cache[key]["timings"]
    handle = handle or Handle()
    candidates = candidates or [LaunchShape(t, b, c) for t in TILES for b in BLOCKS for c in CTAS]
    timings = {}
    best, best_ms = None, float("inf")
    u = work = None
    for sh in candidates:
        try:
            prob = BatchedProblem(Ns, hs, bcs, n, scheme, nonlin, dt, op, precision, sh, handle)
        except LmepError:                      # shape does not fit this GPU's shared memory
            continue
        if u is None:
            u = prob.empty_state().uniform_(-0.1, 0.1)
            work = torch.empty_like(u)
        prob.step(u, work, 1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for t in range(steps):
            lmep_step_batched_once(handle, prob.workspace, u if t % 2 == 0 else work, work if t % 2 == 0 else u)
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b) / steps
        timings[f"{sh.tile}/{sh.block}/{sh.ctas_per_sm}"] = ms
        if ms < best_ms:
            best, best_ms = sh, ms
        del prob
    if use_cache:
        cache[key] = {"shape": best.__dict__, "timings": timings, "when": time.time()}
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    return best, timings
