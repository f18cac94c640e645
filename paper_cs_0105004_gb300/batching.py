"""Many independent scenarios advanced by the same kernel launches.

A batch holds a table of scenarios on the device; every step of the batch is
one link-kernel launch and one node-kernel launch over the tiles of all
members, captured in CUDA graphs, so small networks share the GPU instead of
each paying its own launches.  Each member keeps its own seed, step counter,
target step and statistics, so its results are identical to running it
alone.

The launch shape (occupancy words per warp tile, the link kernel's blocks
per SM, fused or split steps) is chosen by a small autotuner: it times a
short window of the batch for each candidate shape and keeps the fastest.
The shape never changes results, which the autotuner checks.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

from . import transsim as T


@dataclass
class BatchRun:
    seconds: float
    vehicle_updates: int
    steps: int
    tile_words: int
    per_member_updates: List[int] = field(default_factory=list)

    @property
    def updates_per_s(self) -> float:
        return self.vehicle_updates / self.seconds


def make_members(scenarios, tile_words: Optional[int] = None, use_torch_allocator: bool = False):
    return [T.Simulation(sc, use_torch_allocator=use_torch_allocator, tile_words=tile_words) for sc in scenarios]


def _timed(fn, stream):
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / 1000.0


def autotune(scenarios, stream, tile_words: Sequence[int] = (32, 64, 128), grids: Sequence[int] = (0, 4, 2),
             modes: Sequence[int] = (T.STEP_SPLIT, T.STEP_FUSED), window: int = 256):
    """Times `window` batch steps from the empty network for every launch
    shape (occupancy words per warp tile x link-kernel blocks per SM, 0 =
    every resident block x fused or split steps) and returns
    (best, {(tile_words, blocks_per_sm, mode): seconds}).  Every shape must
    give the same totals and digests, which is checked."""
    table, ref = {}, None
    for tw in tile_words:
        sims = make_members(scenarios, tile_words=tw)
        b = T.Batch(len(sims))
        b.add_many(sims, window)
        for grid in grids:
            b.set_link_grid(grid)
            for mode in modes:
                b.set_step_mode(mode)
                b.reset(window, stream)
                b.step(32, stream)  # capture and warm
                b.sync()
                b.reset(window, stream)
                table[(tw, grid, mode)] = _timed(lambda: b.step(window, stream), stream)
                res = [(t["vehicle_updates"], t["last_state_hash"]) for t in (m.totals() for m in sims)]
                if ref is None:
                    ref = res
                elif res != ref:
                    raise RuntimeError(f"launch shape {(tw, grid, mode)} changed the results")
        b.close()
        for m in sims:
            m.close()
    best = min(table, key=table.get)
    return best, table


def apply_shape(batch, shape):
    """Sets a batch's grid and step mode from an autotune() shape (the tile
    words are fixed when its members are made)."""
    _, grid, mode = shape
    batch.set_link_grid(grid)
    batch.set_step_mode(mode)


def run_batched(sims, steps: int, stream, batch: Optional[T.Batch] = None) -> BatchRun:
    """One timed run of all members for `steps` steps from the empty network
    (device-side reset inside the timed region)."""
    own = batch is None
    if own:
        batch = T.Batch(len(sims))
        batch.add_many(sims, steps)
    sec = _timed(lambda: (batch.reset(steps, stream), batch.step(steps, stream)), stream)
    per = [s.totals()["vehicle_updates"] for s in sims]
    if own:
        batch.close()  # releases the members without a table rebuild each
    return BatchRun(sec, sum(per), steps, -1, per)


def run_sequential(sims, steps: int, stream) -> BatchRun:
    """The same members one after another, each with its own launches."""
    import torch
    per = []
    t0 = time.perf_counter()
    total = 0.0
    for s in sims:
        total += _timed(lambda: (s.reset(stream), s.step(steps, stream)), stream)
        per.append(s.totals()["vehicle_updates"])
    torch.cuda.synchronize()
    return BatchRun(total, sum(per), steps, -1, per)
