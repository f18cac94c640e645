"""Relaxation iterations around the micro-simulation (Sec. 1).

Plans depend on congestion and congestion on plans; the paper resolves this
by systematic relaxation: run the micro-simulation on the current plans,
re-plan a fraction of the travellers (never more than about 10 %) on what
the run showed, run again, and repeat until plans and traffic are
consistent, which takes tens of full runs.  Here the micro-simulation runs
on the GPU; the run's per-link travel times (ts_read_link_times) become the
link costs of the re-planning, done on the host with the same shortest-path
builder that made the initial routes.

Readings (the paper gives no cost function or selection rule):
  * link cost = the mean travel time of the traversals of that link the run
    completed, in steps, rounded half up; a link nobody completed costs its
    free-flow time ceil(cells / vmax); every cost is at least 1;
  * each iteration re-plans round(fraction * n) travellers drawn uniformly
    without replacement by a seeded generator; a re-planned traveller keeps
    its origin node, destination node and departure step and takes the
    shortest route under the link costs (ties to the smaller predecessor
    node id, as for the initial routes).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, replace
from typing import Callable, List, Optional, Tuple

import numpy as np

from . import transsim as T
from .inputs import networks as N


@dataclass
class RunResult:
    seconds: float              # device time of the run (CUDA events) or wall time
    vehicle_updates: int
    arrived: int
    state_hash: int
    link_time_sum: np.ndarray   # uint64 [n_links]
    link_time_count: np.ndarray  # uint64 [n_links]

    @property
    def mean_link_time(self) -> float:
        c = int(self.link_time_count.sum())
        return float(self.link_time_sum.sum()) / c if c else 0.0


@dataclass
class Iteration:
    index: int
    run: RunResult
    plan_seconds: float   # host time to re-plan after this run (0 after the last)
    replanned: int        # travellers re-planned after this run


def link_costs(net: N.Network, vmax: int, tsum: np.ndarray, tcnt: np.ndarray) -> np.ndarray:
    """Integer link costs in steps from one run's travel times (see the module
    docstring)."""
    tsum = np.asarray(tsum, np.uint64).astype(np.int64)
    tcnt = np.asarray(tcnt, np.uint64).astype(np.int64)
    cells = np.asarray(net.link_cells, np.int64)
    free = (cells + vmax - 1) // vmax
    mean = (2 * tsum + tcnt) // (2 * np.maximum(tcnt, 1))
    cost = np.where(tcnt > 0, mean, free)
    return np.maximum(cost, 1).astype(np.uint32)


def replan(net: N.Network, demand: N.Demand, costs: np.ndarray, fraction: float,
           rng: np.random.Generator, threads: Optional[int] = None) -> Tuple[N.Demand, np.ndarray]:
    """New plans: round(fraction * n) travellers drawn by rng get the shortest
    route under costs between their origin and destination nodes.  Returns
    the new demand and the sorted indices of the re-planned travellers."""
    n = demand.n
    k = int(round(fraction * n))
    chosen = np.sort(rng.choice(n, size=k, replace=False)) if k else np.zeros(0, np.int64)
    off = np.asarray(demand.route_offsets, np.int64)
    links = np.asarray(demand.route_links, np.uint32)
    if k == 0:
        return demand, chosen
    first = links[off[chosen]]
    last = links[off[chosen + 1] - 1]
    orig = np.asarray(net.link_from, np.uint32)[first]
    dest = np.asarray(net.link_to, np.uint32)[last]
    new_off, new_links = N.build_routes(net, orig, dest, threads=threads, weights=costs)
    new_off = new_off.astype(np.int64)
    lengths = np.diff(off)
    lengths[chosen] = np.diff(new_off)
    out_off = np.zeros(n + 1, np.int64)
    np.cumsum(lengths, out=out_off[1:])
    total = int(out_off[-1])
    if total >= 2 ** 32:
        raise ValueError("route table exceeds 32-bit offsets")
    # every output entry takes the same position of its traveller's old or new route
    trip = np.repeat(np.arange(n), lengths)
    pos = np.arange(total, dtype=np.int64) - out_off[trip]
    rank = np.full(n, -1, np.int64)
    rank[chosen] = np.arange(k)
    r = rank[trip]
    out = np.empty(total, np.uint32)
    old = r < 0
    out[old] = links[off[trip[old]] + pos[old]]
    out[~old] = new_links[new_off[r[~old]] + pos[~old]]
    return N.Demand(demand.depart_step, out_off.astype(np.uint32), out), chosen


def gpu_run(sc: N.Scenario, stream=None) -> RunResult:
    """One full run of the scenario on the GPU (the library, no fallback)."""
    import torch
    sim = T.Simulation(sc)
    s = stream if stream is not None else torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(s)
    sim.step(sc.steps, s)
    b.record(s)
    b.synchronize()
    tot = sim.totals()
    tsum, tcnt = sim.link_times()
    sim.close()
    return RunResult(a.elapsed_time(b) / 1000.0, int(tot["vehicle_updates"]), int(tot["arrived"]),
                     int(tot["last_state_hash"]), tsum, tcnt)


def relax(scenario: N.Scenario, iterations: int, fraction: float = 0.1, seed: int = 0,
          run: Optional[Callable[[N.Scenario], RunResult]] = None,
          threads: Optional[int] = None) -> Tuple[N.Scenario, List[Iteration]]:
    """`iterations` runs with re-planning between them.  run(scenario) runs
    one full simulation (default: gpu_run).  Returns the scenario with the
    last plans and the per-iteration results."""
    run = run or gpu_run
    rng = np.random.default_rng(seed)
    sc = scenario
    out: List[Iteration] = []
    for it in range(iterations):
        r = run(sc)
        t0 = time.perf_counter()
        k = 0
        if it + 1 < iterations:
            costs = link_costs(sc.net, sc.vmax, r.link_time_sum, r.link_time_count)
            demand, chosen = replan(sc.net, sc.demand, costs, fraction, rng, threads)
            sc = replace(sc, demand=demand, init=None)
            k = int(chosen.size)
        out.append(Iteration(it, r, time.perf_counter() - t0 if k else 0.0, k))
    return sc, out
