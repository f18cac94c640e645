"""Continuous-batching job server for simulation jobs.

Requests arrive as a Poisson stream.  A job's inputs are built on a worker
thread when it arrives; it is admitted to the running batch as soon as its
device footprint fits the memory budget; every batch step advances all
admitted jobs by a chunk of time steps, each towards its own target; a job
that reaches its target leaves the batch, its totals are read and its memory
returns to the pool.  State stays on the device between steps, and jobs that
arrive while others run overlap with them on the GPU.  Because each job keeps
its own seed, step counter and statistics, its results are the same alone and
in any mix.

Device memory of the jobs comes from the torch caching allocator through the
library's allocator hook, so finishing a job does not call cudaFree.
"""
from __future__ import annotations

import concurrent.futures as cf
import time
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

from . import transsim as T


@dataclass
class Job:
    jid: int
    kind: str
    arrival: float            # seconds since the start of the stream
    make: Callable            # () -> Scenario
    steps: int
    footprint: int = 0
    admitted: float = 0.0
    finished: float = 0.0
    vehicle_updates: int = 0
    last_state_hash: int = 0
    rejected: bool = False    # its footprint alone exceeds the memory budget


@dataclass
class ServeReport:
    jobs: List[Job]           # served jobs, in completion order
    wall_s: float
    device_busy_s: float
    peak_active: int
    peak_bytes: int
    mean_active: float
    rejected: List[Job] = field(default_factory=list)  # jobs larger than the whole budget

    def latencies(self):
        return np.array([j.finished - j.arrival for j in self.jobs])

    def summary(self):
        lat = self.latencies()
        upd = sum(j.vehicle_updates for j in self.jobs)
        return {"jobs": len(self.jobs), "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)), "mean_latency_s": float(lat.mean()),
                "vehicle_updates": int(upd), "vehicle_updates_per_s": upd / self.wall_s,
                "wall_s": self.wall_s, "peak_active_jobs": self.peak_active,
                "mean_active_jobs": self.mean_active, "peak_job_bytes": self.peak_bytes,
                "rejected_jobs": len(self.rejected)}


def poisson_arrivals(rate_per_s: float, duration_s: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t >= duration_s:
            return np.array(out)
        out.append(t)


class Server:
    def __init__(self, budget_bytes: int, capacity: int = 1024, chunk_steps: int = 128, workers: int = 4):
        import torch
        self.budget = budget_bytes
        self.chunk = chunk_steps
        self.stream = torch.cuda.Stream()
        self.batch = T.Batch(capacity)
        self.capacity = capacity
        self.pool = cf.ThreadPoolExecutor(max_workers=workers)

    def _build(self, job: Job):
        sc = job.make()
        sim = T.Simulation(sc, use_torch_allocator=True)
        return sim

    def run(self, jobs: List[Job], time_scale: float = 1.0) -> ServeReport:
        """Serves `jobs` (sorted by arrival).  time_scale < 1 compresses the
        arrival clock (arrival times are multiplied by it)."""
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        pending = list(jobs)
        building = {}   # jid -> (job, future)
        ready = []      # (job, sim) built, waiting for memory
        active = {}     # jid -> (job, sim)
        used = 0
        done: List[Job] = []
        rejected: List[Job] = []
        busy = 0.0
        peak_active = peak_bytes = 0
        active_samples = []
        while pending or building or ready or active:
            t = now()
            while pending and pending[0].arrival * time_scale <= t:
                j = pending.pop(0)
                j.arrival *= time_scale
                building[j.jid] = (j, self.pool.submit(self._build, j))
            for jid in [k for k, (_, f) in building.items() if f.done()]:
                j, f = building.pop(jid)
                sim = f.result()
                j.footprint = T.footprint_bytes(sim.scenario)
                if j.footprint > self.budget:
                    # it would wait for memory forever: refuse it
                    sim.close()
                    j.rejected = True
                    j.finished = now()
                    rejected.append(j)
                    continue
                ready.append((j, sim))
            adds = []
            while ready and used + ready[0][0].footprint <= self.budget and len(active) + len(adds) < self.capacity:
                j, sim = ready.pop(0)
                j.admitted = now()
                used += j.footprint
                adds.append((j, sim))
            for steps in sorted({j.steps for j, _ in adds}):
                group = [(j, s) for j, s in adds if j.steps == steps]
                self.batch.add_many([s for _, s in group], steps)
                for j, s in group:
                    active[j.jid] = (j, s)
            peak_active = max(peak_active, len(active))
            peak_bytes = max(peak_bytes, used)
            if not active:
                nxt = pending[0].arrival * time_scale - now() if pending else 0.0
                time.sleep(max(0.0, min(nxt, 0.002)) if not building else 0.0005)
                continue
            active_samples.append(len(active))
            b0 = time.perf_counter()
            self.batch.step(self.chunk, self.stream)
            self.batch.sync()
            busy += time.perf_counter() - b0
            for jid in list(active):
                j, sim = active[jid]
                if sim.current_step() >= j.steps:
                    tot = sim.totals()
                    j.vehicle_updates = tot["vehicle_updates"]
                    j.last_state_hash = tot["last_state_hash"]
                    j.finished = now()
                    self.batch.remove(sim)
                    sim.close()
                    used -= j.footprint
                    del active[jid]
                    done.append(j)
        wall = now()
        return ServeReport(done, wall, busy, peak_active, peak_bytes,
                           float(np.mean(active_samples)) if active_samples else 0.0, rejected)

    def close(self):
        self.pool.shutdown()
        self.batch.close()
