"""Continuous-batching job server for simulation jobs.

Requests arrive as a Poisson stream.  A job's inputs are built on a worker
thread when it arrives; it is admitted to the running batch as soon as its
device footprint fits the memory budget; every batch step advances all
admitted jobs by a chunk of time steps, each towards its own target; a job
that reaches its target leaves the batch, its totals are read and its memory
returns to the pool.  Two batches alternate on the stream, so the host's
admission and retirement work on one overlaps the other's chunk on the
device.  State stays on the device between steps, and jobs that
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
    chunks: int = 0           # batch steps enqueued (each `chunk_steps` steps of one batch)

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
                "rejected_jobs": len(self.rejected), "chunks": self.chunks}


def poisson_arrivals(rate_per_s: float, duration_s: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t >= duration_s:
            return np.array(out)
        out.append(t)


class Server:
    """Two batches take turns on the stream: while the device runs one
    batch's chunk of steps, the host retires and admits jobs on the other
    and queues its chunk behind the running one, so admission and
    retirement never leave the device idle.  A job joins whichever batch is
    being served when it is admitted; `capacity` bounds the jobs of both."""

    def __init__(self, budget_bytes: int, capacity: int = 1024, chunk_steps: int = 128, workers: int = 4):
        import torch
        self.budget = budget_bytes
        self.chunk = chunk_steps
        self.stream = torch.cuda.Stream()
        self.batches = [T.Batch(capacity), T.Batch(capacity)]
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
        ready = []      # (job, sim) built, waiting for memory, in arrival order
        active = [{}, {}]   # per batch: jid -> (job, sim)
        queued = [False, False]  # a chunk of the batch is enqueued and not yet waited for
        used = 0
        done: List[Job] = []
        rejected: List[Job] = []
        busy = 0.0
        peak_active = peak_bytes = 0
        active_samples = []
        cur = 0
        chunks = 0
        while pending or building or ready or active[0] or active[1]:
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
            ready.sort(key=lambda r: (r[0].arrival, r[0].jid))
            b = self.batches[cur]
            if queued[cur]:
                # this batch's chunk ran before the other one's (still queued
                # or running); wait for it (bounded) and retire finished jobs
                b0 = time.perf_counter()
                b.sync()
                busy += time.perf_counter() - b0
                queued[cur] = False
                for jid in list(active[cur]):
                    j, sim = active[cur][jid]
                    if sim.current_step() >= j.steps:
                        tot = sim.totals()
                        j.vehicle_updates = tot["vehicle_updates"]
                        j.last_state_hash = tot["last_state_hash"]
                        j.finished = now()
                        b.remove(sim)
                        sim.close()
                        used -= j.footprint
                        del active[cur][jid]
                        done.append(j)
            # first come, first served: the head of the queue is admitted
            # when it fits, and nothing overtakes it
            adds = []
            n_active = len(active[0]) + len(active[1])
            while ready and used + ready[0][0].footprint <= self.budget and n_active + len(adds) < self.capacity:
                j, sim = ready.pop(0)
                j.admitted = now()
                used += j.footprint
                adds.append((j, sim))
            i = 0
            while i < len(adds):  # runs of equal targets, in arrival order
                e = i
                while e < len(adds) and adds[e][0].steps == adds[i][0].steps:
                    e += 1
                b.add_many([s for _, s in adds[i:e]], adds[i][0].steps)
                for j, s in adds[i:e]:
                    active[cur][j.jid] = (j, s)
                i = e
            peak_active = max(peak_active, len(active[0]) + len(active[1]))
            peak_bytes = max(peak_bytes, used)
            if active[cur]:
                active_samples.append(len(active[0]) + len(active[1]))
                b.step(self.chunk, self.stream)
                queued[cur] = True
                chunks += 1
            elif not queued[cur ^ 1]:
                nxt = pending[0].arrival * time_scale - now() if pending else 0.0
                time.sleep(max(0.0, min(nxt, 0.002)) if not building else 0.0005)
            cur ^= 1
        wall = now()
        return ServeReport(done, wall, busy, peak_active, peak_bytes,
                           float(np.mean(active_samples)) if active_samples else 0.0, rejected, chunks)

    def close(self):
        self.pool.shutdown()
        for b in self.batches:
            b.close()
