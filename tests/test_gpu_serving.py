"""Batching and serving: each job's result is the same alone and in the mix."""
import numpy as np
import pytest

import oracle

from paper_cs_0105004_gb300 import batching as Bt
from paper_cs_0105004_gb300 import serving as Sv
from paper_cs_0105004_gb300 import transsim as T
from paper_cs_0105004_gb300.inputs import networks as N

pytestmark = pytest.mark.gpu


def _small(i):
    return N.small_grid_scenario(3 + i % 4, 1 + i % 3, 20 + 3 * i, 60 + 25 * i, 80, 300, gen_seed=40 + i,
                                 seed=500 + i)


def _alone(sc, steps):
    sim = T.Simulation(sc)
    sim.step(steps)
    tot = sim.totals()
    sim.close()
    return tot


def test_served_jobs_equal_their_single_runs():
    scs = [_small(i) for i in range(12)]
    steps = 300
    alone = [_alone(sc, steps) for sc in scs]
    # arrivals closer together than a job lasts, so jobs join a running batch
    jobs = [Sv.Job(i, "grid", 0.002 * i, (lambda sc=sc: sc), steps) for i, sc in enumerate(scs)]
    jobs.sort(key=lambda j: j.arrival)
    srv = Sv.Server(budget_bytes=2**30, chunk_steps=32, workers=2)
    rep = srv.run(jobs)
    srv.close()
    assert len(rep.jobs) == len(scs)
    for j in rep.jobs:
        a = alone[j.jid]
        assert j.vehicle_updates == a["vehicle_updates"]
        assert j.last_state_hash == a["last_state_hash"]
        assert j.finished >= j.admitted >= j.arrival
        # and the oracle's run of the same job
        orc = oracle.Oracle(scs[j.jid])
        o = orc.step(steps)
        orc.close()
        assert j.vehicle_updates == int(o["vehicle_updates"].sum())
        assert j.last_state_hash == int(o["state_hash"][-1])
    assert rep.peak_active > 1  # jobs overlapped on the device


def test_admission_respects_the_memory_budget():
    scs = [_small(i) for i in range(6)]
    fp = max(T.footprint_bytes(sc) for sc in scs)
    jobs = [Sv.Job(i, "grid", 0.0, (lambda sc=sc: sc), 200) for i, sc in enumerate(scs)]
    srv = Sv.Server(budget_bytes=2 * fp, chunk_steps=32, workers=2)
    rep = srv.run(jobs)
    srv.close()
    assert len(rep.jobs) == 6 and rep.peak_bytes <= 2 * fp and rep.peak_active <= 2


def test_batched_run_equals_sequential_runs():
    import torch
    scs = [N.config3_scenario(i, demand_scale=0.05, steps=400) for i in range(4)]
    stream = torch.cuda.Stream()
    best, timings = Bt.autotune(scs, stream, tile_words=(32, 128), grids=(0, 2), window=64)
    assert best in timings and len(timings) == 8
    sims = Bt.make_members(scs, tile_words=best[0])
    batch = T.Batch(len(sims))
    batch.add_many(sims, 400)
    Bt.apply_shape(batch, best)
    b = Bt.run_batched(sims, 400, stream, batch)
    batch.close()
    s = Bt.run_sequential(sims, 400, stream)
    assert b.per_member_updates == s.per_member_updates
    for sim in sims:
        sim.close()
