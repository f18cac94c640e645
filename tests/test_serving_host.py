"""Host logic of the continuous-batching job server, on the CPU: the
library's simulation and batch objects are replaced by fakes that advance a
step counter, so the scheduling (arrival, admission by footprint against the
memory budget, batch capacity, departure at the target step, refusal of jobs
larger than the budget) is tested without a device."""
import types

import numpy as np
import pytest

from paper_cs_0105004_gb300 import serving as S


class FakeSim:
    def __init__(self, sc, use_torch_allocator=False, tile_words=None):
        self.scenario = sc
        self.step = 0
        self.target = None
        self.closed = False

    def current_step(self):
        return self.step

    def totals(self):
        return {"vehicle_updates": 7 * self.step, "last_state_hash": self.scenario.tag}

    def close(self):
        self.closed = True


class FakeBatch:
    log = []  # (event, job tag, members after the event)

    def __init__(self, capacity):
        self.capacity = capacity
        self.members = []

    def add_many(self, sims, target):
        for s in sims:
            assert s.step == 0 and not s.closed
            s.target = target
            self.members.append(s)
            FakeBatch.log.append(("add", s.scenario.tag, len(self.members)))
        assert len(self.members) <= self.capacity

    def step(self, n, stream):
        for s in self.members:
            s.step = min(s.step + n, s.target)  # each member stops at its own target

    def sync(self, timeout_ms=0):
        pass

    def remove(self, sim):
        self.members.remove(sim)
        FakeBatch.log.append(("remove", sim.scenario.tag, len(self.members)))

    def close(self):
        pass


@pytest.fixture
def fakes(monkeypatch):
    import torch
    monkeypatch.setattr(S.T, "Simulation", FakeSim)
    monkeypatch.setattr(S.T, "Batch", FakeBatch)
    monkeypatch.setattr(S.T, "footprint_bytes", lambda sc: sc.bytes)
    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: None)
    FakeBatch.log = []
    return FakeBatch


def _jobs(sizes, steps, spacing=0.001):
    jobs = []
    for i, (b, n) in enumerate(zip(sizes, steps)):
        sc = types.SimpleNamespace(bytes=b, tag=i)
        jobs.append(S.Job(i, "fake", i * spacing, (lambda sc=sc: sc), n))
    return jobs


def test_every_job_runs_to_its_target_within_the_budget(fakes):
    rng = np.random.default_rng(1)
    sizes = rng.integers(10, 60, 40).tolist()
    steps = rng.integers(1, 10, 40).tolist()
    server = S.Server(budget_bytes=150, capacity=64, chunk_steps=3, workers=2)
    rep = server.run(_jobs(sizes, steps))
    server.close()
    assert len(rep.jobs) == 40 and not rep.rejected
    for j in rep.jobs:
        assert j.vehicle_updates == 7 * j.steps  # stepped to its target, not past it
        assert j.arrival <= j.admitted <= j.finished
    assert rep.peak_bytes <= 150
    # the memory in use never exceeds the budget at any admission
    used, tag_bytes = 0, dict(enumerate(sizes))
    for ev, tag, _ in fakes.log:
        used += tag_bytes[tag] if ev == "add" else -tag_bytes[tag]
        assert used <= 150


def test_admission_is_first_come_first_served(fakes):
    # a large job at the head of the queue is not overtaken by small ones
    sizes = [90, 80, 5, 5, 5]
    server = S.Server(budget_bytes=100, capacity=8, chunk_steps=2, workers=1)
    rep = server.run(_jobs(sizes, [6, 6, 2, 2, 2]))
    server.close()
    adds = [tag for ev, tag, _ in fakes.log if ev == "add"]
    assert adds == [0, 1, 2, 3, 4]
    admitted = {j.jid: j.admitted for j in rep.jobs}
    assert admitted[1] >= max(j.finished for j in rep.jobs if j.jid == 0)


def test_batch_capacity_bounds_the_active_jobs(fakes):
    server = S.Server(budget_bytes=10**9, capacity=3, chunk_steps=1, workers=4)
    rep = server.run(_jobs([1] * 12, [4] * 12, spacing=0.0))
    server.close()
    assert len(rep.jobs) == 12 and rep.peak_active <= 3
    assert max(n for ev, _, n in fakes.log if ev == "add") <= 3


def test_a_job_larger_than_the_budget_is_refused(fakes):
    server = S.Server(budget_bytes=100, capacity=8, chunk_steps=2, workers=2)
    rep = server.run(_jobs([40, 101, 30], [3, 3, 3]))
    server.close()
    assert [j.jid for j in rep.rejected] == [1] and rep.rejected[0].rejected
    assert sorted(j.jid for j in rep.jobs) == [0, 2]
    assert rep.summary()["rejected_jobs"] == 1


def test_poisson_arrivals_rate():
    t = S.poisson_arrivals(20.0, 500.0, seed=7)
    assert np.all(np.diff(t) > 0) and t[-1] < 500.0
    assert abs(t.size / 500.0 - 20.0) < 0.6  # 10,000 expected, sd 100
