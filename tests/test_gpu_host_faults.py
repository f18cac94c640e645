"""Failure handling made on the host (nothing here faults, traps or hangs a
GPU): an allocator that fails, a deadline that runs out, and a checkpoint
that is written back into a fresh context and continued."""
import ctypes

import numpy as np
import pytest

from paper_cs_0105004_gb300 import transsim as T
from paper_cs_0105004_gb300.inputs import networks as N

pytestmark = pytest.mark.gpu


def test_failing_allocator_reports_oom():
    calls = []

    def alloc(nbytes, stream, user):
        calls.append(nbytes)
        return None  # the caller's pool is exhausted

    def free(ptr, nbytes, stream, user):
        pass

    fa, ff = T.ALLOC_FN(alloc), T.FREE_FN(free)
    a = T.Allocator(fa, ff, None)
    sc = N.config0()
    net = T._NetArrays(sc.net)
    params = T.Params(sc.vmax, sc.p_threshold, sc.seed, sc.lane_change, 0)
    h = ctypes.c_void_p()
    rc = T.lib().ts_create_network(ctypes.byref(net.desc), ctypes.byref(params), ctypes.byref(a), ctypes.byref(h))
    assert rc == T.TS_ERR_OOM and not h.value and calls
    # the library stays usable
    T.Simulation(sc).close()


def test_short_deadline_times_out_then_the_result_arrives():
    sc = N.config1()
    sim = T.Simulation(sc)
    sim.step(sc.steps)  # no load balancing: the call only enqueues
    st = T.Stats()
    rc = T.lib().ts_read_stats(sim.h, ctypes.byref(st), 0)
    assert rc == T.TS_ERR_TIMEOUT
    assert sim.stats()["step"] == sc.steps - 1
    sim.close()


def test_checkpoint_resume_equals_the_uninterrupted_run():
    sc = N.small_grid_scenario(4, 2, 30, 800, 300, 1500, gen_seed=13, seed=31)
    full = T.Simulation(sc)
    full.step(1500)
    want = full.stats_range(700, 800)
    want_state = full.read_state()
    part = T.Simulation(sc)
    part.step(700)
    ck = part.read_state()
    part.close()
    init = N.InitialState(**{k: ck[k] for k in ("cell_id", "cell_v", "buf_id", "buf_v", "cursor", "dep_head")},
                          step=ck["step"], arrived=ck["arrived"], inserted=ck["inserted"])
    resumed = T.Simulation(sc)
    resumed.write_state(init)
    resumed.step(800)
    got = resumed.stats_range(700, 800)
    for f in T.STATS_FIELDS:
        assert np.array_equal(got[f], want[f]), f
    got_state = resumed.read_state()
    for k in ("cell_id", "cell_v", "buf_id", "buf_v", "cursor", "dep_head"):
        assert np.array_equal(got_state[k], want_state[k]), k
    full.close()
    resumed.close()


def test_checkpoint_bytes_round_trip():
    sc = N.small_grid_scenario(4, 2, 30, 800, 300, 1200, gen_seed=14, seed=32)
    full = T.Simulation(sc)
    full.step(1200)
    part = T.Simulation(sc)
    part.step(500)
    ck = part.save()
    assert ck[:4] == b"TSCK"
    part.close()
    resumed = T.Simulation(sc)
    resumed.load(ck)
    resumed.step(700)
    a, b = full.stats_range(500, 700), resumed.stats_range(500, 700)
    for f in T.STATS_FIELDS:
        assert np.array_equal(a[f], b[f]), f
    # a checkpoint of another network is refused
    other = T.Simulation(N.small_grid_scenario(3, 1, 20, 50, 50, 100, gen_seed=1))
    with pytest.raises(T.TsError, match="INVALID"):
        other.load(ck)
    for s in (full, resumed, other):
        s.close()
