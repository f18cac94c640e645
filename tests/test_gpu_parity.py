"""GPU path vs the CPU oracle, bit-exact, through the C ABI.

Every comparison is exact: all arithmetic of the step is integer (cells,
velocities, 32-bit Philox words against an integer threshold, 64-bit digest
sums), so the CUDA library and the oracle must agree on every field of every
step and on the full state.
"""
import os

import numpy as np
import pytest

import oracle
from helpers import check_invariants, make_scenario
from paper_cs_0105004_gb300 import transsim as T
from paper_cs_0105004_gb300.inputs import networks as N

pytestmark = pytest.mark.gpu

FIELDS = T.STATS_FIELDS


def _cmp_stats(a, b, where=""):
    for f in FIELDS:
        if not np.array_equal(a[f], b[f]):
            bad = np.nonzero(a[f] != b[f])[0]
            i = int(bad[0])
            raise AssertionError(f"{where}: field {f} differs first at row {i} (step {int(a['step'][i])}): "
                                 f"gpu {int(a[f][i])} oracle {int(b[f][i])}")


def _cmp_state(g, o, where=""):
    for k in ("cell_id", "cell_v", "buf_id", "buf_v", "cursor", "dep_head"):
        if not np.array_equal(g[k], o[k]):
            i = int(np.nonzero(g[k] != o[k])[0][0])
            raise AssertionError(f"{where}: state {k} differs at {i}: gpu {g[k][i]} oracle {o[k][i]}")
    for k in ("step", "arrived", "inserted"):
        assert g[k] == o[k], (where, k, g[k], o[k])


def run_parity(sc, steps, chunk=None, state_every=None, tile_words=None, mode=None):
    sim = T.Simulation(sc, tile_words=tile_words)
    if mode is not None:
        sim.set_step_mode(mode)
    orc = oracle.Oracle(sc)
    t0 = sc.init.step if sc.init is not None else 0
    chunk = chunk or min(steps, 4000)
    done = 0
    while done < steps:
        n = min(chunk, steps - done)
        sim.step(n)
        g = sim.stats_range(t0 + done, n)
        o = orc.step(n)
        _cmp_stats(g, o, f"{sc.name} steps {t0 + done}..{t0 + done + n - 1}")
        done += n
        if state_every and (done % state_every == 0 or done == steps):
            _cmp_state(sim.read_state(), orc.get_state(), f"{sc.name} after step {t0 + done - 1}")
    _cmp_state(sim.read_state(), orc.get_state(), f"{sc.name} final")
    sim.close()
    return o


# ------------------------------------------------------------------ hand-built cases

def test_hand_cases_match_oracle():
    cases = [
        make_scenario([(0, 1, 200, 1)], 2, [[0]], [0]),
        make_scenario([(0, 1, 12, 1), (1, 2, 12, 1)], 3, [[0, 1]], [0]),
        make_scenario([(0, 2, 12, 1), (1, 2, 12, 1), (2, 3, 12, 1)], 4, [[0, 2], [1, 2]], [0, 0]),
        make_scenario([(0, 1, 40, 2)], 2, [[0], [0]], [0, 0], placed=[(0, 0, 0, 10, 3), (1, 0, 0, 12, 0)]),
        make_scenario([(0, 1, 40, 2)], 2, [[0], [0]], [0, 0], placed=[(0, 0, 0, 10, 3), (1, 0, 0, 12, 0)],
                      start_step=1),
        make_scenario([(0, 1, 20, 2), (1, 2, 20, 3), (3, 1, 20, 1)], 4, [[0, 1], [2, 1]], [0, 0],
                      bufs=[(0, 0, 1, 3)], placed=[(1, 2, 0, 5, 0)]),
    ]
    for sc in cases:
        run_parity(sc, 40, chunk=1, state_every=1)


def test_single_step_granularity_small_grid():
    sc = N.small_grid_scenario(3, 2, 20, n_trips=80, window=40, steps=120, gen_seed=2, seed=5)
    run_parity(sc, 120, chunk=1, state_every=1)


# ------------------------------------------------------------------ rings (Sec. 5 circle roads)

def _ring(L, n, lanes, p, vmax=5, seed=3, rng_seed=0):
    net = N.ring_network(L, lanes)
    dem, init = N.ring_initial_state(net, n, "random", 0, np.random.default_rng(rng_seed))
    return N.Scenario(f"ring{L}x{lanes}", net, dem, 0, seed, vmax, p, 1, init)


@pytest.mark.parametrize("L,lanes,rho", [(64, 1, 0.3), (320, 1, 0.2), (320, 3, 0.25), (9984, 1, 0.15),
                                         (9984, 3, 0.3), (4128, 2, 0.5)])
def test_rings_match_oracle(L, lanes, rho):
    # 9984 and 4128 cells are longer than one tile: the ring is split into
    # partial tiles whose halos wrap around the ring
    sc = _ring(L, int(rho * L * lanes), lanes, N.P_THRESHOLD_0_2, rng_seed=L + lanes)
    run_parity(sc, 300, chunk=100, state_every=100)


@pytest.mark.parametrize("vmax", [1, 3, 9, 15])
def test_rings_other_vmax(vmax):
    sc = _ring(4160, 2000, 2, N.P_THRESHOLD_0_2, vmax=vmax, rng_seed=vmax)
    run_parity(sc, 200, chunk=50, state_every=50)


# ------------------------------------------------------------------ grids and planar networks

@pytest.mark.parametrize("case", [(3, 1, 20, 100, 1, 5), (4, 2, 25, 400, 2, 5), (4, 3, 15, 500, 3, 5),
                                  (5, 2, 60, 2000, 4, 5), (3, 2, 40, 300, 5, 7), (4, 2, 33, 300, 6, 15)])
@pytest.mark.parametrize("mode", [T.STEP_FUSED, T.STEP_SPLIT])
def test_small_grids_match_oracle(case, mode):
    side, lanes, cells, trips, seed, vmax = case
    sc = N.small_grid_scenario(side, lanes, cells, trips, 200, 800, gen_seed=seed, seed=seed * 7 + 1, vmax=vmax)
    # chunks of 200 steps end inside a captured chunk of 32 (200 = 6*32 + 8)
    run_parity(sc, 800, chunk=200, state_every=200, mode=mode)


def test_long_links_partial_tiles():
    # links longer than a tile (128 words = 4096 one-lane cells), including tails that
    # would leave fewer than 2*vmax+1 cells after a split
    cells = [2048 + 5, 4096 + 3, 2100, 64 * 32 * 2 + 1, 31, 3, 70]
    links, routes = [], []
    n = len(cells) + 1
    for i, c in enumerate(cells):
        links.append((i, i + 1, c, 1 + i % 3))
        links.append((i + 1, i, c, 1 + (i + 1) % 3))
    rng = np.random.default_rng(11)
    dep = []
    for v in range(600):
        a, b = sorted(rng.choice(n, 2, replace=False))
        if rng.random() < 0.5:
            routes.append([2 * i for i in range(a, b)])
        else:
            routes.append([2 * i + 1 for i in range(b - 1, a - 1, -1)])
        dep.append(int(rng.integers(0, 300)))
    sc = make_scenario(links, n, routes, dep, steps=1500, seed=77, p=N.P_THRESHOLD_0_2)
    for tc, mode in ((128, T.STEP_FUSED), (8, T.STEP_FUSED), (8, T.STEP_SPLIT), (256, T.STEP_SPLIT)):
        run_parity(sc, 1500, chunk=500, state_every=500, tile_words=tc, mode=mode)


@pytest.mark.parametrize("mode", [T.STEP_FUSED, T.STEP_AUTO])
def test_config0_full_run(mode):
    sc = N.config0()
    run_parity(sc, sc.steps, chunk=900, state_every=900, mode=mode)


def test_config0_tile_shapes_identical():
    sc = N.config0()
    ref = None
    for tc in (8, 16, 32, 64, 128, 256):
        sim = T.Simulation(sc, tile_words=tc)
        sim.step(1200)
        st = sim.stats_range(0, 1200)
        if ref is None:
            ref = st
        else:
            _cmp_stats(st, ref, f"tile columns {tc}")
        sim.close()


def test_load_balancing_keeps_results():
    # re-tiling from the occupancy every 64 steps with a small vehicle budget
    # splits jammed stretches into many partial tiles; results stay identical
    sc = N.small_grid_scenario(4, 3, 70, n_trips=3000, window=300, steps=1500, gen_seed=8, seed=21)
    sim = T.Simulation(sc)
    sim.set_load_balance(64, 128)
    orc = oracle.Oracle(sc)
    sim.step(1500)
    _cmp_stats(sim.stats_range(0, 1500), orc.step(1500), "load balanced")
    _cmp_state(sim.read_state(), orc.get_state(), "load balanced final")
    sim.close()


def test_planar_network_window():
    sc = N._planar_config("planar-small", 900, 1060, 20000, 5, steps=1200)
    run_parity(sc, 1200, chunk=400, state_every=400)


@pytest.mark.parametrize("mode", [T.STEP_AUTO, T.STEP_FUSED])
def test_config1_first_window(mode):
    # Portland-shaped network, full size, first 1,200 steps (the oracle's
    # share of the test); later steps are covered by the invariants test
    sc = N.config1()
    run_parity(sc, 1200, chunk=400, state_every=1200, mode=mode)


def test_invariants_hold_on_gpu_config1():
    sc = N.config1()
    sim = T.Simulation(sc)
    prev = None
    for k in range(6):
        sim.step(1000 if k else 3000)
        st = sim.stats()
        s = sim.read_state()
        prev = check_invariants(sc, s, st, None)
    sim.close()


# ------------------------------------------------------------------ batching

@pytest.mark.parametrize("mode", [T.STEP_FUSED, T.STEP_SPLIT])
def test_batch_equals_alone(mode):
    scs = [N.small_grid_scenario(3 + i % 3, 1 + i % 3, 20 + 5 * i, 100 + 40 * i, 100, 400, gen_seed=20 + i,
                                 seed=100 + i) for i in range(6)]
    alone = []
    for sc in scs:
        sim = T.Simulation(sc)
        sim.step(400)
        alone.append(sim.stats_range(0, 400))
        sim.close()
    import torch
    stream = torch.cuda.Stream()
    b = T.Batch(8)
    b.set_step_mode(mode)
    sims = [T.Simulation(sc) for sc in scs]
    targets = [400, 400, 250, 400, 123, 400]
    for s, tgt in zip(sims, targets):
        b.add(s, tgt)
    b.step(450, stream)
    b.sync()
    for s, tgt, ref in zip(sims, targets, alone):
        assert s.current_step() == tgt
        _cmp_stats(s.stats_range(0, tgt), ref[:tgt], "batch member")
    # continue two members alone after removing them from the batch
    b.remove(sims[2])
    sims[2].step(150)
    sc2 = scs[2]
    full = T.Simulation(sc2)
    full.step(400)
    _cmp_stats(sims[2].stats_range(250, 150), full.stats_range(250, 150), "resumed member")
    b.close()


def test_batch_switches_between_vmax_instances():
    # members with vmax 5 run in the instances compiled for vmax 5; a member
    # with another vmax joining the batch switches it to the general ones,
    # and its leaving switches it back: every member's steps stay those of
    # its single run, which for the vmax-7 member is checked against the oracle
    import torch
    scs = [N.small_grid_scenario(4, 2, 30, 300, 100, 300, gen_seed=31, seed=71),
           N.small_grid_scenario(3, 3, 25, 250, 100, 300, gen_seed=32, seed=72),
           N.small_grid_scenario(4, 2, 27, 300, 100, 300, gen_seed=33, seed=73, vmax=7)]
    alone = []
    for sc in scs:
        sim = T.Simulation(sc)
        sim.step(300)
        alone.append(sim.stats_range(0, 300))
        sim.close()
    orc = oracle.Oracle(scs[2])
    o = orc.step(300)
    orc.close()
    assert [int(x) for x in o["state_hash"]] == [int(r["state_hash"]) for r in alone[2]]
    stream = torch.cuda.Stream()
    b = T.Batch(4)
    sims = [T.Simulation(sc) for sc in scs]
    b.add(sims[0], 300)
    b.add(sims[1], 300)
    b.step(96, stream)       # vmax-5 instances
    b.add(sims[2], 300)
    b.step(96, stream)       # general instances
    b.remove(sims[2])
    b.step(300, stream)      # vmax-5 instances again
    b.sync()
    sims[2].step(204)        # the vmax-7 member alone
    for s, ref, name in zip(sims, alone, ("first", "second", "vmax 7")):
        assert s.current_step() == 300
        _cmp_stats(s.stats_range(0, 300), ref, name)
    b.close()


# ------------------------------------------------------------------ link travel times

@pytest.mark.parametrize("mode", [T.STEP_FUSED, T.STEP_SPLIT])
def test_link_travel_times_match_oracle(mode):
    for sc in (N.config0(), N.small_grid_scenario(4, 3, 15, 500, 200, 800, gen_seed=3, seed=22)):
        sim = T.Simulation(sc)
        sim.set_step_mode(mode)
        orc = oracle.Oracle(sc)
        for n in (500, sc.steps - 500):   # chunk boundaries inside captured chunks
            sim.step(n)
            orc.step(n)
            g, o = sim.link_times(), orc.link_times()
            assert np.array_equal(g[0], o[0]) and np.array_equal(g[1], o[1]), sc.name
        sim.reset()
        sim.step(100)
        orc2 = oracle.Oracle(sc)
        orc2.step(100)
        assert np.array_equal(sim.link_times()[0], orc2.link_times()[0]), "after reset"
        sim.close()


# ------------------------------------------------------------------ input validation

def test_malformed_routes_are_rejected():
    links = [(0, 1, 12, 1), (1, 2, 12, 1), (2, 0, 12, 1), (0, 0, 64, 1, 1)]  # the last one is a ring
    good = make_scenario(links, 3, [[0, 1]], [0])
    T.Simulation(good).close()
    for routes in ([[0, 2]],        # link 0 ends at node 1, link 2 starts at node 2
                   [[0, 7]],        # no link 7
                   [[3, 3]]):       # a ring link must be the whole route
        sc = make_scenario(links, 3, routes, [0])
        with pytest.raises(T.TsError, match="INVALID"):
            T.Simulation(sc)


# ------------------------------------------------------------------ traffic signals

@pytest.mark.parametrize("mode", [T.STEP_FUSED, T.STEP_SPLIT])
@pytest.mark.parametrize("case", [(4, 2, 20, 500, 2, (30, 15)), (5, 3, 45, 1500, 7, (60, 30)),
                                  (3, 1, 12, 300, 9, (16, 5))])
def test_signalled_grids_match_oracle(case, mode):
    side, lanes, cells, trips, seed, signal = case
    sc = N.small_grid_scenario(side, lanes, cells, trips, 200, 900, gen_seed=seed, seed=seed + 40, signal=signal)
    run_parity(sc, 900, chunk=300, state_every=300, mode=mode)
    sim = T.Simulation(sc)
    orc = oracle.Oracle(sc)
    sim.step(900)
    orc.step(900)
    g, o = sim.link_times(), orc.link_times()
    assert np.array_equal(g[0], o[0]) and np.array_equal(g[1], o[1])
    sim.close()


def test_planar_network_with_signals_matches_oracle():
    # a light at every approach of every node with two or more approaches
    # (signals_by_rank), on a 900-node planar network
    import dataclasses
    sc = N._planar_config("planar-small", 900, 1060, 20000, 5, steps=900)
    sc = dataclasses.replace(sc, net=dataclasses.replace(sc.net, link_signal=N.signals_by_rank(sc.net, 40, 20)))
    run_parity(sc, 900, chunk=300, state_every=300)


def test_car_waits_at_a_red_light_on_gpu():
    sc = make_scenario([(0, 1, 20, 1), (1, 2, 20, 1)], 3, [[0, 1]], [0], p=0, steps=30)
    sc.net.link_signal = np.array([[40, 20, 20], [0, 0, 0]], np.uint32)
    run_parity(sc, 30, chunk=1)


# ------------------------------------------------------------------ edge cases

def _grid_with(side, lanes, cells, trips, steps, seed, **kw):
    sc = N.small_grid_scenario(side, lanes, cells, trips, 150, steps, gen_seed=seed, seed=seed + 3)
    for k, v in kw.items():
        setattr(sc, k, v)
    return sc


def test_no_travellers_at_all():
    sc = N.small_grid_scenario(4, 2, 20, 0, 10, 300, gen_seed=1)
    o = run_parity(sc, 300, chunk=100)
    assert int(o["active"].max()) == 0 and int(o["state_hash"].max()) == 0


def test_four_lane_links():
    sc = N.small_grid_scenario(4, 4, 40, 1500, 200, 700, gen_seed=17, seed=5)
    run_parity(sc, 700, chunk=350, state_every=350)


@pytest.mark.parametrize("mode", [T.STEP_FUSED, T.STEP_SPLIT])
def test_lane_changes_off(mode):
    sc = _grid_with(4, 3, 25, 900, 600, 19, lane_change=0)
    o = run_parity(sc, 600, chunk=300, state_every=300, mode=mode)
    assert int(o["lane_changes"].sum()) == 0


def test_slowdown_almost_always():
    # every draw but 2^32-1 slows a moving vehicle down by one
    sc = _grid_with(4, 2, 30, 600, 500, 23, p_threshold=0xFFFFFFFF)
    run_parity(sc, 500, chunk=250, state_every=250)


def test_vmax_one_grid():
    sc = _grid_with(3, 2, 15, 300, 500, 29, vmax=1)
    run_parity(sc, 500, chunk=250, state_every=250)


def test_longest_link_allowed():
    # cells per link up to 2^22 - 1 (the buffered-vehicle digest packs 22 bits)
    L = (1 << 22) - 1
    routes = [[0, 1]] * 6 + [[1]] * 4
    sc = make_scenario([(0, 1, L, 2), (1, 2, 40, 1)], 3, routes, [0, 0, 1, 2, 3, 4, 0, 1, 2, 5], steps=300,
                       p=N.P_THRESHOLD_0_2, seed=9)
    run_parity(sc, 300, chunk=150, state_every=150)


def test_large_tiles_on_a_loaded_grid():
    # 256-word tiles: every word phase loops twice per tile
    sc = N.small_grid_scenario(6, 3, 60, 4000, 300, 900, gen_seed=31, seed=8)
    run_parity(sc, 900, chunk=300, state_every=300, tile_words=256)


def test_config1_busy_window_from_the_oracle_state():
    # full-size config 1 started from the oracle's own state at step 2,400
    # (congestion building up), then 300 steps on both sides, with the
    # bench's load balancing
    sc = N.config1()
    orc = oracle.Oracle(sc)
    orc.step(2400)
    s = orc.get_state()
    init = N.InitialState(**{k: s[k] for k in ("cell_id", "cell_v", "buf_id", "buf_v", "cursor", "dep_head")},
                          step=s["step"], arrived=s["arrived"], inserted=s["inserted"])
    sim = T.Simulation(sc)
    sim.set_load_balance(64, 768)
    sim.write_state(init)
    sim.step(300)
    _cmp_stats(sim.stats_range(2400, 300), orc.step(300), "config1 from step 2400")
    _cmp_state(sim.read_state(), orc.get_state(), "config1 after step 2699")
    sim.close()


# ------------------------------------------------------------------ full-size networks of the other workloads

def test_config2_network_with_a_trip_sample_matches_oracle():
    # the full config-2 network (200,000 links, 18.2 M lane-cells) with a
    # sample of its 2 M trips: those whose origin is among the first 1,500
    # distinct origins of the draw (so routes need 1,500 shortest-path trees),
    # departures brought forward by 5,000 s (clamped at 0: about 40 % are due
    # at step 0); 128-word tiles with re-tiling from the occupancy every 64
    # steps; 300 steps against the oracle
    net = N.planar_network(85_000, 100_000, 2)
    rng = np.random.default_rng(2 + 7919)
    o, d, dep = N.degree_weighted_trips(net, 2_000_000, 5400.0, 2400.0, 10800, rng)
    _, first = np.unique(o, return_index=True)
    origins = o[np.sort(first)[:1500]]
    keep = np.nonzero(np.isin(o, origins))[0]
    dep2 = np.maximum(dep[keep].astype(np.int64) - 5000, 0).astype(np.uint32)
    sc = N.Scenario("config2-sample", net, N._demand(net, o[keep], d[keep], dep2), steps=300, seed=1)
    sim = T.Simulation(sc, tile_words=128)
    sim.set_load_balance(64, 768)
    orc = oracle.Oracle(sc)
    sim.step(300)
    g = sim.stats_range(0, 300)
    _cmp_stats(g, orc.step(300), "config2 sample")
    _cmp_state(sim.read_state(), orc.get_state(), "config2 sample after step 299")
    assert int(g["active"][-1]) > 10_000
    sim.close()
    orc.close()


# ------------------------------------------------------------------ the loaded regime

def test_config1_departure_peak_from_the_oracle_state():
    # full-size config 1 from the oracle's own state at step 5,400, the
    # departure peak (most of the network jammed), 300 steps on both sides
    # with the bench's load balancing
    sc = N.config1()
    orc = oracle.Oracle(sc)
    orc.step(5400)
    s = orc.get_state()
    init = N.InitialState(**{k: s[k] for k in ("cell_id", "cell_v", "buf_id", "buf_v", "cursor", "dep_head")},
                          step=s["step"], arrived=s["arrived"], inserted=s["inserted"])
    sim = T.Simulation(sc)
    sim.set_load_balance(64, 768)
    sim.write_state(init)
    sim.step(300)
    g = sim.stats_range(5400, 300)
    _cmp_stats(g, orc.step(300), "config1 from step 5400")
    _cmp_state(sim.read_state(), orc.get_state(), "config1 after step 5699")
    assert int(g["active"].min()) > 50_000
    sim.close()
    orc.close()


def test_config2_full_demand_peak_window():
    # the full config-2 network with all 2 M trips, from the seeded
    # peak-hour state at step 5,400 that both sides load (about 618 k
    # vehicles on links, a third of the links queued to their end, link-end
    # buffers taken); 300 steps with the bench's tiles and re-tiling every
    # 64 steps, so tiles at the 768-vehicle budget are compared too
    import dataclasses
    sc = N.config2()
    scl = dataclasses.replace(sc, init=N.loaded_state(sc, 5400, seed=7))
    orc = oracle.Oracle(scl)
    st0 = orc.get_state()
    sim = T.Simulation(scl, tile_words=128)
    sim.set_load_balance(64, 768)
    _cmp_state(sim.read_state(), st0, "config2 peak state as loaded")
    sim.step(300)
    g = sim.stats_range(5400, 300)
    o = orc.step(300)
    _cmp_stats(g, o, "config2 from the peak state")
    s = orc.get_state()
    _cmp_state(sim.read_state(), s, "config2 after step 5699")
    check_invariants(scl, s, o[-1])
    assert int(g["active"].min()) > 500_000 and int(g["transfers"].sum()) > 10_000
    sim.close()
    orc.close()


def _oracle_member(i, steps):
    import oracle as O
    sc = N.config3_scenario(i)
    orc = O.Oracle(sc)
    st = orc.step(steps)
    s = orc.get_state()
    orc.close()
    return st, s


def test_config3_all_16_batch_members_match_oracle():
    # every member of the 16-scenario batch against the oracle (oracle runs in
    # spawned worker processes)
    import multiprocessing as mp
    import torch
    from paper_cs_0105004_gb300 import batching as Bt
    steps = 360
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        ref = pool.starmap(_oracle_member, [(i, steps) for i in range(16)])
    scs = [N.config3_scenario(i) for i in range(16)]
    sims = Bt.make_members(scs, tile_words=128)
    b = T.Batch(len(sims))
    b.add_many(sims, steps)
    stream = torch.cuda.Stream()
    b.step(steps, stream)
    b.sync()
    for i in range(16):
        _cmp_stats(sims[i].stats_range(0, steps), ref[i][0], f"config3 member {i}")
        _cmp_state(sims[i].read_state(), ref[i][1], f"config3 member {i} after step {steps - 1}")
    b.close()


def test_three_lane_circle_on_the_gpu():
    # the 3-lane circle of Sec. 5 at density 0.2 and p = 0.2 (the oracle pin
    # checks its flow per lane against the 1-lane circle): GPU = oracle
    sc = _ring(1024, int(0.2 * 1024 * 3), 3, N.P_THRESHOLD_0_2, rng_seed=11)
    o = run_parity(sc, 2000, chunk=500, state_every=1000)
    assert int(o["lane_changes"].sum()) > 0


def test_kernel_spans_inside_the_graphs():
    # kernel timing on: the same results, one link and one node launch per
    # step, and the summed spans inside the CUDA-event time of the run
    import torch
    sc = N.config0()
    sim = T.Simulation(sc)
    sim.step(640)
    ref = sim.stats_range(0, 640)
    sim.reset()
    sim.set_kernel_timing(True)
    s = torch.cuda.Stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    sim.step(640, s)
    b.record(s)
    b.synchronize()
    kt = sim.kernel_times()
    _cmp_stats(sim.stats_range(0, 640), ref, "with kernel spans")
    assert kt["link_launches"] == 640 and kt["node_launches"] == 640
    assert 0 < kt["link_s"] + kt["node_s"] <= a.elapsed_time(b) / 1000.0
    sim.kernel_times(reset=True)
    assert sim.kernel_times()["link_launches"] == 0
    sim.close()


def test_load_balancing_keeps_ts_step_asynchronous():
    # re-tiling from the occupancy is a kernel on the step stream: ts_step
    # returns while the steps still run (a zero-deadline read times out), and
    # the result equals the oracle
    sc = N.small_grid_scenario(5, 3, 70, n_trips=6000, window=400, steps=3000, gen_seed=12, seed=31)
    sim = T.Simulation(sc)
    sim.set_load_balance(64, 128)
    sim.step(64)  # captures the graphs
    sim.stats()
    sim.step(sc.steps - 64)
    with pytest.raises(T.TsError, match="TIMEOUT"):
        sim.stats(timeout_ms=0)
    orc = oracle.Oracle(sc)
    _cmp_stats(sim.stats_range(0, sc.steps), orc.step(sc.steps), "load balanced on the device")
    _cmp_state(sim.read_state(), orc.get_state(), "load balanced on the device, final")
    sim.close()
