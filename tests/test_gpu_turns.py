"""The intersection rules of Sec. 3 on the GPU vs the CPU oracle, bit-exact,
through the C ABI: plan-following lane changes (turn lanes) and gap
acceptance at unprotected turns (yield approaches) — hand-built cases, grids
with one to four lanes, partial tiles, signals, batches that mix scenarios
with and without those rules, states written from the oracle, and
checkpoints."""
import dataclasses

import numpy as np
import pytest

import oracle
from helpers import make_scenario
from paper_cs_0105004_gb300 import transsim as T
from paper_cs_0105004_gb300.inputs import networks as N
from test_gpu_parity import _cmp_state, _cmp_stats, run_parity

pytestmark = pytest.mark.gpu


def _fork(placed, routes, lane_change=1, start_step=0, depart=None):
    # link 0 (2 lanes, 20 cells) ends at node 1; links 1 and 2 leave it, link
    # 1 taken from lane 0 only and link 2 from lane 1 only
    sc = make_scenario([(0, 1, 20, 2), (1, 2, 10, 1), (1, 3, 10, 1)], 4, routes,
                       depart if depart is not None else [0] * len(routes), p=0, lane_change=lane_change,
                       placed=placed, start_step=start_step, steps=40)
    sc.net.turn_lanes = np.array([0b01, 0b10], np.uint8)
    return sc


def _with_turns(sc):
    return dataclasses.replace(sc, net=dataclasses.replace(sc.net, turn_lanes=N.turn_lanes_by_rank(sc.net)))


@pytest.mark.parametrize("mode", [T.STEP_FUSED, T.STEP_SPLIT])
def test_hand_cases_match_oracle(mode):
    cases = [
        _fork([(0, 0, 1, 0, 0)], [[0, 1]]),
        _fork([(0, 0, 1, 0, 0)], [[0, 1]], lane_change=0),
        _fork([(0, 0, 1, 0, 0)], [[0, 2]], lane_change=0),
        _fork([(0, 0, 1, 10, 0), (1, 0, 0, 8, 0)], [[0, 1], [0, 1]], start_step=1),
        _fork([(0, 0, 1, 18, 0), (1, 0, 0, 16, 0)], [[0, 1], [0, 1]], start_step=1),
        _fork([(0, 0, 1, 19, 0), (1, 0, 0, 18, 0)], [[0, 1], [0, 1]], start_step=1),
        _fork([(0, 0, 0, 5, 3), (1, 0, 0, 7, 0)], [[0, 1], [0, 1]]),
        # departures onto link 0 heading for either turn
        _fork(None, [[0, 1], [0, 2], [0, 1], [0, 2], [0, 2], [0, 1]], depart=[0, 0, 1, 1, 2, 3]),
    ]
    for sc in cases:
        run_parity(sc, 40, chunk=1, state_every=1, mode=mode)


@pytest.mark.parametrize("mode", [T.STEP_FUSED, T.STEP_SPLIT])
@pytest.mark.parametrize("case", [(3, 2, 20, 200, 1, 5, None), (4, 3, 25, 600, 2, 5, 6), (4, 4, 30, 900, 3, 5, 7),
                                  (5, 4, 60, 2000, 4, 5, 8), (3, 3, 40, 400, 5, 7, 9), (4, 4, 33, 500, 6, 15, 10),
                                  (4, 2, 18, 500, 7, 1, None)])
def test_grids_with_turn_lanes_match_oracle(case, mode):
    side, lanes, cells, trips, seed, vmax, lane_seed = case
    sc = N.small_grid_scenario(side, lanes, cells, trips, 200, 800, gen_seed=seed, seed=seed * 5 + 2, vmax=vmax,
                               turns=True, lane_seed=lane_seed)
    o = run_parity(sc, 800, chunk=200, state_every=200, mode=mode)
    assert int(o["arrived"][-1]) > 0


@pytest.mark.parametrize("mode", [T.STEP_FUSED, T.STEP_SPLIT])
def test_turn_lanes_with_signals(mode):
    sc = N.small_grid_scenario(5, 3, 45, 1500, 200, 900, gen_seed=11, seed=12, signal=(60, 30), turns=True,
                               lane_seed=12)
    run_parity(sc, 900, chunk=300, state_every=300, mode=mode)


def test_turn_lanes_on_partial_tiles():
    # a chain of links longer than a tile, both directions: tiles split inside
    # links, and the plan-following decisions near a split are re-computed in
    # the halo columns
    cells = [2048 + 5, 4096 + 3, 2100, 64 * 32 * 2 + 1, 31, 3, 70]
    links, routes = [], []
    n = len(cells) + 1
    for i, c in enumerate(cells):
        links.append((i, i + 1, c, 2 + i % 3))
        links.append((i + 1, i, c, 2 + (i + 1) % 3))
    rng = np.random.default_rng(13)
    dep = []
    for v in range(700):
        a, b = sorted(rng.choice(n, 2, replace=False))
        if rng.random() < 0.5:
            routes.append([2 * i for i in range(a, b)])
        else:
            routes.append([2 * i + 1 for i in range(b - 1, a - 1, -1)])
        dep.append(int(rng.integers(0, 300)))
    sc = _with_turns(make_scenario(links, n, routes, dep, steps=1500, seed=78, p=N.P_THRESHOLD_0_2))
    for tc, mode in ((128, T.STEP_SPLIT), (8, T.STEP_FUSED), (256, T.STEP_SPLIT)):
        run_parity(sc, 1500, chunk=500, state_every=500, tile_words=tc, mode=mode)


def test_planar_network_with_turn_lanes():
    sc = _with_turns(N._planar_config("planar-small", 900, 1060, 20000, 5, steps=1200))
    run_parity(sc, 1200, chunk=400, state_every=400)


def test_config1_with_turn_lanes_first_window():
    sc = _with_turns(N.config1())
    run_parity(sc, 900, chunk=300, state_every=900)


def test_state_from_the_oracle_and_checkpoint():
    # the oracle's state at step 300 written to the GPU (velocity bytes and
    # buffers rebuilt with the allowed lanes), 300 more steps on both sides;
    # then a checkpoint of the GPU state resumed in a fresh context
    sc = N.small_grid_scenario(4, 4, 30, 1200, 300, 900, gen_seed=21, seed=22, turns=True, lane_seed=23)
    orc = oracle.Oracle(sc)
    orc.step(300)
    s = orc.get_state()
    init = N.InitialState(**{k: s[k] for k in ("cell_id", "cell_v", "buf_id", "buf_v", "cursor", "dep_head")},
                          step=s["step"], arrived=s["arrived"], inserted=s["inserted"])
    sim = T.Simulation(sc)
    sim.write_state(init)
    sim.step(300)
    _cmp_stats(sim.stats_range(300, 300), orc.step(300), "from the oracle state")
    _cmp_state(sim.read_state(), orc.get_state(), "after step 599")
    ck = sim.save()
    sim.step(300)
    want = sim.stats_range(600, 300)
    sim.close()
    resumed = T.Simulation(sc)
    resumed.load(ck)
    resumed.step(300)
    _cmp_stats(resumed.stats_range(600, 300), want, "resumed checkpoint")
    _cmp_stats(want, orc.step(300), "oracle")
    resumed.close()


@pytest.mark.parametrize("mode", [T.STEP_FUSED, T.STEP_SPLIT])
def test_batch_mixing_rules_and_no_rules_equals_alone(mode):
    # members with and without turn lanes or yield approaches share the
    # intersection-rule launches
    scs = [N.small_grid_scenario(3 + i % 3, 2 + i % 3, 20 + 5 * i, 150 + 40 * i, 100, 400, gen_seed=40 + i,
                                 seed=140 + i, turns=bool(i % 2), yield_gap=5 + i if i % 3 == 2 else None)
           for i in range(6)]
    alone = []
    for sc in scs:
        sim = T.Simulation(sc)
        sim.step(400)
        alone.append(sim.stats_range(0, 400))
        sim.close()
    for sc, ref in zip(scs, alone):
        _cmp_stats(ref, oracle.Oracle(sc).step(400), "alone vs oracle")
    import torch
    stream = torch.cuda.Stream()
    b = T.Batch(8)
    b.set_step_mode(mode)
    sims = [T.Simulation(sc) for sc in scs]
    for s in sims:
        b.add(s, 400)
    b.step(400, stream)
    b.sync()
    for s, ref in zip(sims, alone):
        _cmp_stats(s.stats_range(0, 400), ref, "batch member")
    b.close()


def test_malformed_turn_tables_are_rejected():
    sc = _fork(None, [[0, 1]])
    T.Simulation(sc).close()
    for bad in ([0b01, 0b00],    # a turn with no lane
                [0b01, 0b100]):  # lane 2 of a two-lane link
        sc.net.turn_lanes = np.array(bad, np.uint8)
        with pytest.raises(T.TsError, match="INVALID"):
            T.Simulation(sc)


# ------------------------------------------------------------------ gap acceptance

def _tee(placed, bufs, gap=5, p_cells=20, p=0):
    sc = make_scenario([(2, 1, 20, 1), (0, 1, p_cells, 1), (1, 3, 20, 1)], 4, [[0, 2], [1, 2]], [0, 0], p=p,
                       placed=placed, bufs=bufs, steps=30)
    sc.net.link_yield = np.array([gap, 0, 0], np.uint8)
    return sc


@pytest.mark.parametrize("mode", [T.STEP_FUSED, T.STEP_SPLIT])
def test_gap_acceptance_hand_cases_match_oracle(mode):
    cases = [
        _tee([(1, 1, 0, 10, 5)], [(0, 0, 0, 2)]),
        _tee([(1, 1, 0, 5, 0)], [(0, 0, 0, 2)]),
        _tee([(1, 1, 0, 0, 0)], [(0, 0, 0, 2)], gap=31, p_cells=4, p=0xFFFFFFFF),
        _tee([(1, 1, 0, 1, 0)], [(0, 0, 0, 2)], gap=31, p_cells=4, p=0xFFFFFFFF),
        # a 40-cell priority link: the gap of 31 cells spans two columns
        _tee([(1, 1, 0, 9, 0)], [(0, 0, 0, 2)], gap=31, p_cells=40, p=0xFFFFFFFF),
        _tee([(1, 1, 0, 8, 0)], [(0, 0, 0, 2)], gap=31, p_cells=40, p=0xFFFFFFFF),
    ]
    for sc in cases:
        run_parity(sc, 30, chunk=1, state_every=1, mode=mode)


@pytest.mark.parametrize("mode", [T.STEP_FUSED, T.STEP_SPLIT])
@pytest.mark.parametrize("case", [(3, 2, 20, 300, 1, 5, None, False, 4), (4, 3, 25, 700, 2, 5, 6, True, 9),
                                  (4, 4, 40, 1200, 3, 5, 7, True, 31), (5, 2, 60, 2000, 4, 5, None, False, 12),
                                  (4, 3, 33, 600, 5, 15, 8, False, 20)])
def test_grids_with_yield_approaches_match_oracle(case, mode):
    side, lanes, cells, trips, seed, vmax, lane_seed, turns, gap = case
    sc = N.small_grid_scenario(side, lanes, cells, trips, 200, 800, gen_seed=seed, seed=seed * 3 + 5, vmax=vmax,
                               turns=turns, lane_seed=lane_seed, yield_gap=gap)
    o = run_parity(sc, 800, chunk=200, state_every=200, mode=mode)
    assert int(o["arrived"][-1]) > 0


def test_yield_with_signals_and_partial_tiles():
    sc = N.small_grid_scenario(4, 3, 45, 1500, 200, 900, gen_seed=13, seed=14, signal=(40, 20), turns=True,
                               lane_seed=15, yield_gap=6)
    run_parity(sc, 900, chunk=300, state_every=300)
    run_parity(sc, 900, chunk=300, state_every=300, tile_words=8, mode=T.STEP_FUSED)


def test_config1_with_turn_lanes_and_yield_first_window():
    sc = _with_turns(N.config1())
    sc = dataclasses.replace(sc, net=dataclasses.replace(sc.net, link_yield=N.yield_by_lanes(sc.net, 8)))
    run_parity(sc, 900, chunk=300, state_every=900)


def test_yield_state_from_the_oracle():
    sc = N.small_grid_scenario(4, 2, 30, 1500, 300, 900, gen_seed=25, seed=26, yield_gap=10)
    orc = oracle.Oracle(sc)
    orc.step(400)
    s = orc.get_state()
    init = N.InitialState(**{k: s[k] for k in ("cell_id", "cell_v", "buf_id", "buf_v", "cursor", "dep_head")},
                          step=s["step"], arrived=s["arrived"], inserted=s["inserted"])
    sim = T.Simulation(sc)
    sim.write_state(init)
    sim.step(300)
    _cmp_stats(sim.stats_range(400, 300), orc.step(300), "from the oracle state")
    _cmp_state(sim.read_state(), orc.get_state(), "after step 699")
    sim.close()


def test_malformed_yield_table_is_rejected():
    sc = _tee([(1, 1, 0, 10, 5)], [(0, 0, 0, 2)])
    T.Simulation(sc).close()
    sc.net.link_yield = np.array([32, 0, 0], np.uint8)
    with pytest.raises(T.TsError, match="INVALID"):
        T.Simulation(sc)


@pytest.mark.parametrize("rules", [None, "all"])
@pytest.mark.parametrize("mode", [T.STEP_FUSED, T.STEP_SPLIT])
def test_every_route_of_a_2x2_grid_matches_oracle(rules, mode):
    # one traveller per simple path of a 2x2 grid (24 paths), three rounds,
    # step by step; "all": turn lanes, yield approaches and signals
    from test_oracle_pins import _simple_paths
    net = N.grid_network(2, 2, 12)
    routes = _simple_paths(net) * 3
    depart = [3 * (i // 24) + i % 5 for i in range(len(routes))]
    off = np.zeros(len(routes) + 1, np.uint32)
    off[1:] = np.cumsum([len(r) for r in routes])
    dem = N.Demand(np.array(depart, np.uint32), off, np.array([x for r in routes for x in r], np.uint32))
    if rules == "all":
        net.turn_lanes = N.turn_lanes_by_rank(net)
        net.link_yield = N.grid_yield(net, 4)
        net.link_signal = N.grid_signals(net, 2, 12, 6)
    sc = N.Scenario("grid2x2-all-routes", net, dem, steps=160, seed=5, p_threshold=N.P_THRESHOLD_0_2)
    o = run_parity(sc, 160, chunk=1, state_every=1, mode=mode)
    assert int(o["arrived"][-1]) == len(routes)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("mode", [T.STEP_FUSED, T.STEP_SPLIT])
def test_random_intersection_rules_match_oracle(seed, mode):
    # arbitrary turn masks (also non-adjacent lanes), acceptance gaps and
    # signal phases on a 3x3 grid (step by step) and a 6x6 grid
    from test_oracle_pins import random_rules_scenario
    run_parity(random_rules_scenario(seed), 220, chunk=1, state_every=1, mode=mode)
    run_parity(random_rules_scenario(seed, side=6, steps=600), 600, chunk=200, state_every=200, mode=mode)


def test_load_balancing_with_intersection_rules():
    # re-tiling from the occupancy every 64 steps with a small vehicle budget
    # (many partial tiles) under turn lanes, yield approaches and signals
    sc = N.small_grid_scenario(5, 4, 70, 3500, 300, 1200, gen_seed=41, seed=42, turns=True, lane_seed=43,
                               yield_gap=9, signal=(30, 15))
    sim = T.Simulation(sc)
    sim.set_load_balance(64, 128)
    orc = oracle.Oracle(sc)
    sim.step(1200)
    _cmp_stats(sim.stats_range(0, 1200), orc.step(1200), "load balanced with rules")
    _cmp_state(sim.read_state(), orc.get_state(), "load balanced with rules, final")
    sim.close()
