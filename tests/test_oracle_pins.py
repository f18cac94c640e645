"""Pins of the CPU oracle against facts fixed outside it.

Each test ties the oracle to something it does not compute itself: published
known-answer vectors, closed forms of the 1-lane circle (Sec. 5), hand-derived
trajectories of the car-following rules (Sec. 3), conservation and exclusion
invariants, and a second naive restatement of the rules on tiny networks.
"""
import math
import os

import numpy as np
import pytest

import oracle
from brute import Brute
from helpers import check_invariants, digest, make_scenario, positions, splitmix64
from paper_cs_0105004_gb300.inputs import networks as N

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# ------------------------------------------------------------------ generators

def test_philox_known_answers():
    for r in _rows("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in r]
        assert list(oracle.philox4x32_10(v[0:4], v[4:6])) == v[6:10]


def test_splitmix64_known_answers():
    for k, r in enumerate(_rows("splitmix64_seed0.txt")):
        z = (k * 0x9E3779B97F4A7C15) % 2**64
        assert oracle.splitmix64(z) == int(r[0], 16)
        assert splitmix64(z) == int(r[0], 16)


# ------------------------------------------------------------------ hand-derived trajectories

def test_single_car_trajectory():
    sc = make_scenario([(0, 1, 200, 1)], 2, [[0]], [0], p=0)
    o = oracle.Oracle(sc)
    for step, x, v in _rows("single_car_p0.txt"):
        o.step(1)
        pos = positions(o.get_state(), sc.net)
        assert pos[0] == (0, 0, int(x), int(v)), step


def test_car_decelerates_to_link_end_and_arrives():
    # 12-cell last link: cells 0,1,3,6,10 after steps 0..4; at cell 10 the gap is
    # 1 free cell + 1 (exit open on the last link) = 2, so it reaches 12 = L and
    # leaves to parking in step 5.
    sc = make_scenario([(0, 1, 12, 1)], 2, [[0]], [0], p=0)
    o = oracle.Oracle(sc)
    st = o.step(6)
    assert [int(s["arrived"]) for s in st] == [0, 0, 0, 0, 0, 1]
    assert int(st[4]["sum_v"]) == 4 and int(st[5]["active"]) == 0


def test_transfer_keeps_velocity_and_then_arrives():
    # link 0 (0->1) then link 1 (1->2), 12 cells each.  Step 5: v = 2 reaches the
    # end of link 0, enters the empty buffer and crosses to cell 0 of link 1
    # with v = 2 in the same step.  Steps 6,7: cells 3 (v 3), 7 (v 4).  Step 8:
    # 4 free cells + exit open = 5 -> reaches 12 and arrives.
    sc = make_scenario([(0, 1, 12, 1), (1, 2, 12, 1)], 3, [[0, 1]], [0], p=0)
    o = oracle.Oracle(sc)
    o.step(6)
    assert positions(o.get_state(), sc.net)[0] == (1, 0, 0, 2)
    st = o.step(3)
    assert positions(o.get_state(), sc.net) == {}
    assert int(st[0]["transfers"]) == 0 and int(st[2]["arrived"]) == 1
    assert [int(s["sum_v"]) for s in st[:2]] == [3, 4]


def test_intersection_priority_lower_link_id_first():
    # Two one-lane links (0: 0->2, 1: 1->2) feed link 2 (2->3).  Both vehicles
    # run identical trajectories and reach their link ends in step 5; the one
    # on the lower link id takes cell 0 of link 2, the other waits in its
    # buffer and crosses one step later keeping v = 2.
    links = [(0, 2, 12, 1), (1, 2, 12, 1), (2, 3, 12, 1)]
    sc = make_scenario(links, 4, [[0, 2], [1, 2]], [0, 0], p=0)
    o = oracle.Oracle(sc)
    st = o.step(6)
    pos = positions(o.get_state(), sc.net)
    assert pos[0] == (2, 0, 0, 2) and pos[1] == (1, 0, 12, 2)
    assert int(st[5]["transfers"]) == 1 and int(st[5]["buffered"]) == 1
    o.step(1)
    pos = positions(o.get_state(), sc.net)
    assert pos[0] == (2, 0, 3, 3) and pos[1] == (2, 0, 0, 2)
    o.step(1)
    pos = positions(o.get_state(), sc.net)
    # vehicle 1: v 3 wanted, 2 free cells before vehicle 0 (at 3 after the
    # lane-change sub-step, there is one lane) -> v 2, cell 2
    assert pos[0] == (2, 0, 7, 4) and pos[1] == (2, 0, 2, 2)


def test_transfer_lane_preference():
    # Buffered vehicle on lane 1 of a 2-lane link moves to lane 1 of a 3-lane
    # next link; with that cell taken it takes the lowest free lane (0).
    links = [(0, 1, 20, 2), (1, 2, 20, 3), (3, 1, 20, 1)]
    routes = [[0, 1], [2, 1]]
    sc = make_scenario(links, 4, routes, [0, 0], p=0, bufs=[(0, 0, 1, 3)], placed=[(1, 2, 0, 5, 0)])
    o = oracle.Oracle(sc)
    o.step(1)
    assert positions(o.get_state(), sc.net)[0] == (1, 1, 0, 3)
    sc2 = make_scenario(links + [(4, 1, 20, 1)], 5, routes + [[3, 1]], [0, 0, 0], p=0,
                        bufs=[(0, 0, 1, 3), (2, 3, 0, 1)], placed=[(1, 2, 0, 5, 0)])
    # link 3 (higher id) buffered vehicle targets link 1 too, but after link 0
    o2 = oracle.Oracle(sc2)
    o2.step(1)
    pos = positions(o2.get_state(), sc2.net)
    assert pos[0] == (1, 1, 0, 3) and pos[2] == (1, 0, 0, 1)


def _lane_change_case(start_step, blocker_behind=False):
    placed = [(0, 0, 0, 10, 3), (1, 0, 0, 12, 0)]
    routes = [[0], [0]]
    if blocker_behind:
        placed.append((2, 0, 1, 7, 0))
        routes.append([0])
    return make_scenario([(0, 1, 40, 2)], 2, routes, [0] * len(routes), p=0, placed=placed,
                         start_step=start_step)


def test_lane_change_even_step_moves_up():
    # Step 0 (d=+1): vehicle 0 at lane 0 cell 10, v 3, sees 1 free cell before
    # vehicle 1; lane 1 offers 5 > 1 and its cells 5..10 are empty -> it
    # changes to lane 1, then accelerates to 4 and lands on cell 14.
    sc = _lane_change_case(0)
    o = oracle.Oracle(sc)
    st = o.step(1)
    pos = positions(o.get_state(), sc.net)
    assert pos[0] == (0, 1, 14, 4) and pos[1] == (0, 0, 13, 1)
    assert int(st[0]["lane_changes"]) == 1


def test_lane_change_odd_step_has_no_target_from_lane0():
    sc = _lane_change_case(1)
    o = oracle.Oracle(sc)
    st = o.step(1)
    pos = positions(o.get_state(), sc.net)
    assert pos[0] == (0, 0, 11, 1) and pos[1] == (0, 0, 13, 1)
    assert int(st[0]["lane_changes"]) == 0


def test_lane_change_needs_room_behind():
    sc = _lane_change_case(0, blocker_behind=True)
    o = oracle.Oracle(sc)
    st = o.step(1)
    assert int(st[0]["lane_changes"]) == 0
    assert positions(o.get_state(), sc.net)[0] == (0, 0, 11, 1)


def _near_end_case(end_state):
    # link 0: 20 cells x 2 lanes into link 1 (1 lane).  Vehicle 0 stands in
    # lane 0, cell 17 (two cells before the last), vehicle 1 stands right
    # ahead of it in cell 18; lane 1 is empty.  end_state: "open" (free
    # link-end buffers, no light), "red" (a light red for steps 0..19) or
    # "full" (both link-end buffers taken by vehicles bound for link 1)
    links = [(0, 1, 20, 2), (1, 2, 20, 1)]
    routes = [[0, 1], [0, 1]]
    bufs = None
    if end_state == "full":
        routes += [[0, 1], [0, 1]]
        bufs = [(2, 0, 0, 0), (3, 0, 1, 0)]
    sc = make_scenario(links, 3, routes, [0] * len(routes), p=0, placed=[(0, 0, 0, 17, 0), (1, 0, 0, 18, 0)],
                       bufs=bufs)
    if end_state == "red":
        sc.net.link_signal = np.array([[40, 20, 20], [0, 0, 0]], np.uint32)
    return sc


@pytest.mark.parametrize("end_state", ["open", "red", "full"])
def test_stopped_vehicle_near_the_end_changes_lane_whatever_the_end_state(end_state):
    # Step 0 (d = +1): vehicle 0 has gap 0 (vehicle 1 ahead) < min(0+1, vmax)
    # = 1, so it has a reason; in lane 1 its target cell and the 5 cells
    # behind are empty and the next cell is free, so the target gap is at
    # least 1 > 0 whether or not the link end lets anyone out: it changes
    # lanes, then accelerates to 1 (the cell ahead in lane 1 is free).
    # Vehicle 1, one cell before the last, has the last cell free ahead, so
    # gap >= 1 = min(0+1, vmax): no reason to change; it moves to cell 19.
    sc = _near_end_case(end_state)
    o = oracle.Oracle(sc)
    st = o.step(1)
    pos = positions(o.get_state(), sc.net)
    assert int(st[0]["lane_changes"]) == 1
    assert pos[0] == (0, 1, 18, 1)
    assert pos[1] == (0, 0, 19, 1)


def test_vehicle_with_vmax_free_cells_ahead_keeps_its_lane():
    # Vehicle 0 in lane 0, cell 2, v = 4, with nothing ahead for 17 cells;
    # lane 1 is empty too.  Its gap is vmax = 5 >= min(4+1, 5): no reason to
    # change, on the even step (target lane 1) as on the odd one (no target
    # from lane 0); it accelerates to 5 each step.
    for start in (0, 1):
        sc = make_scenario([(0, 1, 40, 2)], 2, [[0]], [0], p=0, placed=[(0, 0, 0, 2, 4)], start_step=start)
        o = oracle.Oracle(sc)
        st = o.step(2)
        assert int(st["lane_changes"].sum()) == 0
        assert positions(o.get_state(), sc.net)[0] == (0, 0, 12, 5)


@pytest.mark.parametrize("red", [False, True])
def test_queue_at_a_link_end_moves_only_at_its_front(red):
    # Five standing vehicles fill cells 15..19 of a 20-cell one-lane link
    # bound for link 1.  Each one behind the front has gap 0 (the cell ahead
    # is taken at the start of the step), so it keeps v = 0 and its cell; the
    # front one, in the last cell, accelerates to 1 and enters the link-end
    # buffer (then crosses to cell 0 of link 1) when the way out is open, and
    # stays when the light is red.
    n = 5
    sc = make_scenario([(0, 1, 20, 1), (1, 2, 20, 1)], 3, [[0, 1]] * n, [0] * n, p=0,
                       placed=[(i, 0, 0, 15 + i, 0) for i in range(n)])
    if red:
        sc.net.link_signal = np.array([[40, 20, 20], [0, 0, 0]], np.uint32)
    o = oracle.Oracle(sc)
    st = o.step(1)
    pos = positions(o.get_state(), sc.net)
    for i in range(n - 1):
        assert pos[i] == (0, 0, 15 + i, 0)
    assert pos[n - 1] == ((0, 0, 19, 0) if red else (1, 0, 0, 1))
    assert int(st[0]["moving"]) == (0 if red else 1)
    assert int(st[0]["transfers"]) == (0 if red else 1)


# ------------------------------------------------------------------ 1-lane circle (Sec. 5)

def _ring(L, n, mode, v0=0, lanes=1, p=0, vmax=5, seed=3, rng_seed=0):
    net = N.ring_network(L, lanes)
    dem, init = N.ring_initial_state(net, n, mode, v0, np.random.default_rng(rng_seed))
    return N.Scenario("ring", net, dem, 0, seed, vmax, p, 1, init)


def test_ring_free_flow_exact():
    # gaps >= vmax at v = vmax: every vehicle keeps vmax; flow = rho * vmax exactly
    sc = _ring(320, 32, "uniform", v0=5)
    st = oracle.Oracle(sc).step(200)
    assert np.all(st["sum_v"] == 5 * 32)
    assert np.all(st["moving"] == 32)


def test_ring_jam_exact():
    # L = N (g+1), all gaps g < vmax, v = g: stationary, sum v = L - N
    for g in (1, 2, 3, 4):
        n = 40
        sc = _ring(n * (g + 1), n, "uniform", v0=g)
        st = oracle.Oracle(sc).step(100)
        assert np.all(st["sum_v"] == n * g)
        assert np.all(st["moving"] == n)


def test_megajam_dissolves_one_car_per_step():
    # p = 0, N cars packed at v = 0: only the front car has room in step 0;
    # each step the car behind the last moving one finds a free cell and
    # starts, and no car that moves ever stops again while the leader has
    # not lapped the ring: moving(t) = min(t + 1, N)
    n = 40
    sc = _ring(640, n, "megajam")
    st = oracle.Oracle(sc).step(100)
    assert st["moving"].tolist() == [min(t + 1, n) for t in range(100)]


def test_moving_count_is_bounded_by_speeds_and_matches_the_state():
    # every moving vehicle has 1 <= v <= vmax, standing ones v = 0:
    # moving <= sum_v <= vmax * moving, moving <= active, and the count
    # equals the vehicles in cells with v > 0 in the state after the step
    sc = N.small_grid_scenario(4, 2, 25, n_trips=600, window=200, steps=400, gen_seed=4, seed=9)
    o = oracle.Oracle(sc)
    peak = 0
    for _ in range(8):
        st = o.step(50)
        peak = max(peak, int(st["moving"].max()))
        mv, sv, act = (st[f].astype(np.int64) for f in ("moving", "sum_v", "active"))
        assert np.all(mv <= act) and np.all(mv <= sv) and np.all(sv <= sc.vmax * mv)
        s = o.get_state()
        assert int(st["moving"][-1]) == int(((s["cell_id"] >= 0) & (s["cell_v"] > 0)).sum())
    assert peak > 0


@pytest.mark.parametrize("rho", [0.15, 0.2, 0.3])
def test_three_lane_circle_flow_per_lane_at_least_one_lane_flow(rho):
    # Sec. 5, the 3-lane circle: with lane changes a fast vehicle passes a
    # slow one, so at the same density per lane the flow per lane of the
    # 3-lane circle is at least the 1-lane flow (p = 0.2; measured margin
    # 2-3 %, asserted 1 %); 1,000 steps of warm-up, 5,000 averaged
    L = 1024
    flow = []
    for lanes in (1, 3):
        n = int(round(rho * L * lanes))
        o = oracle.Oracle(_ring(L, n, "random", lanes=lanes, p=N.P_THRESHOLD_0_2, rng_seed=11))
        o.step(1000)
        st = o.step(5000)
        assert int(st["lane_changes"].sum()) > 0 or lanes == 1
        flow.append(st["sum_v"].astype(np.float64).mean() / (L * lanes))
    assert flow[1] >= 1.01 * flow[0], flow


@pytest.mark.parametrize("rho", [0.05, 0.1, 0.3, 0.5, 0.8])
def test_ring_deterministic_fundamental_diagram(rho):
    # p = 0: J = min(rho vmax, 1 - rho) after transients (NaSch deterministic limit)
    L = 640
    n = int(round(rho * L))
    sc = _ring(L, n, "random", rng_seed=int(rho * 1000))
    o = oracle.Oracle(sc)
    o.step(10 * L)
    st = o.step(2 * L)
    J = st["sum_v"].astype(np.float64).mean() / L
    Jth = min(n / L * 5, 1 - n / L)
    assert abs(J - Jth) <= 2.0 / L + 1e-9


@pytest.mark.parametrize("rho", [0.1, 0.3, 0.5, 0.7])
def test_ring_vmax1_stochastic_exact_flow(rho):
    # vmax = 1 with parallel update: J = (1 - sqrt(1 - 4 (1-p) rho (1-rho))) / 2
    # (Schreckenberg, Schadschneider, Nagel, Ito, Phys. Rev. E 51, 1995)
    L = 9984
    n = int(round(rho * L))
    thr = N.P_THRESHOLD_0_2
    sc = _ring(L, n, "random", vmax=1, p=thr, rng_seed=7)
    o = oracle.Oracle(sc)
    o.step(500)
    st = o.step(3000)
    J = st["sum_v"].astype(np.float64).mean() / L
    q = 1 - thr / 2**32
    r = n / L
    Jth = (1 - math.sqrt(1 - 4 * q * r * (1 - r))) / 2
    assert abs(J - Jth) / Jth < 0.01


def test_three_lane_ring_lane_changes_alternate_and_conserve():
    sc = _ring(320, 300, "random", lanes=3, p=N.P_THRESHOLD_0_2, rng_seed=5)
    o = oracle.Oracle(sc)
    prev = positions(o.get_state(), sc.net)
    total_lc = 0
    for t in range(200):
        st = o.step(1)[0]
        s = o.get_state()
        pos = positions(s, sc.net)
        assert len(pos) == 300 and int(st["active"]) == 300
        d = 1 if t % 2 == 0 else -1
        for i, p in pos.items():
            assert p[1] - prev[i][1] in (0, d)
        total_lc += int(st["lane_changes"])
        assert int(st["lane_changes"]) == sum(1 for i in pos if pos[i][1] != prev[i][1])
        prev = pos
    assert total_lc > 0


# ------------------------------------------------------------------ invariants and the naive restatement

def test_invariants_on_grid():
    sc = N.small_grid_scenario(4, 2, 25, n_trips=400, window=100, steps=400, gen_seed=5, seed=9)
    o = oracle.Oracle(sc)
    prev = None
    for t in range(400):
        row = o.step(1)[0]
        s = o.get_state()
        prev = check_invariants(sc, s, row, prev)
        assert int(row["state_hash"]) == digest(s, sc.net)
    assert int(row["arrived"]) > 0


@pytest.mark.parametrize("case", [(3, 2, 20, 60, 0, 5, 1), (3, 3, 12, 150, 1, 5, 1), (2, 1, 8, 40, 2, 3, 1),
                                  (3, 2, 15, 200, 3, 7, 1), (3, 2, 15, 120, 4, 5, 0)])
def test_oracle_matches_naive_restatement(case):
    side, lanes, cells, trips, seed, vmax, lc = case
    sc = N.small_grid_scenario(side, lanes, cells, trips, 60, 250, gen_seed=seed, seed=seed + 11, vmax=vmax)
    sc.lane_change = lc
    o, b = oracle.Oracle(sc), Brute(sc)
    for t in range(250):
        so = o.step(1)[0]
        sb = b.step()
        for k, v in sb.items():
            assert int(so[k]) == v, (t, k)
        st = o.get_state()
        ci, cv, bi, bv = b.state(sc.net)
        assert np.array_equal(st["cell_id"], ci) and np.array_equal(st["cell_v"], cv)
        assert np.array_equal(st["buf_id"], bi) and np.array_equal(st["buf_v"], bv)


def test_oracle_matches_naive_restatement_on_rings():
    for lanes in (1, 2, 3):
        sc = _ring(96, 40 * lanes, "random", lanes=lanes, p=N.P_THRESHOLD_0_2, rng_seed=lanes)
        o, b = oracle.Oracle(sc), Brute(sc)
        for t in range(150):
            so = o.step(1)[0]
            sb = b.step()
            assert int(so["sum_v"]) == sb["sum_v"] and int(so["lane_changes"]) == sb["lane_changes"]
            ci, cv, _, _ = b.state(sc.net)
            st = o.get_state()
            assert np.array_equal(st["cell_id"], ci) and np.array_equal(st["cell_v"], cv)


# ------------------------------------------------------------------ link travel times

def test_link_travel_times_by_hand():
    # The two-link trip of the transfer test: it enters link 0 at the end of
    # step 0 (departure), crosses to link 1 at the end of step 5 and arrives
    # in step 8: link 0 took 5 steps, link 1 took 3.
    sc = make_scenario([(0, 1, 12, 1), (1, 2, 12, 1)], 3, [[0, 1]], [0], p=0)
    o = oracle.Oracle(sc)
    o.step(10)
    tsum, tcnt = o.link_times()
    assert tsum.tolist() == [5, 3] and tcnt.tolist() == [1, 1]
    # one 12-cell link: cells 0,1,3,6,10 after steps 0..4, arrival in step 5
    sc = make_scenario([(0, 1, 12, 1)], 2, [[0]], [0], p=0)
    o = oracle.Oracle(sc)
    o.step(6)
    assert [int(x) for x in o.link_times()[0]] == [5]


def test_link_travel_time_counts_equal_transfers_plus_arrivals():
    sc = N.small_grid_scenario(4, 2, 25, n_trips=400, window=200, steps=900, gen_seed=3, seed=5)
    o = oracle.Oracle(sc)
    st = o.step(900)
    tsum, tcnt = o.link_times()
    assert int(tcnt.sum()) == int(st["transfers"].sum()) + int(st["arrived"][-1])
    # a traversal lasts at least one step, and the first link of a trip is
    # entered only at its departure step or later
    assert np.all(tsum >= tcnt)
    assert int(tcnt.sum()) > 0


# ------------------------------------------------------------------ traffic signals

def test_car_waits_at_a_red_light_by_hand():
    # Link 0 (20 cells) ends at a light red for steps 0..19 (cycle 40, green
    # 20, offset 20: green iff (t + 20) mod 40 < 20).  Cells 1,3,6,10,15
    # after steps 1..5; in step 6 the virtual vehicle at the end leaves a gap
    # of 4 cells, so v = 4 and the car stops in cell 19; it stays there with
    # v = 0 until step 20, when the light is green: v = 1 takes it into the
    # empty buffer and across to cell 0 of link 1, keeping v = 1.
    sc = make_scenario([(0, 1, 20, 1), (1, 2, 20, 1)], 3, [[0, 1]], [0], p=0)
    sc.net.link_signal = np.array([[40, 20, 20], [0, 0, 0]], np.uint32)
    o = oracle.Oracle(sc)
    seen = []
    for _ in range(21):
        o.step(1)
        seen.append(positions(o.get_state(), sc.net)[0])
    assert seen[5] == (0, 0, 15, 5)
    assert seen[6] == (0, 0, 19, 4)
    assert all(p == (0, 0, 19, 0) for p in seen[7:20])
    assert seen[20] == (1, 0, 0, 1)
    assert o.link_times()[0].tolist() == [20, 0]


def test_no_vehicle_reaches_a_red_lane_end():
    sc = N.small_grid_scenario(4, 2, 20, n_trips=500, window=200, steps=600, gen_seed=2, seed=3, signal=(30, 15))
    sig = sc.net.link_signal
    o = oracle.Oracle(sc)
    before = o.get_state()["buf_id"]
    lb = sc.net.lane_base()
    arrived = 0
    for t in range(600):
        st = o.step(1)
        after = o.get_state()["buf_id"]
        red = (t + sig[:, 2]) % sig[:, 0] >= sig[:, 1]
        for l in np.nonzero(red)[0]:
            for ln in range(lb[l], lb[l + 1]):
                # a buffer of a red link can only keep or lose its vehicle
                assert after[ln] == -1 or after[ln] == before[ln], (t, l)
        before = after
        arrived = int(st["arrived"][0])
    assert arrived > 0


# ------------------------------------------------------------------ plan-following lane changes

def _fork(placed, routes, lane_change=1, start_step=0, turns=(0b01, 0b10)):
    # link 0 (2 lanes, 20 cells) ends at node 1, which links 1 and 2 leave;
    # the turn onto link 1 is taken from lane 0 only, onto link 2 from lane 1
    sc = make_scenario([(0, 1, 20, 2), (1, 2, 10, 1), (1, 3, 10, 1)], 4, routes, [0] * len(routes), p=0,
                       lane_change=lane_change, placed=placed, start_step=start_step)
    if turns is not None:
        sc.net.turn_lanes = np.array(turns, np.uint8)
    return sc


def test_turn_table_generator_covers_every_turn_and_lane():
    net = N.small_grid_scenario(4, 4, 20, lane_seed=5, turns=True).net
    off = N.turn_table_offsets(net)
    for l in range(net.n_links):
        masks = net.turn_lanes[off[l]:off[l + 1]].astype(int)
        assert len(masks) == int((net.link_from == net.link_to[l]).sum())
        full = (1 << int(net.link_lanes[l])) - 1
        assert all(0 < m <= full for m in masks)
        assert np.bitwise_or.reduce(masks) == full
    # three lanes, three turns: one lane each, in order
    assert N.turn_lanes_by_rank(N.Network(4, np.array([0, 1, 1, 1], np.uint32), np.array([1, 2, 3, 0], np.uint32),
                                          np.full(4, 10, np.uint32), np.array([3, 1, 1, 1], np.uint32),
                                          np.zeros(4, np.uint8)))[:3].tolist() == [1, 2, 4]


def test_wrong_lane_changes_towards_its_turn_on_the_next_odd_step():
    # vehicle 0 in lane 1 must take the turn onto link 1 (lane 0 only).  Step
    # 0 points to lane 2, which does not exist: it only drives (v 1, cell 1).
    # Step 1 points to lane 0: it changes there and accelerates to cell 3.
    sc = _fork([(0, 0, 1, 0, 0)], [[0, 1]])
    o = oracle.Oracle(sc)
    st = o.step(2)
    assert positions(o.get_state(), sc.net)[0] == (0, 0, 3, 2)
    assert [int(s["lane_changes"]) for s in st] == [0, 1]
    # without a turn table there is no reason to change
    sc = _fork([(0, 0, 1, 0, 0)], [[0, 1]], turns=None)
    o = oracle.Oracle(sc)
    assert [int(s["lane_changes"]) for s in o.step(2)] == [0, 0]


def test_accepted_gap_shrinks_near_the_intersection():
    # vehicle 0 (wrong lane 1) with vehicle 1 stopped two cells behind it in
    # lane 0, at step 1 (d = -1).  Far from the link end the change needs the
    # 5 cells behind the target cell empty: no change.  On cell 18 (one cell
    # before the last) it needs only one: it changes.
    far = _fork([(0, 0, 1, 10, 0), (1, 0, 0, 8, 0)], [[0, 1], [0, 1]], start_step=1)
    o = oracle.Oracle(far)
    assert int(o.step(1)[0]["lane_changes"]) == 0
    near = _fork([(0, 0, 1, 18, 0), (1, 0, 0, 16, 0)], [[0, 1], [0, 1]], start_step=1)
    o = oracle.Oracle(near)
    assert int(o.step(1)[0]["lane_changes"]) == 1
    assert positions(o.get_state(), near.net)[0][:2] == (0, 0)
    # in the last cell it needs only the target cell: a vehicle right behind
    # that cell does not stop it, one in it does
    last = _fork([(0, 0, 1, 19, 0), (1, 0, 0, 18, 0)], [[0, 1], [0, 1]], start_step=1)
    o = oracle.Oracle(last)
    assert int(o.step(1)[0]["lane_changes"]) == 1
    taken = _fork([(0, 0, 1, 19, 0), (1, 0, 0, 19, 0)], [[0, 1], [0, 1]], start_step=1)
    o = oracle.Oracle(taken)
    assert int(o.step(1)[0]["lane_changes"]) == 0


def test_wrong_lane_stops_at_the_link_end():
    # lane changes off: vehicle 0 in lane 1 needs lane 0 for its turn.  It
    # runs cells 1,3,6,10,15 and stops in the last cell (19) with v 4 then 0,
    # never entering the buffer; the same vehicle heading for link 2 (lane 1
    # allowed) crosses.
    sc = _fork([(0, 0, 1, 0, 0)], [[0, 1]], lane_change=0)
    o = oracle.Oracle(sc)
    seen = []
    for _ in range(12):
        o.step(1)
        seen.append(positions(o.get_state(), sc.net)[0])
    assert seen[4] == (0, 1, 15, 5) and seen[5] == (0, 1, 19, 4)
    assert all(p == (0, 1, 19, 0) for p in seen[6:])
    sc = _fork([(0, 0, 1, 0, 0)], [[0, 2]], lane_change=0)
    o = oracle.Oracle(sc)
    o.step(6)
    assert positions(o.get_state(), sc.net)[0] == (2, 0, 0, 5)


def test_speed_change_only_into_an_allowed_lane():
    # vehicle 0 (lane 0, v 3) closes on vehicle 1 stopped two cells ahead at
    # step 0 (d = +1).  Without a table it overtakes by changing to lane 1; when
    # its turn allows lane 0 only, it stays behind.
    placed = [(0, 0, 0, 5, 3), (1, 0, 0, 7, 0)]
    o = oracle.Oracle(_fork(placed, [[0, 1], [0, 1]], turns=None))
    assert int(o.step(1)[0]["lane_changes"]) == 1
    sc = _fork(placed, [[0, 1], [0, 1]])
    o = oracle.Oracle(sc)
    assert int(o.step(1)[0]["lane_changes"]) == 0
    assert positions(o.get_state(), sc.net)[0] == (0, 0, 6, 1)


def test_every_lane_allowed_equals_no_table():
    sc = N.small_grid_scenario(4, 3, 20, n_trips=500, window=200, steps=500, gen_seed=7, seed=8, lane_seed=3)
    a = oracle.Oracle(sc).step(500)
    off = N.turn_table_offsets(sc.net)
    full = np.repeat((1 << sc.net.link_lanes.astype(np.int64)) - 1, np.diff(off)).astype(np.uint8)
    sc.net.turn_lanes = full
    b = oracle.Oracle(sc).step(500)
    assert np.array_equal(a, b)


def test_vehicles_leave_links_only_from_allowed_lanes():
    sc = N.small_grid_scenario(4, 4, 20, n_trips=600, window=200, steps=700, gen_seed=9, seed=10, lane_seed=4,
                               turns=True)
    net, dem = sc.net, sc.demand
    off = N.turn_table_offsets(net)
    outs = {n: sorted(np.nonzero(net.link_from == n)[0].tolist()) for n in range(net.n_nodes)}
    lb = net.lane_base()
    lane_link = np.repeat(np.arange(net.n_links), net.link_lanes.astype(np.int64))
    o = oracle.Oracle(sc)
    prev = None
    for _ in range(700):
        row = o.step(1)[0]
        s = o.get_state()
        prev = check_invariants(sc, s, row, prev)
        for ln in np.nonzero(s["buf_id"] >= 0)[0]:
            i = int(s["buf_id"][ln])
            l = int(lane_link[ln])
            m = int(dem.route_links[dem.route_offsets[i] + s["cursor"][i] + 1])
            mask = int(net.turn_lanes[off[l] + outs[int(net.link_to[l])].index(m)])
            assert mask >> (ln - lb[l]) & 1, (int(row["step"]), i)
    assert int(row["arrived"]) > 300 and int(o.step(1)[0]["lane_changes"]) >= 0


@pytest.mark.parametrize("case", [(3, 2, 15, 120, 0, 5, None), (3, 3, 12, 150, 1, 5, 2), (3, 4, 15, 200, 2, 7, 3),
                                  (2, 4, 10, 60, 3, 3, 4)])
def test_plan_following_matches_naive_restatement(case):
    side, lanes, cells, trips, seed, vmax, lane_seed = case
    sc = N.small_grid_scenario(side, lanes, cells, trips, 60, 250, gen_seed=seed, seed=seed + 21, vmax=vmax,
                               turns=True, lane_seed=lane_seed)
    o, b = oracle.Oracle(sc), Brute(sc)
    changes = 0
    for t in range(250):
        so = o.step(1)[0]
        sb = b.step()
        for k, v in sb.items():
            assert int(so[k]) == v, (t, k)
        changes += sb["lane_changes"]
        st = o.get_state()
        ci, cv, bi, bv = b.state(sc.net)
        assert np.array_equal(st["cell_id"], ci) and np.array_equal(st["cell_v"], cv)
        assert np.array_equal(st["buf_id"], bi) and np.array_equal(st["buf_v"], bv)
    assert changes > 0


# ------------------------------------------------------------------ gap acceptance at unprotected turns

def _tee(placed, bufs, gap=5, p_cells=20, p=0):
    # node 1: link 0 from node 2 (a yield approach with acceptance gap `gap`)
    # and link 1 from node 0 (priority) both lead to link 2 (one lane)
    sc = make_scenario([(2, 1, 20, 1), (0, 1, p_cells, 1), (1, 3, 20, 1)], 4, [[0, 2], [1, 2]], [0, 0], p=p,
                       placed=placed, bufs=bufs)
    if gap is not None:
        sc.net.link_yield = np.array([gap, 0, 0], np.uint8)
    return sc


def test_yield_waits_for_the_gap_on_the_priority_street_by_hand():
    # vehicle 0 waits in link 0's buffer (v 2).  Vehicle 1 drives link 1 at
    # v 5 from cell 10: after step 0 it is in cell 15, inside the last 5
    # cells, so vehicle 0 may not go; in step 1 it reaches the end and, from
    # the priority approach, takes link 2's cell 0 first; in step 2 it moves
    # on to cell 5 and vehicle 0 crosses into cell 0.
    sc = _tee([(1, 1, 0, 10, 5)], [(0, 0, 0, 2)])
    o = oracle.Oracle(sc)
    seen = []
    for _ in range(3):
        o.step(1)
        seen.append(positions(o.get_state(), sc.net))
    assert seen[0][0] == (0, 0, 20, 2) and seen[0][1] == (1, 0, 15, 5)
    assert seen[1][0] == (0, 0, 20, 2) and seen[1][1] == (2, 0, 0, 5)
    assert seen[2][0] == (2, 0, 0, 2) and seen[2][1] == (2, 0, 5, 5)
    # without gap acceptance the lower link id goes first, in step 0
    sc = _tee([(1, 1, 0, 10, 5)], [(0, 0, 0, 2)], gap=None)
    o = oracle.Oracle(sc)
    o.step(1)
    assert positions(o.get_state(), sc.net)[0] == (2, 0, 0, 2)


def test_yield_crosses_when_the_priority_vehicle_is_far():
    # vehicle 1 starts at cell 5 with v 0 and is in cell 6 after step 0: the
    # last 5 cells of link 1 are empty and vehicle 0 crosses at once
    sc = _tee([(1, 1, 0, 5, 0)], [(0, 0, 0, 2)])
    o = oracle.Oracle(sc)
    o.step(1)
    pos = positions(o.get_state(), sc.net)
    assert pos[0] == (2, 0, 0, 2) and pos[1] == (1, 0, 6, 1)


def test_yield_gap_never_counts_cell_zero():
    # every draw slows a vehicle down (threshold 2^32 - 1), so vehicle 1 never
    # leaves its cell.  With a 4-cell priority link and a gap of 31 only cells
    # 1..3 count: vehicle 1 in cell 0 does not hold vehicle 0 back, in cell 1
    # it does.
    sc = _tee([(1, 1, 0, 0, 0)], [(0, 0, 0, 2)], gap=31, p_cells=4, p=0xFFFFFFFF)
    o = oracle.Oracle(sc)
    o.step(1)
    pos = positions(o.get_state(), sc.net)
    assert pos[0] == (2, 0, 0, 2) and pos[1] == (1, 0, 0, 0)
    sc = _tee([(1, 1, 0, 1, 0)], [(0, 0, 0, 2)], gap=31, p_cells=4, p=0xFFFFFFFF)
    o = oracle.Oracle(sc)
    o.step(3)
    pos = positions(o.get_state(), sc.net)
    assert pos[0] == (0, 0, 20, 2) and pos[1] == (1, 0, 1, 0)


def test_generated_yield_tables():
    net = N.grid_network(4, 2, 20)
    g = N.grid_yield(net, 7)
    horizontal = np.abs(net.link_from.astype(int) - net.link_to.astype(int)) == 1
    assert set(g[horizontal].tolist()) == {0} and set(g[~horizontal].tolist()) == {7}
    net = N.small_grid_scenario(4, 3, 20, lane_seed=2).net
    y = N.yield_by_lanes(net, 4)
    for n in range(net.n_nodes):
        inc = np.nonzero(net.link_to == n)[0]
        wide = net.link_lanes[inc].max()
        assert all((y[l] == 4) == (net.link_lanes[l] < wide) for l in inc)


@pytest.mark.parametrize("case", [(3, 2, 15, 200, 0, 5, None, False, None), (3, 3, 12, 200, 1, 5, 2, True, None),
                                  (3, 2, 15, 250, 2, 7, None, False, (20, 10)), (2, 4, 10, 80, 3, 3, 4, True, None)])
def test_gap_acceptance_matches_naive_restatement(case):
    side, lanes, cells, trips, seed, vmax, lane_seed, turns, signal = case
    sc = N.small_grid_scenario(side, lanes, cells, trips, 60, 250, gen_seed=seed, seed=seed + 31, vmax=vmax,
                               turns=turns, lane_seed=lane_seed, signal=signal, yield_gap=3 + seed)
    o, b = oracle.Oracle(sc), Brute(sc)
    for t in range(250):
        so = o.step(1)[0]
        sb = b.step()
        for k, v in sb.items():
            assert int(so[k]) == v, (t, k)
        st = o.get_state()
        ci, cv, bi, bv = b.state(sc.net)
        assert np.array_equal(st["cell_id"], ci) and np.array_equal(st["cell_v"], cv)
        assert np.array_equal(st["buf_id"], bi) and np.array_equal(st["buf_v"], bv)
    assert int(so["arrived"]) > 0


def test_signals_by_rank_alternate_at_every_node():
    net = N.planar_network(300, 400, 4)
    sig = N.signals_by_rank(net, 60, 30)
    for n in range(net.n_nodes):
        inc = sorted(np.nonzero(net.link_to == n)[0].tolist())
        if len(inc) < 2:
            assert all(sig[l, 0] == 0 for l in inc)
            continue
        for r, l in enumerate(inc):
            assert sig[l].tolist() == [60, 30, 0 if r % 2 == 0 else 30]
        # at every step the green approaches all have the same rank parity
        for t in range(60):
            green = [r % 2 for r, l in enumerate(inc) if (t + sig[l, 2]) % 60 < 30]
            assert len(set(green)) == 1


def _simple_paths(net):
    """Every simple path (no node twice) of the network, as link lists."""
    out_links = {}
    for l in range(net.n_links):
        out_links.setdefault(int(net.link_from[l]), []).append(l)
    paths = []

    def grow(path, seen):
        paths.append(list(path))
        for l in out_links.get(int(net.link_to[path[-1]]), []):
            if int(net.link_to[l]) not in seen:
                grow(path + [l], seen | {int(net.link_to[l])})

    for l in range(net.n_links):
        grow([l], {int(net.link_from[l]), int(net.link_to[l])})
    return paths


@pytest.mark.parametrize("rules", [None, "turns", "yield", "all"])
def test_every_route_of_a_2x2_grid_matches_naive_restatement(rules):
    # 4 nodes, 8 links of 2 lanes x 12 cells: one traveller per simple path
    # (all 24 of them, 1 to 3 links), three rounds of departures
    net = N.grid_network(2, 2, 12)
    paths = _simple_paths(net)
    assert len(paths) == 24
    routes = paths * 3
    depart = [3 * (i // len(paths)) + i % 5 for i in range(len(routes))]
    off = np.zeros(len(routes) + 1, np.uint32)
    off[1:] = np.cumsum([len(r) for r in routes])
    dem = N.Demand(np.array(depart, np.uint32), off, np.array([x for r in routes for x in r], np.uint32))
    if rules in ("turns", "all"):
        net.turn_lanes = N.turn_lanes_by_rank(net)
    if rules in ("yield", "all"):
        net.link_yield = N.grid_yield(net, 4)
    if rules == "all":
        net.link_signal = N.grid_signals(net, 2, 12, 6)
    sc = N.Scenario("grid2x2-all-routes", net, dem, steps=160, seed=5, p_threshold=N.P_THRESHOLD_0_2)
    o, b = oracle.Oracle(sc), Brute(sc)
    for t in range(160):
        so = o.step(1)[0]
        sb = b.step()
        for k, v in sb.items():
            assert int(so[k]) == v, (t, k)
        st = o.get_state()
        ci, cv, bi, bv = b.state(sc.net)
        assert np.array_equal(st["cell_id"], ci) and np.array_equal(st["cell_v"], cv)
        assert np.array_equal(st["buf_id"], bi) and np.array_equal(st["buf_v"], bv)
    assert int(so["arrived"]) == len(routes)


def random_rules_scenario(seed, side=3, steps=220):
    """A grid with arbitrary (not rank-structured) turn masks, random
    acceptance gaps (0..31), random signal cycles and offsets and lanes 1..4
    per edge, all drawn from `seed`."""
    rng = np.random.default_rng(100 + seed)
    sc = N.small_grid_scenario(side, 4, int(rng.integers(8, 25)), int(rng.integers(80, 260)) * (side - 2) ** 2,
                               60, steps, gen_seed=seed + 50, seed=seed + 60, vmax=int(rng.integers(1, 9)),
                               lane_seed=seed + 70)
    net = sc.net
    off = N.turn_table_offsets(net)
    masks = np.zeros(int(off[-1]), np.uint8)
    for l in range(net.n_links):
        full = (1 << int(net.link_lanes[l])) - 1
        masks[off[l]:off[l + 1]] = rng.integers(1, full + 1, int(off[l + 1] - off[l]))
    net.turn_lanes = masks
    net.link_yield = np.where(rng.random(net.n_links) < 0.4, rng.integers(1, 32, net.n_links), 0).astype(np.uint8)
    cycle = rng.integers(0, 40, net.n_links)
    cycle[cycle < 4] = 0
    green = np.where(cycle > 0, rng.integers(1, np.maximum(cycle, 2)), 0)
    offset = np.where(cycle > 0, rng.integers(0, np.maximum(cycle, 1)), 0)
    net.link_signal = np.stack([cycle, green, offset], 1).astype(np.uint32)
    return sc


@pytest.mark.parametrize("seed", range(6))
def test_random_intersection_rules_match_naive_restatement(seed):
    sc = random_rules_scenario(seed)
    o, b = oracle.Oracle(sc), Brute(sc)
    for t in range(220):
        so = o.step(1)[0]
        sb = b.step()
        for k, v in sb.items():
            assert int(so[k]) == v, (t, k)
        st = o.get_state()
        ci, cv, bi, bv = b.state(sc.net)
        assert np.array_equal(st["cell_id"], ci) and np.array_equal(st["cell_v"], cv)
        assert np.array_equal(st["buf_id"], bi) and np.array_equal(st["buf_v"], bv)
