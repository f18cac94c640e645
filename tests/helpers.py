"""Test-only helpers: hand-built scenarios, invariant checks, digest recomputation."""
from __future__ import annotations

import numpy as np

from paper_cs_0105004_gb300.inputs.networks import (NO_NODE, Demand, InitialState, Network, Scenario)

M64 = (1 << 64) - 1


def splitmix64(z: int) -> int:
    """The splitmix64 output function (Steele, Lea, Flood 2014)."""
    z = (z + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def vehicle_term(i, link, lane, cell, v) -> int:
    a = (i << 32) | link
    b = (cell << 16) | (lane << 8) | v
    return splitmix64(a ^ splitmix64(b))


def make_scenario(links, n_nodes, routes, depart, steps=50, seed=1, vmax=5, p=0, lane_change=1,
                  placed=None, bufs=None, start_step=0, name="hand"):
    """links: list of (from, to, cells, lanes[, ring]).  routes: list of link lists.
    placed: list of (id, link, lane, cell, v) put on the network at start;
    bufs: list of (id, link, lane, v) put into link-end buffers.  Placed and
    buffered vehicles count as already departed (their cursor is the index of
    their link in their route)."""
    lf = np.array([l[0] if len(l) < 5 or not l[4] else NO_NODE for l in links], np.uint32)
    lt = np.array([l[1] if len(l) < 5 or not l[4] else NO_NODE for l in links], np.uint32)
    net = Network(n_nodes, lf, lt, np.array([l[2] for l in links], np.uint32),
                  np.array([l[3] for l in links], np.uint32),
                  np.array([1 if len(l) >= 5 and l[4] else 0 for l in links], np.uint8))
    off = np.zeros(len(routes) + 1, np.uint32)
    off[1:] = np.cumsum([len(r) for r in routes])
    dem = Demand(np.array(depart, np.uint32), off, np.array([x for r in routes for x in r], np.uint32))
    init = None
    if placed or bufs:
        lb, cb = net.lane_base(), net.lane_cell_base()
        cid = np.full(net.n_lane_cells, -1, np.int32)
        cv = np.zeros(net.n_lane_cells, np.int8)
        bid = np.full(net.n_lanes, -1, np.int32)
        bv = np.zeros(net.n_lanes, np.int8)
        cursor = np.zeros(len(routes), np.uint32)
        on = set()
        for (i, l, k, x, v) in placed or []:
            cid[cb[lb[l] + k] + x] = i; cv[cb[lb[l] + k] + x] = v
            cursor[i] = routes[i].index(l); on.add(i)
        for (i, l, k, v) in bufs or []:
            bid[lb[l] + k] = i; bv[lb[l] + k] = v
            cursor[i] = routes[i].index(l); on.add(i)
        # vehicles already on the network must sit at the head of their first
        # link's departure queue (ordered by departure step, then id)
        dep_head = np.zeros(net.n_links, np.uint32)
        order = sorted(range(len(routes)), key=lambda i: (depart[i], i))
        for l in range(net.n_links):
            q = [i for i in order if routes[i][0] == l]
            h = 0
            while h < len(q) and q[h] in on:
                h += 1
            assert all(i not in on for i in q[h:]), "placed vehicles must lead their queue"
            dep_head[l] = h
        init = InitialState(cid, cv, bid, bv, cursor, dep_head, start_step, 0, len(on))
    return Scenario(name, net, dem, steps, seed, vmax, p, lane_change, init)


def positions(state, net):
    """{id: (link, lane, cell, v)}; buffered vehicles get cell = link length."""
    lb, cb = net.lane_base(), net.lane_cell_base()
    lane_link = np.repeat(np.arange(net.n_links), net.link_lanes.astype(np.int64))
    lane_k = np.arange(net.n_lanes) - lb[lane_link]
    cid = state["cell_id"]
    occ = np.nonzero(cid >= 0)[0]
    lane_of = np.searchsorted(cb, occ, side="right") - 1
    out = {}
    for c, ln in zip(occ, lane_of):
        out[int(cid[c])] = (int(lane_link[ln]), int(lane_k[ln]), int(c - cb[ln]), int(state["cell_v"][c]))
    for ln in np.nonzero(state["buf_id"] >= 0)[0]:
        l = int(lane_link[ln])
        out[int(state["buf_id"][ln])] = (l, int(lane_k[ln]), int(net.link_cells[l]), int(state["buf_v"][ln]))
    return out


def digest(state, net) -> int:
    h = 0
    for i, (l, k, x, v) in positions(state, net).items():
        h = (h + vehicle_term(i, l, k, x, v)) & M64
    return h


def check_invariants(sc, state, stats_row, prev_pos=None, prev_step_parity=None):
    """Invariants that hold after every step: at most one vehicle per cell and
    each vehicle in at most one place; 0 <= v <= vmax; every vehicle sits on
    the link its route cursor names; conservation of travellers; and, against
    the previous state, lane changes only to the adjacent lane in the step's
    direction and no overtaking within a lane."""
    net, dem = sc.net, sc.demand
    cid = state["cell_id"]
    ids = np.concatenate([cid[cid >= 0], state["buf_id"][state["buf_id"] >= 0]])
    assert np.unique(ids).size == ids.size, "vehicle in two places"
    pos = positions(state, net)
    assert all(0 <= p[3] <= sc.vmax for p in pos.values()), "velocity out of range"
    off = dem.route_offsets
    for i, (l, k, x, v) in pos.items():
        assert dem.route_links[off[i] + state["cursor"][i]] == l, "vehicle off its route"
    t = int(stats_row["step"])
    departed = int((dem.depart_step <= t).sum())
    on = int(stats_row["active"]) + int(stats_row["buffered"])
    assert on == len(pos)
    assert int(stats_row["waiting"]) + on + int(stats_row["arrived"]) == departed, "conservation"
    if prev_pos is not None:
        d = 1 if t % 2 == 0 else -1
        by_lane = {}
        for i, (l, k, x, v) in pos.items():
            if i in prev_pos and prev_pos[i][0] == l:
                pk = prev_pos[i][1]
                assert k == pk or (k == pk + d and sc.lane_change), "illegal lane change"
                if k == pk and not net.link_ring[l]:
                    by_lane.setdefault((l, k), []).append((prev_pos[i][2], x, i))
        for lst in by_lane.values():
            lst.sort()
            news = [b for a, b, _ in lst]
            assert all(news[j] < news[j + 1] for j in range(len(news) - 1)), "overtaking within a lane"
    return pos

