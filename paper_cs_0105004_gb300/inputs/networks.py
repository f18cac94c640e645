"""Seeded generators for networks, trips, routes and ring initial states.

Layout conventions shared by every consumer:

* Links are directed.  ``link_from``/``link_to`` are node ids; a periodic
  ring link (the circle roads of Sec. 5) has no nodes and stores
  ``NO_NODE`` in both.
* A lane is (link, lane index k), k = 0 .. lanes-1.  The canonical lane order
  is link-major, then k; the canonical lane-cell order is lane order, then
  cell x = 0 .. cells-1.  Cells are 7.5 m long (Sec. 3).
* A trip's route is the list of links it drives, first link first.

Nothing here evaluates the driving rules.
"""
from __future__ import annotations

import ctypes
import dataclasses
import hashlib
import os
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

NO_NODE = 0xFFFFFFFF
CELL_M = 7.5
# Random slowdown probability 0.2 as a 32-bit threshold: floor(0.2 * 2**32).
P_THRESHOLD_0_2 = 858993459


@dataclass
class Network:
    n_nodes: int
    link_from: np.ndarray
    link_to: np.ndarray
    link_cells: np.ndarray
    link_lanes: np.ndarray
    link_ring: np.ndarray
    # traffic signal at each link's end, [n_links, 3] uint32 (cycle, green,
    # offset): the lanes' ends are green at step t iff (t + offset) mod cycle
    # < green; cycle 0 = no signal.  None: no signals at all.
    link_signal: Optional[np.ndarray] = None
    # turn lanes (plan-following lane changes): for every non-ring link l and
    # every non-ring link m leaving l's end node (ascending link id), in that
    # order, one uint8 whose bit k says that lane k of l may be used to
    # continue onto m.  None: every lane for every turn.
    turn_lanes: Optional[np.ndarray] = None
    # gap acceptance at unprotected turns, uint8 [n_links]: 0 = a priority
    # approach, G in 1..31 = a yield approach whose vehicles cross only while
    # the priority approaches of the node have no vehicle in their last G
    # cells.  None: every approach has priority.
    link_yield: Optional[np.ndarray] = None

    @property
    def n_links(self) -> int:
        return int(self.link_cells.shape[0])

    @property
    def n_lanes(self) -> int:
        return int(self.link_lanes.sum())

    @property
    def n_lane_cells(self) -> int:
        return int((self.link_cells.astype(np.int64) * self.link_lanes).sum())

    def lane_base(self) -> np.ndarray:
        out = np.zeros(self.n_links + 1, np.int64)
        np.cumsum(self.link_lanes, out=out[1:])
        return out

    def lane_cell_base(self) -> np.ndarray:
        """Offset of each canonical lane's cell 0 in the lane-cell order."""
        per_lane = np.repeat(self.link_cells.astype(np.int64), self.link_lanes.astype(np.int64))
        out = np.zeros(per_lane.shape[0] + 1, np.int64)
        np.cumsum(per_lane, out=out[1:])
        return out


@dataclass
class Demand:
    depart_step: np.ndarray   # uint32 [n]
    route_offsets: np.ndarray  # uint32 [n+1]
    route_links: np.ndarray    # uint32 [route_offsets[-1]]

    @property
    def n(self) -> int:
        return int(self.depart_step.shape[0])


@dataclass
class InitialState:
    """A canonical state to start from instead of the empty network."""
    cell_id: np.ndarray   # int32 [n_lane_cells], -1 = empty
    cell_v: np.ndarray    # int8  [n_lane_cells]
    buf_id: np.ndarray    # int32 [n_lanes], -1 = empty link-end buffer
    buf_v: np.ndarray     # int8  [n_lanes]
    cursor: np.ndarray    # uint32 [n_vehicles], index into the vehicle's route
    dep_head: np.ndarray  # uint32 [n_links], queue entries already inserted
    step: int = 0
    arrived: int = 0
    inserted: int = 0


@dataclass
class Scenario:
    name: str
    net: Network
    demand: Demand
    steps: int
    seed: int = 1
    vmax: int = 5
    p_threshold: int = P_THRESHOLD_0_2
    lane_change: int = 1
    init: Optional[InitialState] = None
    meta: dict = field(default_factory=dict)


# ---------------------------------------------------------------- networks

def _links_from_edges(n_nodes, a, b, cells, lanes) -> Network:
    """Each undirected edge e=(a,b) becomes links 2e (a->b) and 2e+1 (b->a)."""
    m = a.shape[0]
    lf = np.empty(2 * m, np.uint32)
    lt = np.empty(2 * m, np.uint32)
    lf[0::2], lt[0::2] = a, b
    lf[1::2], lt[1::2] = b, a
    return Network(
        n_nodes=int(n_nodes),
        link_from=lf,
        link_to=lt,
        link_cells=np.repeat(np.asarray(cells, np.uint32), 2),
        link_lanes=np.repeat(np.asarray(lanes, np.uint32), 2),
        link_ring=np.zeros(2 * m, np.uint8),
    )


def _grid_edges(n: int):
    a, b = [], []
    for r in range(n):
        for c in range(n):
            u = r * n + c
            if c + 1 < n:
                a.append(u); b.append(u + 1)
            if r + 1 < n:
                a.append(u); b.append(u + n)
    return np.array(a, np.uint32), np.array(b, np.uint32)


def grid_network(n_side: int, lanes: int, cells: int) -> Network:
    """n_side x n_side nodes, every adjacent pair joined by two directed links."""
    a, b = _grid_edges(n_side)
    m = a.shape[0]
    return _links_from_edges(n_side * n_side, a, b, np.full(m, cells), np.full(m, lanes))


def random_grid_network(rng: np.random.Generator, side_lo=10, side_hi=60,
                        cells_lo=30, cells_hi=120) -> Network:
    """Square grid, side ~ U{side_lo..side_hi}; per edge lanes ~ U{1,2,3} and
    cells ~ U{cells_lo..cells_hi}, shared by both directions."""
    n = int(rng.integers(side_lo, side_hi + 1))
    a, b = _grid_edges(n)
    m = a.shape[0]
    lanes = rng.integers(1, 4, m)
    cells = rng.integers(cells_lo, cells_hi + 1, m)
    return _links_from_edges(n * n, a, b, cells, lanes)


def planar_network(n_nodes: int, n_edges: int, seed: int) -> Network:
    """Seeded random planar road network.

    Points uniform in the unit square; the Euclidean minimum spanning tree
    for connectivity, then the shortest remaining Delaunay edges (Delaunay
    edges never cross) until n_edges undirected edges exist.  Each edge
    gets a length ~ lognormal(median 300 m, sigma 0.8), cells =
    max(3, round(len / 7.5 m)), and lanes 1/2/3 with probability
    0.5/0.35/0.15, shared by both directions.
    """
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import minimum_spanning_tree
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)
    pts = rng.random((n_nodes, 2))
    tri = Delaunay(pts)
    s = tri.simplices
    e = np.concatenate([s[:, [0, 1]], s[:, [1, 2]], s[:, [0, 2]]])
    e.sort(axis=1)
    e = np.unique(e, axis=0)
    if n_edges > e.shape[0] or n_edges < n_nodes - 1:
        raise ValueError("n_edges outside [n_nodes-1, #Delaunay edges]")
    ln = np.linalg.norm(pts[e[:, 0]] - pts[e[:, 1]], axis=1)
    g = coo_matrix((ln, (e[:, 0], e[:, 1])), shape=(n_nodes, n_nodes)).tocsr()
    mst = minimum_spanning_tree(g).tocoo()
    mst_pairs = np.stack([np.minimum(mst.row, mst.col), np.maximum(mst.row, mst.col)], 1)
    key = e[:, 0].astype(np.int64) * n_nodes + e[:, 1]
    mkey = mst_pairs[:, 0].astype(np.int64) * n_nodes + mst_pairs[:, 1]
    in_mst = np.isin(key, mkey)
    rest = np.nonzero(~in_mst)[0]
    rest = rest[np.argsort(ln[rest], kind="stable")][: n_edges - int(in_mst.sum())]
    chosen = np.sort(np.concatenate([np.nonzero(in_mst)[0], rest]))
    ea = e[chosen, 0].astype(np.uint32)
    eb = e[chosen, 1].astype(np.uint32)
    m = ea.shape[0]
    length = rng.lognormal(np.log(300.0), 0.8, m)
    cells = np.maximum(3, np.rint(length / CELL_M)).astype(np.uint32)
    lanes = rng.choice(np.array([1, 2, 3]), size=m, p=[0.5, 0.35, 0.15])
    return _links_from_edges(n_nodes, ea, eb, cells, lanes)


def ring_network(cells: int, lanes: int = 1) -> Network:
    """One periodic link: the circle road of Sec. 5 (1-lane and 3-lane)."""
    return Network(
        n_nodes=0,
        link_from=np.array([NO_NODE], np.uint32),
        link_to=np.array([NO_NODE], np.uint32),
        link_cells=np.array([cells], np.uint32),
        link_lanes=np.array([lanes], np.uint32),
        link_ring=np.array([1], np.uint8),
    )


# ---------------------------------------------------------------- demand

def uniform_trips(net: Network, n: int, window: int, rng: np.random.Generator):
    """Origin != destination uniform over nodes; departure floor(U * window)."""
    N = net.n_nodes
    o = rng.integers(0, N, n)
    d = rng.integers(0, N - 1, n)
    d = d + (d >= o)
    dep = np.floor(rng.random(n) * window).astype(np.uint32)
    return o.astype(np.uint32), d.astype(np.uint32), dep


def degree_weighted_trips(net: Network, n: int, mean_s: float, sigma_s: float,
                          horizon: int, rng: np.random.Generator):
    """Origin and destination drawn in proportion to node degree (O != D);
    departure ~ Normal(mean_s, sigma_s) redrawn until inside [0, horizon)."""
    N = net.n_nodes
    deg = np.bincount(net.link_from, minlength=N).astype(np.float64)
    w = deg / deg.sum()
    o = rng.choice(N, size=n, p=w)
    d = rng.choice(N, size=n, p=w)
    bad = np.nonzero(o == d)[0]
    while bad.size:
        d[bad] = rng.choice(N, size=bad.size, p=w)
        bad = bad[o[bad] == d[bad]]
    dep = rng.normal(mean_s, sigma_s, n)
    out = np.nonzero((dep < 0) | (dep >= horizon))[0]
    while out.size:
        dep[out] = rng.normal(mean_s, sigma_s, out.size)
        out = out[(dep[out] < 0) | (dep[out] >= horizon)]
    return o.astype(np.uint32), d.astype(np.uint32), np.floor(dep).astype(np.uint32)


_routes_lib = None


def _load_routes_lib():
    global _routes_lib
    if _routes_lib is not None:
        return _routes_lib
    here = os.path.dirname(os.path.abspath(__file__))
    so = os.path.join(here, "libroutes.so")
    src = os.path.join(here, "routes.c")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        from .. import build as _build
        _build.build_routes_lib()
    lib = ctypes.CDLL(so)
    P = ctypes.POINTER
    lib.routes_build.restype = ctypes.c_int
    lib.routes_build.argtypes = [
        ctypes.c_uint32, ctypes.c_uint32, P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32),
        ctypes.c_uint64, P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint64), P(ctypes.c_uint64),
        ctypes.c_uint64, P(ctypes.c_uint64), P(P(ctypes.c_uint32)), ctypes.c_int]
    lib.routes_free.argtypes = [P(ctypes.c_uint32)]
    _routes_lib = lib
    return lib


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def build_routes(net: Network, orig: np.ndarray, dest: np.ndarray, threads: Optional[int] = None,
                 weights: Optional[np.ndarray] = None):
    """Shortest path from orig[i] to dest[i] as link lists, under integer link
    weights (default: the link length in cells).

    Ties between equally short paths go to the predecessor with the
    smaller node id, which makes every route unique."""
    lib = _load_routes_lib()
    orig = np.ascontiguousarray(orig, np.uint32)
    dest = np.ascontiguousarray(dest, np.uint32)
    n = orig.shape[0]
    order = np.argsort(orig, kind="stable").astype(np.uint64)
    so = orig[order.astype(np.int64)]
    starts = np.nonzero(np.diff(so.astype(np.int64), prepend=-1))[0]
    grp_off = np.append(starts, n).astype(np.uint64)
    lf = np.ascontiguousarray(net.link_from, np.uint32)
    lt = np.ascontiguousarray(net.link_to, np.uint32)
    w = np.ascontiguousarray(net.link_cells if weights is None else weights, np.uint32)
    off = np.zeros(n + 1, np.uint64)
    out = ctypes.POINTER(ctypes.c_uint32)()
    if threads is None:
        threads = min(32, os.cpu_count() or 1)
    rc = lib.routes_build(net.n_nodes, net.n_links, _ptr(lf, ctypes.c_uint32), _ptr(lt, ctypes.c_uint32),
                          _ptr(w, ctypes.c_uint32), n, _ptr(orig, ctypes.c_uint32), _ptr(dest, ctypes.c_uint32),
                          _ptr(order, ctypes.c_uint64), _ptr(grp_off, ctypes.c_uint64), grp_off.shape[0] - 1,
                          _ptr(off, ctypes.c_uint64), ctypes.byref(out), threads)
    if rc != 0:
        raise RuntimeError(f"route builder failed with code {rc}")
    total = int(off[-1])
    if total >= 2**32:
        raise ValueError("route table exceeds 32-bit offsets")
    links = np.ctypeslib.as_array(out, shape=(max(total, 1),))[:total].copy()
    lib.routes_free(out)
    return off.astype(np.uint32), links.astype(np.uint32)


def _demand(net, o, d, dep, threads=None) -> Demand:
    off, links = build_routes(net, o, d, threads)
    return Demand(depart_step=np.ascontiguousarray(dep, np.uint32), route_offsets=off, route_links=links)


# ---------------------------------------------------------------- initial ring states

def ring_initial_state(net: Network, n_veh: int, mode: str, v0: int = 0,
                       rng: Optional[np.random.Generator] = None):
    """Vehicles placed directly on the single ring link of ``net``.

    mode 'uniform': vehicle i at cell floor(i * L / n) of lane i % lanes.
    mode 'megajam': vehicles packed into consecutive cells from cell 0.
    mode 'random' : distinct cells drawn uniformly (needs rng).
    Every vehicle gets velocity v0, route [0], departure step 0, and counts
    as already inserted.
    """
    L = int(net.link_cells[0]); K = int(net.link_lanes[0])
    C = L * K
    if n_veh > C:
        raise ValueError("more vehicles than cells")
    if mode == "uniform":
        lane = np.arange(n_veh) % K
        per = np.bincount(lane, minlength=K)
        x = np.empty(n_veh, np.int64)
        for k in range(K):
            idx = np.nonzero(lane == k)[0]
            x[idx] = (np.arange(per[k]) * L) // max(per[k], 1)
        flat = lane * L + x
    elif mode == "megajam":
        flat = np.arange(n_veh)
    elif mode == "random":
        flat = np.sort(rng.choice(C, size=n_veh, replace=False))
    else:
        raise ValueError(mode)
    cell_id = np.full(C, -1, np.int32)
    cell_v = np.zeros(C, np.int8)
    cell_id[flat] = np.arange(n_veh, dtype=np.int32)
    cell_v[flat] = v0
    dem = Demand(depart_step=np.zeros(n_veh, np.uint32),
                 route_offsets=np.arange(n_veh + 1, dtype=np.uint32),
                 route_links=np.zeros(n_veh, np.uint32))
    init = InitialState(cell_id=cell_id, cell_v=cell_v,
                        buf_id=np.full(K, -1, np.int32), buf_v=np.zeros(K, np.int8),
                        cursor=np.zeros(n_veh, np.uint32),
                        dep_head=np.array([n_veh], np.uint32), step=0, arrived=0, inserted=n_veh)
    return dem, init


# ---------------------------------------------------------------- configurations

def _cache_dir():
    d = os.environ.get("TRANSSIM_INPUT_CACHE")
    if d is None:
        d = os.path.join(os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))),
                         "_build", "inputs")
    os.makedirs(d, exist_ok=True)
    return d


def _cached(key: str, make):
    path = os.path.join(_cache_dir(), hashlib.sha1(key.encode()).hexdigest()[:16] + ".npz")
    if os.path.exists(path):
        z = np.load(path)
        net = Network(int(z["n_nodes"]), z["lf"], z["lt"], z["lc"], z["ll"], z["lr"])
        return net, Demand(z["dep"], z["off"], z["links"])
    net, dem = make()
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, n_nodes=net.n_nodes, lf=net.link_from, lt=net.link_to, lc=net.link_cells,
             ll=net.link_lanes, lr=net.link_ring, dep=dem.depart_step, off=dem.route_offsets,
             links=dem.route_links)
    os.replace(tmp, path)
    return net, dem


def grid_signals(net: Network, n_side: int, cycle: int, green: int) -> np.ndarray:
    """A signal at every link end of a grid_network: links running east-west
    are green for the first `green` steps of each cycle, links running
    north-south for the `green` steps that follow (green <= cycle / 2), so
    crossing streams are never green together."""
    horizontal = np.abs(net.link_from.astype(np.int64) - net.link_to.astype(np.int64)) == 1
    sig = np.zeros((net.n_links, 3), np.uint32)
    sig[:, 0] = cycle
    sig[:, 1] = green
    sig[:, 2] = np.where(horizontal, 0, cycle - green)  # (t + offset) mod cycle < green
    return sig


def turn_table_offsets(net: Network) -> np.ndarray:
    """First turn-table entry of every link (n_links + 1 entries): a non-ring
    link has one entry per non-ring link leaving its end node."""
    ring = np.asarray(net.link_ring, bool)
    outdeg = np.bincount(np.asarray(net.link_from, np.int64)[~ring], minlength=net.n_nodes)
    per = np.where(ring, 0, outdeg[np.where(ring, 0, np.asarray(net.link_to, np.int64))])
    off = np.zeros(net.n_links + 1, np.int64)
    np.cumsum(per, out=off[1:])
    return off


def turn_lanes_by_rank(net: Network) -> np.ndarray:
    """Synthetic turn lanes: the n links leaving a link's end node, in
    ascending id, share the link's L lanes in order, lane k serving turns
    [k n / L, (k+1) n / L): turn j may use lane k iff those ranges overlap
    (j L < (k+1) n and k n < (j+1) L).  Every turn gets at least one lane and
    every lane at least one turn; a one-lane link serves every turn."""
    off = turn_table_offsets(net)
    out = np.zeros(int(off[-1]), np.uint8)
    lanes = np.asarray(net.link_lanes, np.int64)
    for l in range(net.n_links):
        n = int(off[l + 1] - off[l])
        L = int(lanes[l])
        for j in range(n):
            m = 0
            for k in range(L):
                if j * L < (k + 1) * n and k * n < (j + 1) * L:
                    m |= 1 << k
            out[off[l] + j] = m
    return out


def signals_by_rank(net: Network, cycle: int, green: int) -> np.ndarray:
    """A fixed-time light at the end of every non-ring link of any network:
    the approaches of a node, in ascending link id, alternate between the
    first `green` steps of each cycle (even rank) and the `green` steps that
    follow (odd rank; green <= cycle / 2), so approaches of different rank
    are never green together.  A node with one approach gets no light."""
    ring = np.asarray(net.link_ring, bool)
    to = np.asarray(net.link_to, np.int64)
    sig = np.zeros((net.n_links, 3), np.uint32)
    idx = np.nonzero(~ring)[0]
    order = idx[np.lexsort((idx, to[idx]))]          # by end node, then link id
    nodes = to[order]
    start = np.r_[0, np.nonzero(np.diff(nodes))[0] + 1]
    count = np.diff(np.r_[start, nodes.size])
    rank = np.arange(nodes.size) - np.repeat(start, count)
    many = np.repeat(count, count) > 1
    lit = order[many]
    sig[lit, 0] = cycle
    sig[lit, 1] = green
    sig[lit, 2] = np.where(rank[many] % 2 == 0, 0, cycle - green)  # (t + offset) mod cycle < green
    return sig


def grid_yield(net: Network, gap: int) -> np.ndarray:
    """Unprotected turns on a grid_network: links running north-south yield
    (acceptance gap `gap` cells) to links running east-west."""
    horizontal = np.abs(net.link_from.astype(np.int64) - net.link_to.astype(np.int64)) == 1
    return np.where(horizontal, 0, gap).astype(np.uint8)


def yield_by_lanes(net: Network, gap: int) -> np.ndarray:
    """Unprotected turns on any network: at every node, the approaches with
    fewer lanes than the node's widest approach yield (acceptance gap `gap`
    cells); a node whose approaches are all equally wide has no yield."""
    ring = np.asarray(net.link_ring, bool)
    to = np.where(ring, 0, np.asarray(net.link_to, np.int64))
    lanes = np.asarray(net.link_lanes, np.int64)
    widest = np.zeros(net.n_nodes, np.int64)
    np.maximum.at(widest, to[~ring], lanes[~ring])
    return np.where(~ring & (lanes < widest[to]), gap, 0).astype(np.uint8)


def small_grid_scenario(n_side=3, lanes=2, cells=20, n_trips=60, window=60, steps=200,
                        gen_seed=0, seed=1, vmax=5, p_threshold=P_THRESHOLD_0_2, signal=None,
                        turns=False, lane_seed=None, yield_gap=None) -> Scenario:
    """signal = (cycle, green): a traffic light at every link end (grid_signals).
    turns: turn lanes by rank (turn_lanes_by_rank).  lane_seed: lanes per
    undirected edge ~ U{1..lanes} from that seed instead of `lanes` everywhere.
    yield_gap: north-south links yield to east-west links with that
    acceptance gap (grid_yield)."""
    net = grid_network(n_side, lanes, cells)
    if lane_seed is not None:
        per_edge = np.random.default_rng(lane_seed).integers(1, lanes + 1, net.n_links // 2)
        net = dataclasses.replace(net, link_lanes=np.repeat(per_edge, 2).astype(np.uint32))
    if signal is not None:
        net = dataclasses.replace(net, link_signal=grid_signals(net, n_side, *signal))
    if turns:
        net = dataclasses.replace(net, turn_lanes=turn_lanes_by_rank(net))
    if yield_gap is not None:
        net = dataclasses.replace(net, link_yield=grid_yield(net, yield_gap))
    rng = np.random.default_rng(gen_seed)
    o, d, dep = uniform_trips(net, n_trips, window, rng)
    return Scenario(f"grid{n_side}x{n_side}", net, _demand(net, o, d, dep, 1), steps, seed, vmax, p_threshold)


def config0() -> Scenario:
    """5x5 grid, 2 lanes x 60 cells, 2,000 uniform trips departing in the
    first 600 s, 3,600 steps, Philox seed 1, generator seed 0."""
    def make():
        net = grid_network(5, 2, 60)
        o, d, dep = uniform_trips(net, 2000, 600, np.random.default_rng(0))
        return net, _demand(net, o, d, dep)
    net, dem = _cached("config0-v1", make)
    return Scenario("config0", net, dem, steps=3600, seed=1)


def _planar_config(name, n_nodes, n_edges, n_trips, gen_seed, steps=10800):
    def make():
        net = planar_network(n_nodes, n_edges, gen_seed)
        rng = np.random.default_rng(gen_seed + 7919)
        o, d, dep = degree_weighted_trips(net, n_trips, 5400.0, 2400.0, 10800, rng)
        return net, _demand(net, o, d, dep)
    net, dem = _cached(f"{name}-v1-{n_nodes}-{n_edges}-{n_trips}-{gen_seed}", make)
    return Scenario(name, net, dem, steps=steps, seed=1)


def config1() -> Scenario:
    """Portland-shaped: 8,500 nodes, 10,012 edges = 20,024 directed links,
    300,000 degree-weighted trips over 3 h, 10,800 steps."""
    return _planar_config("config1", 8500, 10012, 300_000, 1)


def config2() -> Scenario:
    """Scale-up: 85,000 nodes, 100,000 edges = 200,000 directed links,
    2,000,000 trips over 3 h, 10,800 steps."""
    return _planar_config("config2", 85_000, 100_000, 2_000_000, 2)


def config3_scenario(i: int, demand_scale: float = 1.0, steps: int = 3600) -> Scenario:
    """Batch member i: random square grid (generator seed 1000+i), demand
    d ~ U(0.1, 0.4) trips per lane-cell departing uniformly over 600 s,
    Philox seed 1000+i.  demand_scale < 1 thins the trips (for tests)."""
    def make():
        rng = np.random.default_rng(1000 + i)
        net = random_grid_network(rng)
        dens = rng.uniform(0.1, 0.4)
        n = int(round(dens * net.n_lane_cells * demand_scale))
        o, d, dep = uniform_trips(net, n, 600, rng)
        return net, _demand(net, o, d, dep)
    net, dem = _cached(f"config3-v1-{i}-{demand_scale}", make)
    return Scenario(f"config3[{i}]", net, dem, steps=steps, seed=1000 + i)


# ---------------------------------------------------------------- a loaded network state

def loaded_state(sc: Scenario, step: int, seed: int, jam_share: float = 0.3,
                 buffer_share: float = 0.5) -> InitialState:
    """A seeded state of scenario `sc` at `step` with its traffic on the network.

    Stands in for a peak-hour state (the paper's step time grows with
    congestion, Sec. 8) without running any simulation: it places vehicles,
    it evaluates no driving rule.  Every trip whose departure step is before
    `step` has left its queue; it sits on a link of its route drawn
    uniformly (its cursor).  A share `jam_share` of the links hold their
    vehicles as a queue packed from the link end backwards over the lanes,
    with v = 0, and each lane of such a link hands its front vehicle to the
    lane's link-end buffer with probability `buffer_share` (if that vehicle
    has a next link); the other links hold theirs in distinct cells drawn
    uniformly, with v uniform in 0..vmax.  Vehicles for which a link has no
    cell left count as arrived.
    """
    net, dem = sc.net, sc.demand
    rng = np.random.default_rng(seed)
    n = dem.n
    off = dem.route_offsets.astype(np.int64)
    rlen = np.diff(off)
    departed = np.nonzero(dem.depart_step < step)[0]
    cursor = np.zeros(n, np.uint32)
    cur = np.floor(rng.random(departed.size) * rlen[departed]).astype(np.int64)
    cursor[departed] = cur
    link_of = dem.route_links[off[departed] + cur].astype(np.int64)
    L = net.n_links
    cells = net.link_cells.astype(np.int64)
    lanes = net.link_lanes.astype(np.int64)
    jam = (rng.random(L) < jam_share) & (net.link_ring == 0)
    # every lane-cell of every link, ranked within its link: from the link end
    # backwards over the lanes on a jammed link, in a random order elsewhere
    lb, cb = net.lane_base(), net.lane_cell_base()
    C = int(cb[-1])
    lane_of_cell = np.repeat(np.arange(net.n_lanes), np.diff(cb))
    lane_link = np.repeat(np.arange(L), lanes)
    cl = lane_link[lane_of_cell]
    ck = lane_of_cell - lb[cl]
    cx = np.arange(C, dtype=np.int64) - cb[lane_of_cell]
    key = np.where(jam[cl], (cells[cl] - 1 - cx) * lanes[cl] + ck, rng.random(C) * cells[cl] * lanes[cl])
    order = np.lexsort((key, cl))
    first = np.zeros(L + 1, np.int64)
    np.cumsum(cells * lanes, out=first[1:])
    # vehicles of each link in a random order, matched to its ranked cells
    vorder = np.lexsort((rng.random(departed.size), link_of))
    vl = link_of[vorder]
    vstart = np.searchsorted(vl, np.arange(L))
    rank = np.arange(departed.size) - vstart[vl]
    fits = rank < cells[vl] * lanes[vl]
    ids = departed[vorder][fits]
    slot = order[first[vl[fits]] + rank[fits]]
    cell_id = np.full(C, -1, np.int32)
    cell_v = np.zeros(C, np.int8)
    cell_id[slot] = ids
    v = rng.integers(0, sc.vmax + 1, ids.size)
    cell_v[slot] = np.where(jam[cl[slot]], 0, v).astype(np.int8)
    # front vehicles of jammed lanes into the link-end buffers
    buf_id = np.full(net.n_lanes, -1, np.int32)
    buf_v = np.zeros(net.n_lanes, np.int8)
    front = cb[1:] - 1                      # last cell of every lane
    fid = cell_id[front]
    lane_l = lane_link
    take = (fid >= 0) & jam[lane_l] & (rng.random(net.n_lanes) < buffer_share)
    take &= cursor[np.maximum(fid, 0)] + 1 < rlen[np.maximum(fid, 0)]
    buf_id[take] = fid[take]
    cell_id[front[take]] = -1
    cell_v[front[take]] = 0
    # departure queues: entries with departure step before `step` have left
    first_link = dem.route_links[off[:-1]].astype(np.int64)
    dep_head = np.bincount(first_link[departed], minlength=L).astype(np.uint32)
    on = int(ids.size)
    return InitialState(cell_id=cell_id, cell_v=cell_v, buf_id=buf_id, buf_v=buf_v, cursor=cursor,
                        dep_head=dep_head, step=int(step), arrived=int(departed.size - on),
                        inserted=int(departed.size))
