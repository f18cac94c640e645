"""The seeded input generators have the shapes the workloads are described
with: planar, strongly connected networks with both directions of every
edge, the config-1 link count, trips with origin != destination and
departures inside the horizon, and routes that are shortest paths with ties
to the smaller predecessor node id (checked against scipy's Dijkstra)."""
import numpy as np
import pytest

from paper_cs_0105004_gb300.inputs import networks as N

sp = pytest.importorskip("scipy.sparse")
csgraph = pytest.importorskip("scipy.sparse.csgraph")


def _graph(net, weights=None):
    w = (net.link_cells if weights is None else weights).astype(np.float64)
    return sp.csr_matrix((w, (net.link_from.astype(np.int64), net.link_to.astype(np.int64))),
                         shape=(net.n_nodes, net.n_nodes))


def _segments_cross(p, q, r, s):
    # proper crossing of segments pq and rs (shared end points do not count)
    def orient(a, b, c):
        v = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
        return np.sign(v)
    return orient(p, q, r) * orient(p, q, s) < 0 and orient(r, s, p) * orient(r, s, q) < 0


def test_planar_network_shape():
    net = N.planar_network(200, 260, seed=3)
    assert net.n_links == 520 and net.n_nodes == 200
    a, b = net.link_from[0::2], net.link_to[0::2]
    assert np.array_equal(net.link_from[1::2], b) and np.array_equal(net.link_to[1::2], a)
    assert np.array_equal(net.link_cells[0::2], net.link_cells[1::2])
    assert np.array_equal(net.link_lanes[0::2], net.link_lanes[1::2])
    assert net.link_cells.min() >= 3 and set(np.unique(net.link_lanes).tolist()) <= {1, 2, 3}
    n_comp, _ = csgraph.connected_components(_graph(net), directed=True, connection="strong")
    assert n_comp == 1
    # planarity: no two edges cross (the generator's points are the same draw)
    pts = np.random.default_rng(3).random((200, 2))
    edges = list(zip(a.tolist(), b.tolist()))
    for i in range(len(edges)):
        for j in range(i + 1, len(edges)):
            (u, v), (x, y) = edges[i], edges[j]
            if len({u, v, x, y}) == 4:
                assert not _segments_cross(pts[u], pts[v], pts[x], pts[y]), (edges[i], edges[j])


def test_config1_network_size_and_connectivity():
    net = N.planar_network(8500, 10012, seed=1)
    assert net.n_links == 20024
    n_comp, _ = csgraph.connected_components(_graph(net), directed=True, connection="strong")
    assert n_comp == 1
    # lanes 1/2/3 with probability 0.5/0.35/0.15 per edge
    frac = np.bincount(net.link_lanes[0::2], minlength=4)[1:] / 10012
    assert np.all(np.abs(frac - [0.5, 0.35, 0.15]) < 0.02)
    # cells = max(3, round(lognormal(median 300 m, sigma 0.8) / 7.5 m)): median 40 cells
    assert 37 <= np.median(net.link_cells) <= 43


def test_trips():
    net = N.planar_network(300, 400, seed=5)
    o, d, dep = N.degree_weighted_trips(net, 50_000, 5400.0, 2400.0, 10800, np.random.default_rng(2))
    assert np.all(o != d) and dep.max() < 10800
    assert abs(float(dep.mean()) - 5400.0) < 60.0
    # origins in proportion to node degree
    deg = np.bincount(net.link_from, minlength=net.n_nodes)
    hits = np.bincount(o, minlength=net.n_nodes)
    assert np.corrcoef(deg, hits)[0, 1] > 0.95
    o, d, dep = N.uniform_trips(net, 20_000, 600, np.random.default_rng(3))
    assert np.all(o != d) and dep.max() < 600 and o.max() < net.n_nodes and d.max() < net.n_nodes


@pytest.mark.parametrize("kind", ["planar", "grid"])
def test_routes_are_shortest_with_ties_to_the_smaller_predecessor(kind):
    # the grid has equal link lengths: many equally short routes, so the tie
    # rule decides every one of them
    net = N.planar_network(150, 200, seed=7) if kind == "planar" else N.grid_network(6, 1, 10)
    rng = np.random.default_rng(11)
    o, d, _ = N.uniform_trips(net, 300, 10, rng)
    off, links = N.build_routes(net, o, d)
    g = _graph(net)
    w = {(int(a), int(b)): int(c) for a, b, c in zip(net.link_from, net.link_to, net.link_cells)}
    preds = {}
    for a, b in w:
        preds.setdefault(b, []).append(a)
    for i in range(o.size):
        r = links[off[i]:off[i + 1]]
        assert net.link_from[r[0]] == o[i] and net.link_to[r[-1]] == d[i]
        assert all(net.link_to[x] == net.link_from[y] for x, y in zip(r[:-1], r[1:]))
        dist = csgraph.dijkstra(g, directed=True, indices=int(o[i]))
        assert int(net.link_cells[r].sum()) == int(dist[d[i]])
        for x in r:
            u, v = int(net.link_from[x]), int(net.link_to[x])
            tight = [p for p in preds[v] if dist[p] + w[(p, v)] == dist[v]]
            assert u == min(tight)


def test_config3_members():
    # side U{10..60}, lanes U{1,2,3} and cells U{30..120} per edge (both
    # directions alike), trips = round(d * lane-cells) with d in [0.1, 0.4],
    # departures over the first 600 s
    for i in range(6):
        sc = N.config3_scenario(i)
        net = sc.net
        side = int(round(np.sqrt(net.n_nodes)))
        assert side * side == net.n_nodes and 10 <= side <= 60
        assert net.n_links == 4 * side * (side - 1)
        assert np.array_equal(net.link_cells[0::2], net.link_cells[1::2])
        assert net.link_cells.min() >= 30 and net.link_cells.max() <= 120
        assert set(np.unique(net.link_lanes).tolist()) <= {1, 2, 3}
        d = sc.demand.n / net.n_lane_cells
        assert 0.1 - 1e-6 <= d <= 0.4 + 1e-6
        assert sc.demand.depart_step.max() < 600 and sc.seed == 1000 + i
