"""Re-planning between relaxation iterations (host logic), run with the
oracle as the micro-simulation.  The GPU loop is compared with this one in
test_gpu_relaxation.py."""
import numpy as np
import pytest

import oracle
from paper_cs_0105004_gb300 import relaxation as R
from paper_cs_0105004_gb300.inputs import networks as N


def oracle_run(sc):
    o = oracle.Oracle(sc)
    st = o.step(sc.steps)
    tsum, tcnt = o.link_times()
    o.close()
    return R.RunResult(0.0, int(st["vehicle_updates"].sum()), int(st["arrived"][-1]), int(st["state_hash"][-1]),
                       tsum, tcnt)


def _route_cost(links, costs):
    return int(sum(int(costs[l]) for l in links))


def _dijkstra_costs(net, costs, src):
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    g = sp.csr_matrix((costs.astype(np.float64), (net.link_from.astype(np.int64), net.link_to.astype(np.int64))),
                      shape=(net.n_nodes, net.n_nodes))
    return csgraph.dijkstra(g, directed=True, indices=src)


def test_link_costs_rounding_and_free_flow():
    net = N.grid_network(2, 1, 23)  # every link 23 cells
    tsum = np.zeros(net.n_links, np.uint64)
    tcnt = np.zeros(net.n_links, np.uint64)
    tsum[0], tcnt[0] = 15, 2   # mean 7.5 -> 8 (half up)
    tsum[1], tcnt[1] = 14, 2   # 7
    tsum[2], tcnt[2] = 0, 3    # 0 -> at least 1
    c = R.link_costs(net, 5, tsum, tcnt)
    assert c[0] == 8 and c[1] == 7 and c[2] == 1
    assert np.all(c[3:] == 5)  # ceil(23 / 5), nobody completed the link


def test_replan_changes_exactly_the_drawn_fraction_with_shortest_routes():
    sc = N.small_grid_scenario(5, 2, 30, n_trips=600, window=300, steps=10, gen_seed=4, seed=9)
    rng = np.random.default_rng(3)
    costs = rng.integers(1, 40, sc.net.n_links).astype(np.uint32)
    dem, chosen = R.replan(sc.net, sc.demand, costs, 0.1, np.random.default_rng(7))
    assert chosen.size == 60
    old_off, new_off = sc.demand.route_offsets, dem.route_offsets
    lf, lt = sc.net.link_from, sc.net.link_to
    for i in range(sc.demand.n):
        old = sc.demand.route_links[old_off[i]:old_off[i + 1]]
        new = dem.route_links[new_off[i]:new_off[i + 1]]
        assert lf[new[0]] == lf[old[0]] and lt[new[-1]] == lt[old[-1]]
        assert all(lt[a] == lf[b] for a, b in zip(new[:-1], new[1:]))
        if i not in set(chosen.tolist()):
            assert np.array_equal(old, new)
    # re-planned routes are shortest under the costs (checked with scipy's Dijkstra)
    for i in chosen[:20]:
        new = dem.route_links[new_off[i]:new_off[i + 1]]
        dist = _dijkstra_costs(sc.net, costs, int(lf[new[0]]))
        assert _route_cost(new, costs) == int(dist[int(lt[new[-1]])])
    assert np.array_equal(dem.depart_step, sc.demand.depart_step)
    # the draw is the seed's
    dem2, chosen2 = R.replan(sc.net, sc.demand, costs, 0.1, np.random.default_rng(7))
    assert np.array_equal(chosen, chosen2) and np.array_equal(dem.route_links, dem2.route_links)


def test_relaxation_with_the_oracle_moves_travellers_off_congested_links():
    # a grid loaded in a short window: the first run congests the shortest
    # routes; re-planning on the measured times spreads the load
    sc = N.small_grid_scenario(4, 1, 20, n_trips=700, window=120, steps=900, gen_seed=6, seed=2)
    last, its = R.relax(sc, 3, fraction=0.2, seed=1, run=oracle_run)
    assert [it.replanned for it in its] == [140, 140, 0]
    # every iteration runs every traveller to arrival within the horizon
    assert all(it.run.arrived == sc.demand.n for it in its)
    # re-planning on the congested run's times shortens the time travellers
    # spend on links (vehicle updates = vehicle-steps on links)
    assert its[1].run.vehicle_updates < its[0].run.vehicle_updates
    assert its[1].run.mean_link_time <= its[0].run.mean_link_time
    assert not np.array_equal(last.demand.route_links, sc.demand.route_links)


def test_relaxation_keeps_the_intersection_rules():
    # re-planning changes routes only; the network's turn lanes, yield
    # approaches and signals stay, and every iteration still runs (oracle)
    sc = N.small_grid_scenario(4, 3, 20, n_trips=500, window=120, steps=900, gen_seed=8, seed=3, turns=True,
                               lane_seed=4, yield_gap=6, signal=(30, 15))
    last, its = R.relax(sc, 3, fraction=0.1, seed=2, run=oracle_run)
    assert [it.replanned for it in its] == [50, 50, 0]
    assert last.net is sc.net
    assert all(it.run.arrived > 0 for it in its)
    assert not np.array_equal(last.demand.route_links, sc.demand.route_links)
    # the last plans, run again, give the last iteration's result
    again = oracle_run(last)
    assert again.state_hash == its[-1].run.state_hash and again.arrived == its[-1].run.arrived
