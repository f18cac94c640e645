"""Relaxation iterations with the GPU micro-simulation equal the same
iterations with the oracle: every run's statistics and link travel times,
and the final plans."""
import numpy as np
import pytest

from paper_cs_0105004_gb300 import relaxation as R
from paper_cs_0105004_gb300.inputs import networks as N
from test_relaxation import oracle_run

pytestmark = pytest.mark.gpu


def test_gpu_relaxation_equals_oracle_relaxation():
    sc = N.small_grid_scenario(5, 2, 25, n_trips=1500, window=200, steps=1200, gen_seed=12, seed=4)
    g_last, g_its = R.relax(sc, 3, fraction=0.1, seed=5)
    o_last, o_its = R.relax(sc, 3, fraction=0.1, seed=5, run=oracle_run)
    for g, o in zip(g_its, o_its):
        assert g.replanned == o.replanned
        assert (g.run.vehicle_updates, g.run.arrived) == (o.run.vehicle_updates, o.run.arrived), g.index
        assert np.array_equal(g.run.link_time_sum, o.run.link_time_sum), g.index
        assert np.array_equal(g.run.link_time_count, o.run.link_time_count), g.index
    assert np.array_equal(g_last.demand.route_links, o_last.demand.route_links)
    assert np.array_equal(g_last.demand.route_offsets, o_last.demand.route_offsets)
