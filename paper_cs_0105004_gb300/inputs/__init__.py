"""Seeded synthetic inputs: road networks, trips, routes and initial ring states.

This module only builds inputs.  It holds none of the cellular-automaton
arithmetic: the CUDA library and the CPU oracle both consume what it makes,
and neither is imported here.

The paper's own inputs (the Portland EMME/2 network, the TIGER network, the
Dallas plans, Sec. 6 and Sec. 7) are not available, so seeded generators with
the paper's shapes stand in for them: a 20,024-link and a 200,000-link planar
network (Sec. 6 quotes both sizes), square grids, and ring roads for the
1-lane and 3-lane circle experiments of Sec. 5.
"""
from .networks import (  # noqa: F401
    Network,
    Demand,
    InitialState,
    Scenario,
    grid_network,
    random_grid_network,
    planar_network,
    ring_network,
    uniform_trips,
    degree_weighted_trips,
    build_routes,
    ring_initial_state,
    config0,
    config1,
    config2,
    config3_scenario,
    small_grid_scenario,
    P_THRESHOLD_0_2,
)
