"""Runs a fast selection of the oracle's pins against one build of oracle.c
(test helper of test_oracle_mutants.py, executed in a child process so that
a build that aborts on an impossible state cannot take the test run down).

    python tests/mutant_checks.py <path of the oracle build>

Exit status 0: every check passed; 1: a check failed (the name is printed).
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402


def checks():
    import test_oracle_pins as P
    return [
        ("philox known answers", P.test_philox_known_answers),
        ("single car", P.test_single_car_trajectory),
        ("deceleration to the link end", P.test_car_decelerates_to_link_end_and_arrives),
        ("transfer keeps velocity", P.test_transfer_keeps_velocity_and_then_arrives),
        ("intersection priority", P.test_intersection_priority_lower_link_id_first),
        ("transfer lane preference", P.test_transfer_lane_preference),
        ("lane change on even steps", P.test_lane_change_even_step_moves_up),
        ("lane change needs room behind", P.test_lane_change_needs_room_behind),
        ("lane change near a link end", lambda: P.test_stopped_vehicle_near_the_end_changes_lane_whatever_the_end_state("red")),
        ("free flow keeps its lane", P.test_vehicle_with_vmax_free_cells_ahead_keeps_its_lane),
        ("ring free flow", P.test_ring_free_flow_exact),
        ("ring jam", P.test_ring_jam_exact),
        ("megajam dissolves", P.test_megajam_dissolves_one_car_per_step),
        ("link travel times", P.test_link_travel_times_by_hand),
        ("red light", P.test_car_waits_at_a_red_light_by_hand),
        ("wrong lane changes towards its turn", P.test_wrong_lane_changes_towards_its_turn_on_the_next_odd_step),
        ("accepted gap shrinks", P.test_accepted_gap_shrinks_near_the_intersection),
        ("yield waits for the gap", P.test_yield_waits_for_the_gap_on_the_priority_street_by_hand),
        ("yield gap skips cell 0", P.test_yield_gap_never_counts_cell_zero),
        ("invariants and digest", P.test_invariants_on_grid),
        ("naive restatement", lambda: P.test_oracle_matches_naive_restatement((3, 2, 15, 120, 4, 5, 1))),
        ("naive restatement, all routes and rules", lambda: P.test_every_route_of_a_2x2_grid_matches_naive_restatement("all")),
        ("naive restatement, random rules", lambda: P.test_random_intersection_rules_match_naive_restatement(0)),
    ]


def main(path):
    oracle._lib = oracle.bind(path)
    for name, fn in checks():
        try:
            fn()
        except AssertionError:
            print(f"caught by: {name}", flush=True)
            return 1
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1]))
