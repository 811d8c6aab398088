"""Pin strength: each planted mistake in the oracle (built as a separate variant with
-DORACLE_MUTANT=m, on the CPU) must make at least one pin of test_oracle_pins fail.
The mistakes are the plausible ones: a dropped pixel-centre offset, a mirrored axis,
truncation instead of floor, a dropped projection term, a reversed DDA tie rule, an
inclusive range test, exit instead of entry depth, no owner test, parent-only exclusion,
a strict depth comparison, highest-index yaw ties, a flipped yaw sign, an exact route
that double counts, and in the interval mode (Eq. 5-7): a depth sample at the portion's
entry instead of its midpoint, a screen parameter without perspective correction, a strict
depth comparison, and a voxel sample at the voxel's entry instead of its traversal midpoint;
in the panoramic mode: a wedge test that includes its upper boundary (double ownership) and
a yaw window shifted by one column; in the exact-yaw variant, the highest yaw on ties."""
import pytest

import oracle
import test_oracle_exact_yaw as xpins  # noqa: E402
import test_oracle_interval as ipins  # noqa: E402
import test_oracle_pano as ppins  # noqa: E402
import test_oracle_pins as pins  # noqa: E402
from synth import Sensor

MUTANTS = list(range(1, 21))

PIN_CALLS = [
    lambda o: pins.test_dda_matches_exact_slab_brute_force(o),
    lambda o: pins.test_dda_tie_rule_x_then_y_then_z(o),
    lambda o: pins.test_dda_stops_at_range_and_grid(o),
    lambda o: pins.test_ray_directions_match_float_pinhole(o, Sensor(87, 58, 48, 28, 5.0, 12, 10.0)),
    lambda o: pins.test_projection_matches_float_pinhole(o, Sensor(87, 58, 48, 28, 5.0, 12, 10.0)),
    lambda o: pins.test_depth_of_fronto_parallel_wall(o),
    lambda o: pins.test_ancestor_test_is_smaller_or_equal(o),
    lambda o: pins.test_depth_of_range_endpoint(o),
    lambda o: pins.test_owner_set_equals_voxel_centric_brute_force(o),
    lambda o: pins.test_absolute_gain_frustum_volume_closed_form(o),
    lambda o: pins.test_marginal_invariants(o, 1),
    lambda o: pins.test_fixed_yaw_ordering_abs_sp_all(o),
    lambda o: pins.test_disjoint_frusta_and_identical_pose(o),
    lambda o: pins.test_exact_routes_agree_and_telescope(o, 2),
    lambda o: pins.test_tiny_config_gap_is_small_and_positive(o),
    lambda o: ipins.test_interval_segment_matches_float_camera(o, ipins.SENSORS[1]),
    lambda o: ipins.test_interval_walk_tiles_the_clipped_segment(o, ipins.SENSORS[1]),
    lambda o: ipins.test_interval_depth_sample_is_perspective_midpoint_smaller_or_equal(o, ipins.SENSORS[0]),
    lambda o: ipins.test_interval_equal_depth_counts_as_observed(o),
    lambda o: ipins.test_interval_sample_parameter_is_perspective_correct(o, ipins.SENSORS[0]),
    lambda o: ipins.test_interval_voxel_sample_is_traversal_midpoint(o),
    lambda o: ipins.test_interval_mode_invariants(o, 1),
    lambda o: ipins.test_interval_mode_special_cases(o),
    lambda o: ipins.test_interval_mode_gap_to_exact_tiny(o),
    lambda o: ppins.test_pano_tables_match_float_model(o, ppins.SENSORS[0]),
    lambda o: ppins.test_pano_cells_match_float_azimuth_elevation(o, ppins.SENSORS[0]),
    lambda o: ppins.test_pano_owner_set_equals_voxel_centric_brute_force(o, 3),
    lambda o: ppins.test_pano_window_sums_and_identity(o, ppins.SENSORS[2]),
    lambda o: ppins.test_pano_mode_invariants(o, 1),
    lambda o: xpins.test_exact_yaw_matches_hash_set_walk(o, 3),
    lambda o: xpins.test_exact_yaw_special_cases(o),
]


@pytest.mark.parametrize("mutant", MUTANTS)
def test_planted_mistake_fails_a_pin(mutant):
    o = oracle.load_variant(mutant)
    o.build()
    failed = []
    for i, call in enumerate(PIN_CALLS):
        try:
            call(o)
        except (AssertionError, o.OracleError, RuntimeError):
            failed.append(i)
    assert failed, f"mutant {mutant} passed every pin"


def test_unmutated_oracle_passes_every_pin():
    o = oracle
    o.build()
    for call in PIN_CALLS:
        call(o)
