"""Every planted mistake in the oracle makes at least one physics pin fail.

oracle/mutants.py lists numbered mistakes (a dropped term, a flipped sign, a transposed
operand, a wrong factor or index), each a patch of one snippet of the oracle's source compiled
into a library of its own; the oracle the other tests use has no switch.  For each mistake this
test runs the pins of the other oracle test files against the patched library and requires
that some pin fails, so the pins can tell a correct oracle from a plausibly wrong one.
"""
import numpy as np
import pytest

from oracle.mutants import MUTANTS, build_mutant
from oracle.oracle import using_library

import test_oracle_contact as tc
import test_oracle_dynamics as td
import test_oracle_energy as te
import test_oracle_more_pins as tm
import test_oracle_next_rows as tn
import test_oracle_rotations as tr
import test_oracle_statics as ts

PINS = [
    tr.test_director_update_direction_for_spin_about_d3,
    lambda: ts.test_uniform_stretch_closed_form(5.0),
    lambda: ts.test_uniform_bending_closed_form(1e-4),
    td.test_kirchhoff_helix_is_balanced,
    tm.test_stretched_arc_couple_scales_with_inverse_cube_stretch,
    tm.test_base_actuation_couple_static_balance,
    tm.test_free_fall,
    tm.test_damping_and_drag_rates,
    tm.test_angular_momentum_conserved,
    tc.test_crossing_segments_closed_form,
    lambda: tc.test_cell_list_pairs_equal_exhaustive(1, 1.0),
    tm.test_axial_mode_period,
    td.test_linear_momentum_conserved_for_free_rod,
    lambda: ts.test_timoshenko_cantilever(0.1, 0.02),
    tn.test_field_along_the_magnetization_exerts_no_couple,
    tn.test_muscle_couples_bend_a_free_rod_to_tau_over_B,
    tn.test_segment_resting_on_a_wall_sinks_by_mg_over_k,
    tn.test_sliding_on_a_wall_decelerates_at_mu_g,
    tn.test_sliding_crossing_feels_coulomb_friction,
    te.test_rigid_translation,
    te.test_uniform_angular_velocity,
    te.test_uniform_shear_and_stretch,
    te.test_uniform_bending,
    te.test_gravity_and_tip_force_potential,
]

MUTATIONS = {k: v[0] for k, v in MUTANTS.items()}


def _baseline_passes():
    for pin in PINS:
        pin()


def test_pins_pass_without_mutation():
    _baseline_passes()


def test_the_default_oracle_has_no_mutation_switch():
    import os
    here = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")
    for name in ("rod_oracle.c", "rod_oracle.h"):
        with open(os.path.join(here, name)) as f:
            text = f.read()
        assert "mut" not in text.lower(), name


@pytest.mark.parametrize("mid", sorted(MUTATIONS))
def test_each_mutation_fails_some_pin(mid):
    caught = None
    with using_library(build_mutant(mid)):
        with np.errstate(all="ignore"):
            for pin in PINS:
                try:
                    pin()
                except Exception as exc:  # AssertionError, or a NaN blow-up in the oracle
                    caught = f"{getattr(pin, '__name__', 'pin')}: {type(exc).__name__}"
                    break
    assert caught is not None, f"mutation {mid} ({MUTATIONS[mid]}) passed every pin"
