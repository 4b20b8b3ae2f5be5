"""Every planted mistake in the oracle makes at least one physics pin fail.

The oracle carries a switch that plants one numbered mistake at a time (a dropped term, a
flipped sign, a transposed operand, a wrong factor or index).  For each one this test runs the
pins of the other oracle test files and requires that some pin fails, so the pins can tell a
correct oracle from a plausibly wrong one.
"""
import numpy as np
import pytest

from oracle.oracle import set_mutation

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

MUTATIONS = {
    1: "bending couple without the (kappa x m) averaging term",
    2: "shear couple with the wrong sign",
    3: "internal force without the 1/e factor",
    4: "shear strain from Q^T l instead of Q l",
    5: "angular balance without the (J w/e^2) de/dt term",
    6: "angular balance without the (J w/e) x w term",
    7: "director update exp(+h[w]x) instead of exp(-h[w]x)",
    8: "bending couple divided by eps^2 instead of eps^3",
    9: "curvature from +log instead of -log",
    10: "contact force split (s, 1-s) instead of (1-s, s)",
    11: "dashpot with the wrong sign",
    12: "cell list missing the -x neighbour cells",
    14: "node mass doubled",
    15: "no rotational damping",
    17: "angular acceleration without the e factor",
    19: "gravity with the wrong sign",
    20: "actuation couple on the clamped element",
    21: "no Stokes drag",
    22: "magnetic couple with Q^T b instead of Q b",
    23: "muscle couples tau_i - tau_{i-1} instead of tau_{i-1} - tau_i",
    24: "wall contact without the rod radius",
    25: "friction along the sliding direction instead of against it",
    26: "energy: bend/twist term over one element's rest length instead of the Voronoi length",
    27: "energy: rotational kinetic term with I_1 about every axis",
    28: "energy: shear terms with the axial stiffness E A",
    29: "energy: work potential of gravity with the wrong sign",
    30: "energy: translational kinetic term without the 1/2",
}


def _baseline_passes():
    for pin in PINS:
        pin()


def test_pins_pass_without_mutation():
    set_mutation(0)
    _baseline_passes()


@pytest.mark.parametrize("mid", sorted(MUTATIONS))
def test_each_mutation_fails_some_pin(mid):
    caught = None
    try:
        set_mutation(mid)
        with np.errstate(all="ignore"):
            for pin in PINS:
                try:
                    pin()
                except Exception as exc:  # AssertionError, or a NaN blow-up in the oracle
                    caught = f"{getattr(pin, '__name__', 'pin')}: {type(exc).__name__}"
                    break
    finally:
        set_mutation(0)
    assert caught is not None, f"mutation {mid} ({MUTATIONS[mid]}) passed every pin"
