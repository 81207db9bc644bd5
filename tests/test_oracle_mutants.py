"""Mutation tests of the oracle's pins: each plausible mistake planted in a copy of an oracle
source (tests/oracle_mutants.py) must make the pins named for it fail, so that the pins are known
to detect a dropped term, a wrong sign, constant or index, or a transposed operand in every part
of the kinetics and the integrator (including mistakes made consistently in the rates and in the
analytic Jacobian), the species-equation assembly and PaSR factor, the transport mixture rules,
and the surrogate's network, training step and post-processing.  The mistakes are planted on the
CPU, in copies; the oracle itself is untouched."""
import numpy as np
import pytest

import oracle
import test_oracle_fvm as F
import test_oracle_integrator as I
import test_oracle_kinetics as K
import test_oracle_surrogate as S
import test_oracle_transport as TT
from oracle_mutants import MUTANTS, PY_MUTANTS, build_all, load, planted_module

# the pins that must fail for each planted mistake (others may fail too)
CAUGHT_BY = {
    "reverse_rate_times_Kc": ["detailed_balance"],
    "Kc_standard_state_inverted": ["detailed_balance"],
    "gibbs_entropy_sign": ["detailed_balance", "isomerisation"],
    "third_body_dropped": ["pressure_order"],
    "arrhenius_units": ["activation_energy", "troe_lindemann"],
    "falloff_without_M": ["pressure_order", "troe_lindemann"],
    "troe_centre_sign": ["troe_broadening"],
    "troe_width_constant": ["troe_broadening"],
    "nasa_h_coefficient": ["h_s_integrate_cp", "step_conservation"],
    "nasa_s_log10": ["h_s_integrate_cp"],
    "nasa_cp_power": ["h_s_integrate_cp"],
    "energy_equation_sign": ["source_conservation", "step_conservation"],
    "species_source_without_W": ["source_conservation", "isomerisation"],
    "concentration_times_W": ["detailed_balance", "isomerisation"],
    "density_without_molar_mass": ["detailed_balance"],
    "jacobian_T_row_sign": ["jacobian_complex_step"],
    "jacobian_density_term_dropped": ["jacobian_complex_step"],
    "rodas4_coefficient_digits": ["order_conditions", "linear_convergence"],
    "rodas4_error_weights": ["order_conditions"],
    "rodas4_stage_C_times_h": ["linear_convergence", "isomerisation"],
    "rodas4_gamma_dropped": ["linear_convergence", "isomerisation"],
    "lu_forward_transposed": ["linear_convergence", "isomerisation"],
    "step_acceptance_loose": ["tolerance"],
    "final_step_not_clipped": ["isomerisation", "tolerance"],
    "rk4_weight": ["rk4_brute_force"],
}


# the same for the Python oracle modules
PY_CAUGHT_BY = {
    "fvm_interpolation_weight_swapped": ["linear_diffusivity"],
    "fvm_downwind": ["uniform_flow"],
    "fvm_neighbour_flux_sign": ["closed_box", "budget"],
    "fvm_delta_dropped": ["seven_point", "linear_field"],
    "fvm_boundary_value_dropped": ["linear_field"],
    "fvm_inflow_convects_cell_value": ["budget"],
    "fvm_old_mass_new_density": ["time_term", "budget"],
    "fvm_source_without_volume": ["ldu_round_trip", "budget"],
    "fvm_ldu_lower_upper_swapped": ["ldu_round_trip"],
    "fvm_rows_diffusion_sign": ["row_form"],
    "pasr_mixing_time_without_sqrt": ["pasr_limits"],
    "pasr_factor_inverted": ["pasr_limits"],
    "wilke_mass_ratio_inverted": ["wilke_reciprocity"],
    "wilke_denominator_inverted": ["wilke_reciprocity"],
    "wilke_numerator_without_X": ["pure_limit", "wilke_identical"],
    "mathur_harmonic_not_inverted": ["pure_limit"],
    "diffusion_mole_fraction": ["binary_diffusion"],
    "diffusion_pressure_inverted": ["pressure_scaling"],
    "mole_fractions_are_mass_fractions": ["binary_diffusion", "wilke_reciprocity"],
    "gelu_grad_sign": ["gelu_forms", "finite_differences"],
    "backward_derivative_at_activation": ["finite_differences"],
    "loss_gradient_scale": ["finite_differences"],
    "hidden_activations_not_rounded": ["bf16_points"],
    "hidden_weights_not_rounded": ["bf16_points"],
    "adam_no_bias_correction": ["adam"],
    "adam_first_moment_not_carried": ["adam_constant", "adam_alternating"],
    "adam_second_moment_not_carried": ["adam_constant", "adam_alternating"],
    "adam_bias_correction_first_step": ["adam_constant", "adam_alternating"],
    "bf16_ties_down": ["bf16_known"],
    "first_layer_drops_weight_correction": ["first_layer"],
    "boxcox_inverse_exponent": ["boxcox"],
    "projection_unweighted": ["projection"],
    "projection_normal_matrix_unweighted": ["projection"],
    "newton_step_sign": ["T_from_h"],
    "heat_release_without_W": ["heat_release"],
    "features_pressure_not_logarithm": ["features"],
    "hrr_error_normalised_by_surrogate": ["hrr_error"],
    "equilibrium_pressure_sign": ["detailed_balance_off_1atm"],
    "equilibrium_mole_fractions_as_mass": ["detailed_balance"],
    "equilibrium_entropy_dropped": ["detailed_balance"],
    "hp_frozen_composition": ["long_time_equilibrium"],
}

# where the pin modules hold what they use of each oracle module: (pin module, name there, name
# in the oracle module, or None for the module itself)
_PY_TARGET = {"fvm": [(F, "fvm", None)], "transport": [(TT, "ot", None)], "mlp": [(S, "mlp", None)],
              "surrogate": [(S, "sur", None)],
              "equilibrium": [(K, "equilibrate_tp", "equilibrate_tp"), (K, "element_moles", "element_moles"),
                              (I, "equilibrate_hp", "equilibrate_hp")]}


def _py_pins(om, h2, h2_tr):
    return {
        "seven_point": F.test_uniform_diffusion_is_the_seven_point_stencil,
        "linear_field": F.test_linear_field_has_zero_laplacian_on_a_stretched_permuted_mesh,
        "closed_box": F.test_closed_box_conserves_the_species_mass,
        "uniform_flow": F.test_upwind_convection_of_a_uniform_field_through_a_uniform_flow,
        "ldu_round_trip": F.test_ldu_round_trip_and_source_term,
        "linear_diffusivity": F.test_linear_diffusivity_is_interpolated_exactly_to_the_faces,
        "time_term": F.test_time_term_alone_carries_each_cells_species_mass,
        "budget": F.test_open_box_species_budget,
        "row_form": F.test_row_form_matches_the_dense_matrix,
        "pasr_limits": F.test_pasr_limits,
        "pure_limit": lambda: TT.test_pure_species_limit(h2_tr),
        "wilke_identical": TT.test_wilke_reduces_to_pure_value_for_identical_species,
        "binary_diffusion": lambda: TT.test_binary_mixture_diffusion_identity(h2_tr),
        "pressure_scaling": lambda: TT.test_diffusion_scales_inversely_with_pressure_and_viscosity_does_not(h2_tr),
        "wilke_reciprocity": lambda: TT.test_wilke_interaction_factors_obey_reciprocity(h2_tr),
        "bf16_known": S.test_bf16_rounding_known_values,
        "gelu_forms": S.test_gelu_closed_forms,
        "first_layer": S.test_compensated_first_layer_error_bound,
        "finite_differences": S.test_backward_matches_finite_differences,
        "adam": S.test_adam_first_step_is_signed_lr,
        "adam_constant": S.test_adam_constant_gradient_three_steps,
        "adam_alternating": S.test_adam_alternating_gradient_three_steps,
        "bf16_points": S.test_bf16_emulation_rounds_where_the_gpu_holds_bf16,
        "boxcox": S.test_boxcox_roundtrip_and_log_limit,
        "features": S.test_features_are_T_log_p_and_boxcox,
        "hrr_error": S.test_heat_release_error_closed_forms,
        "projection": lambda: S.test_projection_conserves_and_is_weighted_least_squares(h2, om),
        "T_from_h": lambda: S.test_temperature_from_enthalpy(h2, om),
        "heat_release": lambda: S.test_heat_release_matches_energy_equation(h2, om),
        "detailed_balance": lambda: K.test_detailed_balance_at_gibbs_equilibrium(
            "h2", "H2", _Fixtures(om_h2=om, h2=h2)),
        "detailed_balance_off_1atm": lambda: [K.test_detailed_balance_away_from_one_atmosphere(pa, om, h2)
                                              for pa in (0.05, 40.0)],
        "long_time_equilibrium": lambda: I.test_long_time_limit_is_gibbs_equilibrium(om, h2),
    }


def _failing(pins, names):
    """The named pins that pass (should be empty)."""
    survived = []
    for pin in names:
        try:
            with np.errstate(all="ignore"):
                pins[pin]()
        except Exception:      # an assertion, or a pin's own solver giving up on the wrong arithmetic
            continue
        survived.append(pin)
    return survived


class _Fixtures:
    """Stands in for pytest's request object when a pin is called with the planted oracle."""

    def __init__(self, **kw):
        self.kw = kw

    def getfixturevalue(self, name):
        return self.kw[name]


def _pins(om, h2, ch4):
    req = _Fixtures(om_h2=om, h2=h2)
    return {
        "h_s_integrate_cp": lambda: K.test_nasa7_h_and_s_integrate_cp("h2", req),
        "source_conservation": lambda: K.test_source_terms_conserve_mass_elements_enthalpy("h2", "H2", req),
        "detailed_balance": lambda: K.test_detailed_balance_at_gibbs_equilibrium("h2", "H2", req),
        "pressure_order": lambda: K.test_reaction_order_in_pressure("h2", req),
        "activation_energy": lambda: K.test_arrhenius_apparent_activation_energy("h2", req),
        "troe_lindemann": lambda: K.test_troe_reduces_to_lindemann_and_limits(h2),
        "troe_broadening": lambda: K.test_troe_broadening_centre_and_half_widths(ch4),
        "jacobian_complex_step": lambda: K.test_jacobian_matches_complex_step("h2", "H2", req),
        "order_conditions": I.test_rodas4_order_conditions_and_L_stability,
        "linear_convergence": I.test_rodas4_convergence_order_on_linear_system,
        "isomerisation": I.test_isomerisation_closed_form,
        "rk4_brute_force": lambda: I.test_rodas4_matches_rk4_brute_force(om, h2),
        "tolerance": I.test_global_error_stays_within_the_requested_tolerance,
        "step_conservation": lambda: I.test_step_conserves_elements_and_enthalpy("h2", "H2", req),
    }


@pytest.fixture(scope="module")
def h2_transport(h2):
    from synth.transport import generate_transport
    return h2, generate_transport(h2)


@pytest.fixture(scope="module")
def mutant_libs():
    return build_all()


def test_every_mutant_has_catching_pins():
    assert set(CAUGHT_BY) == set(MUTANTS) and set(PY_CAUGHT_BY) == set(PY_MUTANTS)
    known = set(_pins(None, None, None))
    assert all(CAUGHT_BY[n] and set(CAUGHT_BY[n]) <= known for n in CAUGHT_BY)
    known = set(_py_pins(None, None, None))
    assert all(PY_CAUGHT_BY[n] and set(PY_CAUGHT_BY[n]) <= known for n in PY_CAUGHT_BY)


def test_every_pin_passes_through_the_harness_on_the_real_oracle(h2, ch4, om_h2, h2_transport):
    """The control: called through the same harness on the untouched oracle, no pin fails, so a
    failure under a planted mistake is the mistake's doing and not the harness's."""
    om = oracle.OracleMech(h2)
    failed = [pin for pin in _pins(om, h2, ch4) if not _failing(_pins(om, h2, ch4), [pin])]
    assert not failed, failed
    failed = [pin for pin in _py_pins(om_h2, h2, h2_transport)
              if not _failing(_py_pins(om_h2, h2, h2_transport), [pin])]
    assert not failed, failed


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_is_caught(name, mutant_libs, h2, ch4, monkeypatch):
    L = load(mutant_libs[name])
    monkeypatch.setattr(oracle, "_lib", L)
    om = oracle.OracleMech(h2)
    try:
        survived = _failing(_pins(om, h2, ch4), CAUGHT_BY[name])
        assert not survived, f"{name} ({MUTANTS[name][0]}) passes {survived}"
    finally:
        L.or_mech_free(om.h)
        om.h = None


@pytest.mark.parametrize("name", list(PY_MUTANTS))
def test_planted_mistake_in_python_oracle_is_caught(name, h2, om_h2, h2_transport, monkeypatch):
    planted = planted_module(name)
    for module, attr, fn in _PY_TARGET[PY_MUTANTS[name][0]]:
        monkeypatch.setattr(module, attr, planted if fn is None else getattr(planted, fn))
    survived = _failing(_py_pins(om_h2, h2, h2_transport), PY_CAUGHT_BY[name])
    assert not survived, f"{name} ({PY_MUTANTS[name][1]}) passes {survived}"
