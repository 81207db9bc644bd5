"""Mutation tests of the oracle's pins: each plausible mistake planted in a copy of the oracle's
C source (tests/oracle_mutants.py) must make the pins named for it fail, so that the pins are
known to detect a dropped term, a wrong sign, constant or index, or a transposed operand in every
part of the kinetics and the integrator, including mistakes made consistently in the rates and
in the analytic Jacobian.  The mistakes are planted on the CPU, in copies built beside the
oracle; the oracle itself is untouched."""
import numpy as np
import pytest

import oracle
import test_oracle_integrator as I
import test_oracle_kinetics as K
from oracle_mutants import MUTANTS, build_all, load

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
    "rk4_weight": ["rk4_brute_force"],
}


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
        "step_conservation": lambda: I.test_step_conserves_elements_and_enthalpy("h2", "H2", req),
    }


@pytest.fixture(scope="module")
def mutant_libs():
    return build_all()


def test_every_mutant_has_catching_pins():
    assert set(CAUGHT_BY) == set(MUTANTS)
    known = set(_pins(None, None, None))
    assert all(CAUGHT_BY[n] and set(CAUGHT_BY[n]) <= known for n in CAUGHT_BY)


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_is_caught(name, mutant_libs, h2, ch4, monkeypatch):
    L = load(mutant_libs[name])
    monkeypatch.setattr(oracle, "_lib", L)
    om = oracle.OracleMech(h2)
    try:
        pins = _pins(om, h2, ch4)
        survived = []
        for pin in CAUGHT_BY[name]:
            try:
                with np.errstate(all="ignore"):
                    pins[pin]()
            except Exception:      # an assertion, or a pin's own solver giving up on the wrong arithmetic
                continue
            survived.append(pin)
        assert not survived, f"{name} ({MUTANTS[name][0]}) passes {survived}"
    finally:
        L.or_mech_free(om.h)
        om.h = None
