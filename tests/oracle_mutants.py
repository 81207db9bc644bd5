"""Planted mistakes in the oracle, for the mutation tests (test infrastructure).

Each entry names a plausible mistake (a dropped term, a wrong sign, constant or index, a
transposed operand) as text replacements in a copy of an oracle source (chem_oracle.cpp, or one
of the Python modules fvm.py, transport.py, mlp.py, surrogate.py), applied in every place the
same arithmetic appears, so that the copy stays self-consistent where the original is (a
mistake made the same way in the rates and in the analytic Jacobian is the hard case for the
pins).  Every replacement stays inside the arrays it touches.  The C copies are compiled beside
the oracle's own build; the Python copies are executed as fresh module objects.  The oracle's
files are never changed."""
import ctypes
import os
import subprocess
import types
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "chem_oracle.cpp")
OUT = os.path.join(ROOT, "oracle", "_build", "mutants")

# name -> (what is wrong, [(original text, planted text, occurrences)])
MUTANTS = {
    "reverse_rate_times_Kc": ("reverse rate constant kf Kc instead of kf / Kc",
                              [("S kr = kf / Kc;", "S kr = kf * Kc;", 1)]),
    "Kc_standard_state_inverted": ("Kc with (R T / p0)^dnu instead of (p0 / (R T))^dnu",
                                   [("pow(S(PATM) / (S(RU) * T), S((double)dnu))",
                                     "pow(S(RU) * T / S(PATM), S((double)dnu))", 1)]),
    "gibbs_entropy_sign": ("products' s/R added to the Gibbs change instead of subtracted",
                           [("if (kp >= 0) { dG += h_RT[kp] - s_R[kp]; dnu += 1; }",
                             "if (kp >= 0) { dG += h_RT[kp] + s_R[kp]; dnu += 1; }", 1)]),
    "third_body_dropped": ("third-body rate without [M], in the rates and the Jacobian alike",
                           [("if (m.rtype[j] == 1) q = q * M;", "if (m.rtype[j] == 1) q = q;", 1),
                            ("if (m.rtype[j] == 1) v = e.M * v + S(m.eff[(size_t)j * ns + k]) * (e.fwd - e.rev);",
                             "if (m.rtype[j] == 1) v = v;", 1),
                            ("if (m.rtype[j] == 1) dqdT = e.M * dqdT;", "if (m.rtype[j] == 1) dqdT = dqdT;", 1)]),
    "arrhenius_units": ("Ea divided by R in erg instead of cal, in the rates and the Jacobian alike",
                        [("exp(-S(m.Ea[j]) / (S(RC) * T))", "exp(-S(m.Ea[j]) / (S(RU) * T))", 1),
                         ("const double Ta = m.Ea[j] / RC;", "const double Ta = m.Ea[j] / RU;", 1)]),
    "falloff_without_M": ("fall-off reduced pressure k0 / kinf without [M]",
                          [("S Pr = k0 * M / kf;", "S Pr = k0 / kf;", 1),
                           ("S Pr = k0 * e.M / kinf;", "S Pr = k0 / kinf;", 1)]),
    "troe_centre_sign": ("Troe c = -0.4 + 0.67 log Fcent, rates and Jacobian alike",
                         [("S c = S(-0.4) - S(0.67) * L;", "S c = S(-0.4) + S(0.67) * L;", 2),
                          ("S(-0.67) * d", "S(0.67) * d", 1),
                          ("S(-1.27 + 0.14 * 0.67)", "S(-1.27 - 0.14 * 0.67)", 1)]),
    "troe_width_constant": ("Troe N = 0.75 - 1.72 log Fcent, rates and Jacobian alike",
                            [("S n = S(0.75) - S(1.27) * L;", "S n = S(0.75) - S(1.72) * L;", 2),
                             ("S(-1.27 + 0.14 * 0.67)", "S(-1.72 + 0.14 * 0.67)", 1)]),
    "nasa_h_coefficient": ("h/RT with a3 T^2 / 2 instead of a3 T^2 / 3",
                           [("S(a[2]) * T2 / S(3.0)", "S(a[2]) * T2 / S(2.0)", 1)]),
    "nasa_s_log10": ("s/R with a1 log10 T instead of a1 ln T",
                     [("s_R[k] = S(a[0]) * log(T)", "s_R[k] = S(a[0]) * log10(T)", 1)]),
    "nasa_cp_power": ("cp/R with a4 T^2 instead of a4 T^3",
                      [("S(a[3]) * T3 + S(a[4]) * T4;", "S(a[3]) * T2 + S(a[4]) * T4;", 1)]),
    "energy_equation_sign": ("dT/dt = +sum h wdot / (rho cp)",
                             [("f[0] = -Q / (rho * cp);", "f[0] = Q / (rho * cp);", 1)]),
    "species_source_without_W": ("dY/dt = wdot / rho without the molar mass",
                                 [("f[k + 1] = S(m.W[k]) * wdot[k] / rho;", "f[k + 1] = wdot[k] / rho;", 1)]),
    "concentration_times_W": ("C = rho Y W instead of rho Y / W, rates and Jacobian alike",
                              [("C[k] = rho * Y[k] / S(m.W[k]);", "C[k] = rho * Y[k] * S(m.W[k]);", 2)]),
    "density_without_molar_mass": ("rho = p / (R T) without the mean molar mass, everywhere",
                                   [("S rho = p / (S(RU) * T * sumYW);", "S rho = p / (S(RU) * T);", 3)]),
    "jacobian_T_row_sign": ("Jacobian dT'/dT with the heat-capacity term's sign flipped",
                            [("J[0] = -num / rcp + Q / (rcp * rcp) * drcp_dT;",
                              "J[0] = -num / rcp - Q / (rcp * rcp) * drcp_dT;", 1)]),
    "jacobian_density_term_dropped": ("Jacobian dY'/dT without the density's temperature dependence",
                                      [("J[(size_t)(k + 1) * N + 0] = S(m.W[k]) / rho * dWdTY[k] + fk / T;",
                                        "J[(size_t)(k + 1) * N + 0] = S(m.W[k]) / rho * dWdTY[k];", 1)]),
    "rodas4_coefficient_digits": ("Rodas4 C21 with two digits swapped",
                                  [("{-5.6688, 0, 0, 0, 0, 0},", "{-5.6868, 0, 0, 0, 0, 0},", 1)]),
    "rodas4_error_weights": ("Rodas4 error estimate from stage 5 instead of stage 6",
                             [("const double RD_E[6] = {0, 0, 0, 0, 0, 1.0};",
                               "const double RD_E[6] = {0, 0, 0, 0, 1.0, 0};", 1)]),
    "rodas4_stage_C_times_h": ("stage right-hand side with C_ij h instead of C_ij / h",
                               [("v += S(RD_C[s][j]) / h * u[(size_t)j * N + i];",
                                 "v += S(RD_C[s][j]) * h * u[(size_t)j * N + i];", 1)]),
    "rodas4_gamma_dropped": ("iteration matrix I / h - J instead of I / (gamma h) - J",
                             [("S ig = S(1.0) / (S(RD_GAMMA) * h);", "S ig = S(1.0) / h;", 1)]),
    "lu_forward_transposed": ("forward substitution reads the upper triangle (transposed index)",
                              [("for (int j = 0; j < i; ++j) x[i] -= a[(size_t)i * N + j] * x[j];",
                                "for (int j = 0; j < i; ++j) x[i] -= a[(size_t)j * N + i] * x[j];", 1)]),
    "step_acceptance_loose": ("steps accepted with an error norm up to 100 instead of 1",
                              [("if (env <= 1.0) {", "if (env <= 100.0) {", 1)]),
    "final_step_not_clipped": ("the last step runs its full length past the end of the interval",
                               [("if (re(h) >= dt - re(t)) { h = S(dt) - t; last = true; }",
                                 "if (re(h) >= dt - re(t)) { last = true; }", 1)]),
    "rk4_weight": ("brute-force RK4 with weight 1 on k3 instead of 2",
                   [("2.0 * k2[i] + 2.0 * k3[i] + k4[i]", "2.0 * k2[i] + k3[i] + k4[i]", 1)]),
}


def planted_source(name):
    text = open(SRC).read()
    for old, new, count in MUTANTS[name][1]:
        found = text.count(old)
        if found != count:
            raise ValueError(f"{name}: {old!r} occurs {found} times, expected {count}")
        text = text.replace(old, new)
    return text


def build(name):
    """Compile the planted copy beside the oracle's own build (same compiler and flags)."""
    os.makedirs(OUT, exist_ok=True)
    src = os.path.join(OUT, f"{name}.cpp")
    lib = os.path.join(OUT, f"{name}.so")
    text = planted_source(name)
    if not (os.path.exists(src) and open(src).read() == text and os.path.exists(lib)):
        # private names while building, so that concurrent test processes never share a file
        tag = f".{os.getpid()}"
        with open(src + tag, "w") as f:
            f.write(text)
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
                               "-I", os.path.join(ROOT, "oracle"), "-x", "c++", "-o", lib + tag, src + tag])
        os.replace(lib + tag, lib)
        os.replace(src + tag, src)
    return lib


def build_all(names=None, workers=None):
    names = list(MUTANTS) if names is None else names
    with ThreadPoolExecutor(max_workers=workers or min(8, os.cpu_count() or 1)) as ex:
        return dict(zip(names, ex.map(build, names)))


def load(path):
    import oracle
    return oracle.declare(ctypes.CDLL(path))


# Python oracle modules: name -> (module, what is wrong, [(original, planted, occurrences)])
PY_MUTANTS = {
    "fvm_interpolation_weight_swapped": ("fvm", "face gamma with the owner's weight on the neighbour",
        [("g = mesh.weight[f] * gamma[o] + (1.0 - mesh.weight[f]) * gamma[nb]",
          "g = mesh.weight[f] * gamma[nb] + (1.0 - mesh.weight[f]) * gamma[o]", 2)]),
    "fvm_downwind": ("fvm", "convected value taken from the downwind cell",
        [("up = o if F >= 0.0 else nb", "up = nb if F >= 0.0 else o", 1),
         ("if Fout >= 0.0:\n                    row[P] += Fout\n                else:\n                    row[other] += Fout",
          "if Fout >= 0.0:\n                    row[other] += Fout\n                else:\n                    row[P] += Fout", 1)]),
    "fvm_neighbour_flux_sign": ("fvm", "the neighbour's row gains the face flux instead of losing it",
        [("A[nb, up] -= F", "A[nb, up] += F", 1),
         ("Fout = phi[f] if o == P else -phi[f]", "Fout = phi[f]", 1)]),
    "fvm_delta_dropped": ("fvm", "diffusion coefficient without the delta coefficient",
        [("a = g * mesh.mag_sf[f] * mesh.delta[f]", "a = g * mesh.mag_sf[f]", 2)]),
    "fvm_boundary_value_dropped": ("fvm", "fixed-value boundary diffusion without the boundary value",
        [("            s[P] += a * Y_b[b]", "            s[P] += 0.0 * a * Y_b[b]", 1),
         ("                s += a * Y_b[b]", "                s += 0.0 * a * Y_b[b]", 1)]),
    "fvm_inflow_convects_cell_value": ("fvm", "an inflow face convects the cell's value",
        [("                s[P] -= phi_b[b] * Y_b[b]", "                A[P, P] += phi_b[b]", 1),
         ("                    s -= phi_b[b] * Y_b[b]", "                    row[P] += phi_b[b]", 1)]),
    "fvm_old_mass_new_density": ("fvm", "old species mass with the new density",
        [("s[P] += rho_old[P] * Y_old[P] * V[P] / dt", "s[P] += rho[P] * Y_old[P] * V[P] / dt", 1),
         ("s += rho_old[P] * Y_old[P] * V[P] / dt", "s += rho[P] * Y_old[P] * V[P] / dt", 1)]),
    "fvm_source_without_volume": ("fvm", "chemistry source not integrated over the cell volume",
        [("s += V * k * S", "s += k * S", 1),
         ("s += V[P] * (1.0 if kappa is None else kappa[P]) * S[P]",
          "s += (1.0 if kappa is None else kappa[P]) * S[P]", 1)]),
    "fvm_ldu_lower_upper_swapped": ("fvm", "lower and upper exchanged in the ldu split",
        [("return A[nb, o].copy(), A[o, nb].copy(), np.diag(A).copy()",
          "return A[o, nb].copy(), A[nb, o].copy(), np.diag(A).copy()", 1)]),
    "fvm_rows_diffusion_sign": ("fvm", "the row form adds the neighbour's diffusion coefficient",
        [("                row[other] -= a\n", "                row[other] += a\n", 1)]),
    "pasr_mixing_time_without_sqrt": ("fvm", "mixing time without the square root",
        [("tmix = c_mix * np.sqrt(mu_eff[i] / (rho[i] * eps[i]))",
          "tmix = c_mix * mu_eff[i] / (rho[i] * eps[i])", 1)]),
    "pasr_factor_inverted": ("fvm", "kappa = tau_mix / (tau_c + tau_mix)",
        [("kappa[i] = tau_c[i] / (tau_c[i] + tmix)", "kappa[i] = tmix / (tau_c[i] + tmix)", 1)]),
    "wilke_mass_ratio_inverted": ("transport", "Wilke's factor with (W_k / W_j)^(1/4)",
        [("(W[j] / W[k]) ** 0.25", "(W[k] / W[j]) ** 0.25", 1)]),
    "wilke_denominator_inverted": ("transport", "Wilke's factor with (8 (1 + W_j / W_k))^(1/2)",
        [("np.sqrt(8.0 * (1.0 + W[k] / W[j]))", "np.sqrt(8.0 * (1.0 + W[j] / W[k]))", 1)]),
    "wilke_numerator_without_X": ("transport", "mixture viscosity sums mu_k / den without X_k",
        [("mu = float(np.sum(X * mu_k / mu_den))", "mu = float(np.sum(mu_k / mu_den))", 1)]),
    "mathur_harmonic_not_inverted": ("transport", "Mathur average with sum X / lambda not inverted",
        [("1.0 / float(np.sum(X / lam_k))", "float(np.sum(X / lam_k))", 1)]),
    "diffusion_mole_fraction": ("transport", "D_km = (1 - X_k) / ... instead of (1 - Y_k)",
        [("Dm[k] = (1.0 - Y[k]) / s", "Dm[k] = (1.0 - X[k]) / s", 1)]),
    "diffusion_pressure_inverted": ("transport", "D proportional to p instead of 1 / p",
        [("* (PATM / p)", "* (p / PATM)", 1)]),
    "mole_fractions_are_mass_fractions": ("transport", "X = Y",
        [("X = (Y / W) / np.sum(Y / W)", "X = Y / np.sum(Y)", 1)]),
    "gelu_grad_sign": ("mlp", "GELU derivative with the density term's sign flipped",
        [("+ x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)",
          "- x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)", 1)]),
    "backward_derivative_at_activation": ("mlp", "GELU derivative taken at the activation",
        [('dz = da * gelu_grad(cache["z"][l - 1])', 'dz = da * gelu_grad(cache["a"][l])', 1)]),
    "loss_gradient_scale": ("mlp", "loss gradient divided by the batch only",
        [("dz = 2.0 * (out - target) / (M * n_out)", "dz = 2.0 * (out - target) / M", 1)]),
    "hidden_activations_not_rounded": ("mlp", "BF16 emulation leaves the hidden activations unrounded",
        [("            a = rnd(gelu(z))\n            acts.append(a)\n", "            a = gelu(z)\n            acts.append(a)\n", 1)]),
    "hidden_weights_not_rounded": ("mlp", "BF16 emulation leaves the weights of layers 2-5 unrounded",
        [("        W = rnd(Ws[l])\n", "        W = np.asarray(Ws[l], np.float64)\n", 1)]),
    "adam_no_bias_correction": ("mlp", "Adam's first moment without bias correction",
        [("mh = m[i] / (1.0 - beta1 ** step)", "mh = m[i]", 1)]),
    "adam_first_moment_not_carried": ("mlp", "Adam's first moment without the b1 m carry",
        [("m[i] = beta1 * m[i] + (1.0 - beta1) * grads[i]", "m[i] = (1.0 - beta1) * grads[i]", 1)]),
    "adam_second_moment_not_carried": ("mlp", "Adam's second moment without the b2 v carry",
        [("v[i] = beta2 * v[i] + (1.0 - beta2) * grads[i] * grads[i]",
          "v[i] = (1.0 - beta2) * grads[i] * grads[i]", 1)]),
    "adam_bias_correction_first_step": ("mlp", "Adam's bias correction frozen at step 1",
        [("mh = m[i] / (1.0 - beta1 ** step)", "mh = m[i] / (1.0 - beta1)", 1),
         ("vh = v[i] / (1.0 - beta2 ** step)", "vh = v[i] / (1.0 - beta2)", 1)]),
    "bf16_ties_down": ("mlp", "BF16 rounding with ties always down",
        [("bias = ((u >> 16) & 1) + 0x7FFF", "bias = 0x7FFF + 0 * u", 1)]),
    "first_layer_drops_weight_correction": ("mlp", "compensated first layer without x_hi W_lo",
        [("return xh @ wh.T + xl @ wh.T + xh @ wl.T", "return xh @ wh.T + xl @ wh.T", 1)]),
    "boxcox_inverse_exponent": ("surrogate", "Box-Cox inverse with exponent lambda",
        [("np.power(base, 1.0 / lam)", "np.power(base, lam)", 1)]),
    "projection_unweighted": ("surrogate", "projection without the D weighting, consistently",
        [("G = (A * D[None, :]) @ A.T", "G = A @ A.T", 1),
         ("Ypp = Yp - D * (A.T @ lam)", "Ypp = Yp - (A.T @ lam)", 1)]),
    "projection_normal_matrix_unweighted": ("surrogate", "normal matrix without D, update with D",
        [("G = (A * D[None, :]) @ A.T", "G = A @ A.T", 1)]),
    "newton_step_sign": ("surrogate", "Newton on T stepping the wrong way",
        [("        T -= dT", "        T += dT", 1)]),
    "heat_release_without_W": ("surrogate", "heat release with molar enthalpies times mass fractions",
        [("hk * (np.asarray(Y1) - np.asarray(Y0)) / om.W", "hk * (np.asarray(Y1) - np.asarray(Y0))", 1)]),
    "features_pressure_not_logarithm": ("surrogate", "pressure feature p instead of ln p",
        [("np.log(np.asarray(p))[:, None]", "np.asarray(p, np.float64)[:, None]", 1)]),
    "hrr_error_normalised_by_surrogate": ("surrogate", "heat-release error divided by the surrogate's field",
        [("return float(np.sum(np.abs(q_sur - q_ref)) / np.sum(np.abs(q_ref)))",
          "return float(np.sum(np.abs(q_sur - q_ref)) / np.sum(np.abs(q_sur)))", 1)]),
    "equilibrium_pressure_sign": ("equilibrium", "Gibbs function with - ln(p / p_atm)",
        [("g = (h_RT - s_R)[keep] + np.log(p / om.PATM)", "g = (h_RT - s_R)[keep] - np.log(p / om.PATM)", 1)]),
    "equilibrium_mole_fractions_as_mass": ("equilibrium", "equilibrium mole fractions returned as mass fractions",
        [("    Y = x_full * om.W\n", "    Y = x_full * 1.0\n", 1)]),
    "equilibrium_entropy_dropped": ("equilibrium", "Gibbs function h/RT without - s/R",
        [("g = (h_RT - s_R)[keep] + np.log(p / om.PATM)", "g = (h_RT - 0.0 * s_R)[keep] + np.log(p / om.PATM)", 1)]),
    "hp_frozen_composition": ("equilibrium", "adiabatic temperature from the initial composition's enthalpy",
        [("        r = om.enthalpy_mass(T, Y) - h0\n", "        r = om.enthalpy_mass(T, Y0) - h0\n", 1),
         ("        return om.enthalpy_mass(T, Y) - h0\n", "        return om.enthalpy_mass(T, Y0) - h0\n", 1)]),
}


def planted_module(name):
    """A fresh module object holding the planted copy of one Python oracle module."""
    mod, _, reps = PY_MUTANTS[name]
    path = os.path.join(ROOT, "oracle", mod + ".py")
    text = open(path).read()
    for old, new, count in reps:
        found = text.count(old)
        if found != count:
            raise ValueError(f"{name}: {old!r} occurs {found} times, expected {count}")
        text = text.replace(old, new)
    m = types.ModuleType(f"oracle.{mod}")
    m.__file__ = path
    m.__package__ = "oracle"
    exec(compile(text, f"{path} [{name}]", "exec"), m.__dict__)
    return m
