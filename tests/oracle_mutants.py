"""Planted mistakes in the oracle's C source, for the mutation tests (test infrastructure).

Each entry names a plausible mistake (a dropped term, a wrong sign, constant or index, a
transposed operand) as text replacements in a copy of chem_oracle.cpp, applied in every place
the same arithmetic appears, so that the copy stays self-consistent where the original is (a
mistake made the same way in the rates and in the analytic Jacobian is the hard case for the
pins).  Every replacement stays inside the arrays it touches."""
import ctypes
import os
import subprocess
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
        with open(src, "w") as f:
            f.write(text)
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
                               "-I", os.path.join(ROOT, "oracle"), "-o", lib + ".tmp", src])
        os.replace(lib + ".tmp", lib)
    return lib


def build_all(names=None, workers=None):
    names = list(MUTANTS) if names is None else names
    with ThreadPoolExecutor(max_workers=workers or min(8, os.cpu_count() or 1)) as ex:
        return dict(zip(names, ex.map(build, names)))


def load(path):
    import oracle
    return oracle.declare(ctypes.CDLL(path))
