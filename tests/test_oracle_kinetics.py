"""Pins of the oracle's thermodynamics, rates, right-hand side and Jacobian.

Each check compares the oracle with something other than itself: quadrature of its own cp for
h and s, conservation laws the exact source terms must satisfy, an independent Gibbs
minimisation (detailed balance), limiting forms of the fall-off expression, and complex-step /
finite-difference derivatives of the right-hand side for the analytic Jacobian.
"""
import numpy as np
import pytest
from scipy.integrate import quad

import oracle
from oracle.equilibrium import element_moles, equilibrate_tp
from synth.mechanism import TROE
from synth.states import PATM

from helpers import random_states


@pytest.mark.parametrize("which", ["h2", "ch4"])
def test_nasa7_h_and_s_integrate_cp(which, request):
    """h/R(T) - h/R(300) = int cp/R dT and s/R(T) - s/R(300) = int cp/(R T) dT (quadrature)."""
    om = request.getfixturevalue("om_" + which)
    for k in range(0, om.ns, max(1, om.ns // 9)):
        cpk = lambda T: om.thermo(T)[0][k]
        for T in (650.0, 1000.0, 1800.0, 3200.0):
            h1 = om.thermo(T)[1][k] * T
            h0 = om.thermo(300.0)[1][k] * 300.0
            pts = [1000.0] if T > 1000.0 else None
            Ih, _ = quad(cpk, 300.0, T, points=pts, epsabs=0, epsrel=1e-13, limit=200)
            assert abs((h1 - h0) - Ih) <= 1e-11 * abs(h1) + 1e-9
            s1 = om.thermo(T)[2][k]
            s0 = om.thermo(300.0)[2][k]
            Is, _ = quad(lambda t: cpk(t) / t, 300.0, T, points=pts, epsabs=0, epsrel=1e-13, limit=200)
            assert abs((s1 - s0) - Is) <= 1e-11 * abs(s1) + 1e-10


@pytest.mark.parametrize("which", ["h2", "ch4"])
def test_nasa7_continuity_and_range(which, request):
    om = request.getfixturevalue("om_" + which)
    a = om.thermo(1000.0 - 1e-9)
    b = om.thermo(1000.0)
    for u, v in zip(a[:3], b[:3]):
        assert np.max(np.abs(u - v)) < 1e-8
    for T in np.linspace(300.0, 3500.0, 33):
        cp = om.thermo(T)[0]
        assert np.all(cp > 3.0 - 0.1) and np.all(cp < 6.0 + 0.1)


@pytest.mark.parametrize("which,fuel", [("h2", "H2"), ("ch4", "CH4")])
def test_source_terms_conserve_mass_elements_enthalpy(which, fuel, request):
    om = request.getfixturevalue("om_" + which)
    mech = om.mech
    T, p, Y = random_states(mech, 12, 7, fuel)
    comp = np.asarray(mech.comp, np.float64)
    for i in range(T.size):
        w, q, kf, kr = om.rates(T[i], p[i], Y[:, i])
        flux = np.abs(om.W * w).sum() + 1e-300
        assert abs(np.sum(om.W * w)) <= 1e-12 * flux               # mass
        for e in range(comp.shape[1]):
            scale = np.sum(np.abs(comp[:, e] * w)) + 1e-300
            assert abs(np.sum(comp[:, e] * w)) <= 1e-12 * scale     # elements
        # enthalpy at constant p: dh/dt = cp dT/dt + sum_k h_k/W_k dY_k/dt = 0
        f = om.rhs(p[i], np.r_[T[i], Y[:, i]])
        cp_R, h_RT, _, _ = om.thermo(T[i])
        hk = om.RU * T[i] * h_RT / om.W
        terms = np.r_[om.cp_mass(T[i], Y[:, i]) * f[0], hk * f[1:]]
        assert abs(terms.sum()) <= 1e-12 * np.abs(terms).sum()


@pytest.mark.parametrize("which,fuel", [("h2", "H2"), ("ch4", "CH4")])
def test_detailed_balance_at_gibbs_equilibrium(which, fuel, request):
    """At the independent Gibbs minimum every reaction's net rate vanishes (relative to its
    forward flux): the equilibrium constants and the thermo agree."""
    om = request.getfixturevalue("om_" + which)
    mech = om.mech
    T, p, Y = random_states(mech, 4, 11, fuel, Tlo=1500.0, Thi=2500.0)
    for i in range(T.size):
        Yeq, _, info = equilibrate_tp(om, T[i], p[i], element_moles(om, Y[:, i]))
        assert info["resid"] < 1e-12
        w, q, kf, kr = om.rates(T[i], p[i], Yeq)
        C = om.density(T[i], p[i], Yeq) * Yeq / om.W
        for j in range(mech.nr):
            fwd = kf[j] * np.prod([C[k] for k in mech.reac[j] if k >= 0])
            if mech.rtype[j] == 1:
                fwd *= np.dot(mech.eff[j], C)
            if fwd > 1e-250:
                assert abs(q[j]) <= 1e-8 * fwd, (j, q[j], fwd)


@pytest.mark.parametrize("p_atm", [0.05, 40.0])
def test_detailed_balance_away_from_one_atmosphere(p_atm, om_h2, h2):
    """The same at 0.05 and 40 atm: the pressure enters the Gibbs minimisation through
    ln(p / p_atm) and the kinetics through Kc's (p_atm / RT)^dnu, independently."""
    T, _, Y = random_states(h2, 3, 13, "H2", Tlo=1500.0, Thi=2500.0)
    p = p_atm * PATM
    for i in range(T.size):
        Yeq, _, info = equilibrate_tp(om_h2, T[i], p, element_moles(om_h2, Y[:, i]))
        assert info["resid"] < 1e-12
        w, q, kf, kr = om_h2.rates(T[i], p, Yeq)
        C = om_h2.density(T[i], p, Yeq) * Yeq / om_h2.W
        for j in range(h2.nr):
            fwd = kf[j] * np.prod([C[k] for k in h2.reac[j] if k >= 0])
            if h2.rtype[j] == 1:
                fwd *= np.dot(h2.eff[j], C)
            if fwd > 1e-250:
                assert abs(q[j]) <= 1e-8 * fwd, (p_atm, j, q[j], fwd)


def _troe_mech(mech):
    j = int(np.nonzero(mech.rtype == TROE)[0][0])
    return j


def test_troe_reduces_to_lindemann_and_limits(h2):
    """With Fcent = 1 the Troe form is Lindemann, k = kinf Pr/(1+Pr); it tends to kinf at
    high pressure and to k0 [M] at low pressure."""
    m = h2.copy()
    j = _troe_mech(m)
    m.troe[j, 3] = 0.0          # a = 0
    m.troe[j, 4] = 1e300        # exp(-T/T3) = 1
    m.has_t2[j] = 0
    om = oracle.OracleMech(m)
    T = 1400.0
    Y = np.full(m.ns, 1.0 / m.ns)
    kinf = m.A[j] * T ** m.b[j] * np.exp(-m.Ea[j] / (8.314462618e7 / 4.184e7 * T))
    k0 = m.troe[j, 0] * T ** m.troe[j, 1] * np.exp(-m.troe[j, 2] / (8.314462618e7 / 4.184e7 * T))
    for p in (1e2, PATM, 1e10):
        C = om.density(T, p, Y) * Y / om.W
        M = np.dot(m.eff[j], C)
        Pr = k0 * M / kinf
        _, _, kf, _ = om.rates(T, p, Y)
        assert abs(kf[j] - kinf * Pr / (1 + Pr)) <= 1e-12 * kf[j]
    # pressure limits of the Lindemann form: kinf at high pressure, k0 [M] at low pressure
    _, _, kf_hi, _ = om.rates(T, 1e16, Y)
    assert abs(kf_hi[j] / kinf - 1.0) < 1e-3
    _, _, kf_lo, _ = om.rates(T, 1e-6, Y)
    C = om.density(T, 1e-6, Y) * Y / om.W
    assert abs(kf_lo[j] / (k0 * np.dot(m.eff[j], C)) - 1.0) < 1e-3
    # the full Troe form reaches kinf at high pressure and lies below Lindemann elsewhere
    om_full = oracle.OracleMech(h2)
    _, _, kf_full_hi, _ = om_full.rates(T, 1e16, Y)
    assert abs(kf_full_hi[j] / kinf - 1.0) < 1e-3
    _, _, kf_full, _ = om_full.rates(T, PATM, Y)
    _, _, kf_lind, _ = om.rates(T, PATM, Y)
    assert 0.0 < kf_full[j] <= kf_lind[j]


@pytest.mark.parametrize("which,fuel", [("h2", "H2"), ("ch4", "CH4")])
def test_jacobian_matches_complex_step(which, fuel, request):
    om = request.getfixturevalue("om_" + which)
    T, p, Y = random_states(om.mech, 4 if which == "ch4" else 10, 3, fuel)
    for i in range(T.size):
        y = np.r_[T[i], Y[:, i]]
        J = om.jacobian(p[i], y)
        Jc = om.jacobian_complex_step(p[i], y)
        assert np.allclose(om.rhs_complex(p[i], y).real, om.rhs(p[i], y), rtol=1e-10, atol=0)
        for c in range(J.shape[1]):
            scale = np.max(np.abs(Jc[:, c])) + 1e-300
            assert np.max(np.abs(J[:, c] - Jc[:, c])) <= 1e-10 * scale, c


def test_jacobian_matches_central_differences(om_h2, h2):
    T, p, Y = random_states(h2, 3, 5, "H2")
    for i in range(T.size):
        y = np.r_[T[i], Y[:, i]]
        J = om_h2.jacobian(p[i], y)
        for c in range(y.size):
            d = 1e-6 * max(abs(y[c]), 1e-6)
            yp = y.copy(); yp[c] += d
            ym = y.copy(); ym[c] -= d
            fd = (om_h2.rhs(p[i], yp) - om_h2.rhs(p[i], ym)) / (2 * d)
            scale = np.max(np.abs(fd)) + 1e-300
            assert np.max(np.abs(J[:, c] - fd)) <= 1e-5 * scale


def test_planted_jacobian_error_is_caught(om_h2, h2):
    """A dropped term (here: the density dependence of one column) exceeds the tolerance."""
    T, p, Y = random_states(h2, 1, 5, "H2")
    y = np.r_[T[0], Y[:, 0]]
    J = om_h2.jacobian(p[0], y)
    Jc = om_h2.jacobian_complex_step(p[0], y)
    f = om_h2.rhs(p[0], y)
    bad = J.copy()
    bad[1:, 2] -= f[1:] / (np.sum(y[1:] / om_h2.W) * om_h2.W[1])
    scale = np.max(np.abs(Jc[:, 2]))
    assert np.max(np.abs(bad[:, 2] - Jc[:, 2])) > 1e-10 * scale


RC_CAL = 8.314462618 / 4.184     # gas constant in cal/(mol K) (thermochemical calorie)


def _reactant_state(om, mech, j):
    """Equal mass fractions of reaction j's distinct reactants and nothing else."""
    Y = np.zeros(mech.ns)
    ks = sorted({int(k) for k in mech.reac[j] if k >= 0})
    Y[ks] = 1.0 / len(ks)
    return Y


@pytest.mark.parametrize("which", ["h2", "ch4"])
def test_reaction_order_in_pressure(which, request):
    """Law of mass action: with only its reactants present (no reverse flux) and T fixed, every
    concentration scales with p, so a reaction of n reactant molecules runs at a rate
    proportional to p^n, and p^(n+1) with a third body; a fall-off reaction tends to p^(n+1) at
    low pressure and to p^n at high pressure (checked to 0.01 in the exponent at 1e-25 and 1e25
    dyn/cm^2: the broadening factor approaches its limits slowly)."""
    om = request.getfixturevalue("om_" + which)
    mech = om.mech
    T = 1350.0
    for j in range(mech.nr):
        Y = _reactant_state(om, mech, j)
        n = int(np.sum(mech.reac[j] >= 0))
        order = n + (1 if mech.rtype[j] == 1 else 0)
        if mech.rtype[j] == 2:
            for p, want in ((1e-25, n + 1), (1e25, n)):
                q1 = om.rates(T, p, Y)[1][j]
                q2 = om.rates(T, 2 * p, Y)[1][j]
                assert abs(np.log2(q2 / q1) - want) < 1e-2, (j, p, np.log2(q2 / q1))
            continue
        q1 = om.rates(T, PATM, Y)[1][j]
        q2 = om.rates(T, 2 * PATM, Y)[1][j]
        assert q1 > 0.0
        assert q2 / q1 == pytest.approx(2.0 ** order, rel=1e-13), (j, q2 / q1, order)


@pytest.mark.parametrize("which", ["h2", "ch4"])
def test_arrhenius_apparent_activation_energy(which, request):
    """The apparent activation energy R T^2 d ln k/dT of k = A T^b exp(-Ea/(R T)) is Ea + b R T,
    with Ea in cal/mol; the derivative is taken by central differences of the oracle's kf."""
    om = request.getfixturevalue("om_" + which)
    mech = om.mech
    Y = np.full(mech.ns, 1.0 / mech.ns)
    for T in (800.0, 1250.0, 2100.0):
        e = 1e-5 * T
        kp = om.rates(T + e, PATM, Y)[2]
        km = om.rates(T - e, PATM, Y)[2]
        for j in range(mech.nr):
            if mech.rtype[j] == 2:
                continue
            Eapp = RC_CAL * T * T * (np.log(kp[j]) - np.log(km[j])) / (2 * e)
            want = mech.Ea[j] + mech.b[j] * RC_CAL * T
            assert abs(Eapp - want) <= 1e-6 * (abs(mech.Ea[j]) + abs(mech.b[j]) * RC_CAL * T) + 1e-4, (j, T)


def test_troe_broadening_centre_and_half_widths(ch4):
    """Troe's broadening factor (Gilbert, Luther & Troe 1983): with c = -0.4 - 0.67 log Fcent,
    N = 0.75 - 1.27 log Fcent and u = log Pr + c, log F = log Fcent / (1 + (u / (N - 0.14 u))^2).
    F equals Fcent at the centre u = 0, where it is extremal, and Fcent^(1/2) at u = N / 1.14 and
    u = -N / 0.86.  F is read from the oracle's kf as kf / (kinf Pr / (1 + Pr))."""
    om = oracle.OracleMech(ch4)
    RCv = 8.314462618e7 / 4.184e7
    for j in np.nonzero(ch4.rtype == TROE)[0][:8]:
        Y = _reactant_state(om, ch4, j)
        for T in (900.0, 1700.0):
            a, T3, T1, T2 = ch4.troe[j, 3:7]
            Fc = (1 - a) * np.exp(-T / T3) + a * np.exp(-T / T1) + (np.exp(-T2 / T) if ch4.has_t2[j] else 0.0)
            L = np.log10(Fc)
            c, N = -0.4 - 0.67 * L, 0.75 - 1.27 * L
            kinf = ch4.A[j] * T ** ch4.b[j] * np.exp(-ch4.Ea[j] / (RCv * T))
            k0 = ch4.troe[j, 0] * T ** ch4.troe[j, 1] * np.exp(-ch4.troe[j, 2] / (RCv * T))
            M1 = np.dot(ch4.eff[j], om.density(T, PATM, Y) * Y / om.W)
            Pr1 = k0 * M1 / kinf            # Pr at 1 atm; Pr is proportional to p

            def F_at(u):
                Pr = 10.0 ** (u - c)
                kf = om.rates(T, PATM * Pr / Pr1, Y)[2][j]
                return kf / (kinf * Pr / (1 + Pr))

            assert F_at(0.0) == pytest.approx(Fc, rel=1e-11)
            assert F_at(N / 1.14) == pytest.approx(np.sqrt(Fc), rel=1e-11)
            assert F_at(-N / 0.86) == pytest.approx(np.sqrt(Fc), rel=1e-11)
            for du in (-0.05, 0.05):
                assert (F_at(du) - Fc) * np.sign(L) < 0.0 or Fc == 1.0
