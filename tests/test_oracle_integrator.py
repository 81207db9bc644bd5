"""Pins of the oracle's Rodas4 integrator.

* the tableau satisfies the Rosenbrock order conditions (order 4, embedded order 3) and is
  L-stable, R(inf) = 0 (Hairer & Wanner, Solving ODEs II, §IV.7);
* fixed-step convergence order 4 on a linear system against the matrix exponential;
* the closed-form relaxation of an isomerisation A <=> B with equal enthalpies;
* brute-force classical RK4 with tiny steps on small cells;
* element and enthalpy conservation over a step; special cases (all rates zero, dt -> 0,
  equilibrium input, non-finite input);
* the long-time limit equals an independent HP Gibbs minimisation.
"""
import numpy as np
import pytest
from scipy.linalg import expm

import oracle
from oracle.equilibrium import equilibrate_hp
from synth.mechanism import Mechanism
from synth.states import PATM, fuel_air

from helpers import prereacted_mixing_states, random_states


def _standard_form():
    g, A, C, M, E = oracle.rodas4_tableau()
    Ginv = np.diag(np.full(6, 1.0 / g)) - C
    Gam = np.linalg.inv(Ginv)             # gamma_ij including the diagonal gamma
    alpha = A @ Gam
    b = M @ Gam
    bh = (M - E) @ Gam
    return g, alpha, Gam, b, bh


def test_rodas4_order_conditions_and_L_stability():
    g, alpha, Gam, b, bh = _standard_form()
    beta = alpha + np.tril(Gam, -1)      # strictly lower beta_ij = alpha_ij + gamma_ij
    ai = alpha.sum(axis=1)
    bp = beta.sum(axis=1)

    def conds(w):
        return np.array([
            w.sum() - 1.0,
            w @ bp - (0.5 - g),
            w @ ai ** 2 - 1.0 / 3.0,
            w @ (beta @ bp) - (1.0 / 6.0 - g + g * g),
            w @ ai ** 3 - 0.25,
            w @ (ai * (alpha @ bp)) - (1.0 / 8.0 - g / 3.0),
            w @ (beta @ ai ** 2) - (1.0 / 12.0 - g / 3.0),
            w @ (beta @ (beta @ bp)) - (1.0 / 24.0 - g / 2.0 + 1.5 * g * g - g ** 3),
        ])

    assert np.max(np.abs(conds(b))) < 1e-10
    assert np.max(np.abs(conds(bh)[:4])) < 1e-10      # embedded method: order 3
    assert np.max(np.abs(conds(bh)[4:])) > 1e-6        # ... and not order 4
    B = alpha + Gam
    R_inf = 1.0 - b @ np.linalg.solve(B, np.ones(6))
    assert abs(R_inf) < 1e-12


def test_rodas4_convergence_order_on_linear_system():
    rng = np.random.default_rng(0)
    Q = np.linalg.qr(rng.standard_normal((5, 5)))[0]
    L = Q @ np.diag([-1.0, -3.0, -10.0, -0.5, -2.0]) @ Q.T
    y0 = rng.standard_normal(5)
    exact = expm(L * 1.0) @ y0
    errs = []
    for n in (8, 16, 32):
        y, _ = oracle.rodas4_linear(L, y0, 1.0 / n, n)
        errs.append(np.max(np.abs(y - exact)))
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    for r in ratios:
        assert 12.0 < r < 22.0, ratios        # 2^4 = 16
    # stiff component decays to zero in one huge step (L-stability)
    Ls = np.diag([-1e12, -1.0])
    y, _ = oracle.rodas4_linear(Ls, np.array([1.0, 1.0]), 1.0, 1)
    assert abs(y[0]) < 1e-10


def _isomer_mech():
    lo = np.array([3.5, 1e-4, 0.0, 0.0, 0.0, -1000.0, 5.0])
    hi = lo.copy()
    mA = lo.copy(); mB = lo.copy(); mB[6] = 5.7       # equal h and cp, different entropy
    return Mechanism(
        name="iso", elements=["O"], species=["A", "B"], comp=np.array([[2], [2]], np.int32),
        elem_mass=np.array([15.999]), W=np.array([31.998, 31.998]),
        nasa_lo=np.stack([mA, mB]), nasa_hi=np.stack([mA, mB]),
        rtype=np.array([0], np.int32), reac=np.array([[0, -1, -1]], np.int32),
        prod=np.array([[1, -1, -1]], np.int32), A=np.array([3e5]), b=np.array([0.3]),
        Ea=np.array([8000.0]), troe=np.zeros((1, 7)), has_t2=np.zeros(1, np.int32),
        eff=np.ones((1, 2)))


def test_isomerisation_closed_form():
    m = _isomer_mech()
    om = oracle.OracleMech(m)
    T0, p = 1300.0, PATM
    Y0 = np.array([0.8, 0.2])
    _, _, kf, kr = om.rates(T0, p, Y0)
    ksum = kf[0] + kr[0]
    Yeq = kr[0] / ksum
    for dt in (1e-7, 3e-6, 1e-4):
        y, st, nsub, _ = om.rodas4(p, np.r_[T0, Y0], dt, 1e-11, 1e-15)
        assert st == 0
        exact = Yeq + (Y0[0] - Yeq) * np.exp(-ksum * dt)
        assert abs(y[1] - exact) < 1e-9
        assert y[0] == pytest.approx(T0, abs=1e-9)


def test_global_error_stays_within_the_requested_tolerance():
    """The adaptive control delivers the accuracy it is asked for: on the isomerisation with its
    closed-form solution, over one and five relaxation times and at rtol from 1e-3 to 1e-6, the
    global error of Y_B stays below rtol (Y_B is of order one)."""
    m = _isomer_mech()
    om = oracle.OracleMech(m)
    T0, p = 1300.0, PATM
    Y0 = np.array([0.8, 0.2])
    _, _, kf, kr = om.rates(T0, p, Y0)
    ksum = kf[0] + kr[0]
    Yeq = kr[0] / ksum
    for n_tau in (1.0, 5.0):
        dt = n_tau / ksum
        exact = Yeq + (Y0[0] - Yeq) * np.exp(-ksum * dt)
        for rtol in (1e-3, 1e-4, 1e-5, 1e-6):
            y, st, _, _ = om.rodas4(p, np.r_[T0, Y0], dt, rtol, 1e-20)
            assert st == 0
            assert abs(y[1] - exact) <= rtol, (n_tau, rtol, abs(y[1] - exact))


def test_rodas4_matches_rk4_brute_force(om_h2, h2):
    T, p, Y = prereacted_mixing_states(om_h2, h2, 16, 12345)
    dt = 1e-6
    for i in range(0, 16, 2):
        y0 = np.r_[T[i], Y[:, i]]
        rho = np.max(np.abs(np.linalg.eigvals(om_h2.jacobian(p[i], y0))))
        n = int(max(2000, np.ceil(10.0 * rho * dt)))
        if n > 400000:
            continue
        y_rk = om_h2.rk4(p[i], y0, dt, n)
        y_rk2 = om_h2.rk4(p[i], y0, dt, 2 * n)
        assert np.max(np.abs(y_rk - y_rk2)[1:]) < 1e-11
        y_ro, st, _, _ = om_h2.rodas4(p[i], y0, dt, 1e-10, 1e-14)
        assert st == 0
        assert abs(y_ro[0] - y_rk2[0]) <= 1e-8 * y_rk2[0]
        assert np.max(np.abs(y_ro[1:] - y_rk2[1:])) <= 1e-8 * np.max(y_rk2[1:])


@pytest.mark.parametrize("which,fuel", [("h2", "H2"), ("ch4", "CH4")])
def test_step_conserves_elements_and_enthalpy(which, fuel, request):
    om = request.getfixturevalue("om_" + which)
    mech = om.mech
    T, p, Y = random_states(mech, 6, 21, fuel)
    comp = np.asarray(mech.comp, np.float64)
    # elements are linear invariants: conserved to rounding at any tolerance; the enthalpy is a
    # nonlinear invariant: conserved to the integration tolerance
    for rtol, htol in ((1e-6, 1e-6), (1e-10, 1e-9)):
        T1, Y1, st, _ = om.advance(T, p, Y, 1e-6, rtol, rtol * 1e-4)
        assert np.all(st == 0)
        for i in range(T.size):
            b0 = comp.T @ (Y[:, i] / om.W)
            b1 = comp.T @ (Y1[:, i] / om.W)
            assert np.max(np.abs(b1 - b0)) <= 1e-12 * np.max(b0)
            h0 = om.enthalpy_mass(T[i], Y[:, i])
            h1 = om.enthalpy_mass(T1[i], Y1[:, i])
            scale = om.cp_mass(T[i], Y[:, i]) * T[i]
            assert abs(h1 - h0) <= htol * scale


def test_special_cases(om_h2, h2):
    T, p, Y = random_states(h2, 8, 4, "H2")
    # all rate constants zero -> output bitwise equal to the input
    m0 = h2.copy()
    m0.A[:] = 0.0
    m0.troe[:, 0] = 0.0
    om0 = oracle.OracleMech(m0)
    T1, Y1, st, nsub = om0.advance(T, p, Y, 1e-6)
    assert np.all(st == 0)
    assert np.array_equal(T1, T) and np.array_equal(Y1, Y)
    # vanishing step: the increment is f(y0) dt to first order
    dt = 1e-15
    T2, Y2, st, _ = om_h2.advance(T, p, Y, dt)
    assert np.all(st == 0)
    for i in range(T.size):
        f = om_h2.rhs(p[i], np.r_[T[i], Y[:, i]])
        dy = np.r_[T2[i] - T[i], Y2[:, i] - Y[:, i]]
        assert np.all(np.abs(dy - f * dt) <= 1e-5 * np.abs(f * dt) + 1e-13 * np.abs(np.r_[T[i], Y[:, i]]))
    # equilibrium input stays put within atol
    Teq, Yeq = equilibrate_hp(om_h2, 1800.0, PATM, Y[:, 0])
    y, st, _, _ = om_h2.rodas4(PATM, np.r_[Teq, Yeq], 1e-6)
    assert st == 0
    assert np.max(np.abs(y[1:] - Yeq)) < 1e-10 and abs(y[0] - Teq) < 1e-6
    # non-finite inputs are reported and left unchanged
    Tn = T.copy(); Yn = Y.copy()
    Tn[1] = np.nan; Yn[3, 2] = np.inf
    T3, Y3, st, _ = om_h2.advance(Tn, p, Yn, 1e-6)
    assert st[1] == oracle.NONFINITE and st[2] == oracle.NONFINITE
    assert np.isnan(T3[1]) and np.isinf(Y3[3, 2]) and np.all(st[[0, 3, 4]] == 0)


def test_long_time_limit_is_gibbs_equilibrium(om_h2, h2):
    for Z, T0 in ((0.0285, 1500.0), (0.02, 2000.0)):
        Y0 = fuel_air(h2, "H2", np.array([Z]))[:, 0]
        Teq, Yeq = equilibrate_hp(om_h2, T0, PATM, Y0)
        y = np.r_[T0, Y0]
        t = 0.0
        for t_next in np.logspace(-9, 3, 49):
            y, st, _, _ = om_h2.rodas4(PATM, y, t_next - t, 1e-10, 1e-16)
            assert st == 0
            t = t_next
        assert abs(y[0] - Teq) <= 1e-6 * Teq
        assert np.max(np.abs(y[1:] - Yeq)) <= 1e-6 * np.max(Yeq)


def test_op_counts_are_consistent(om_h2, h2):
    T, p, Y = random_states(h2, 1, 2, "H2")
    counts, st, nsub, nrej = om_h2.count_ops(p[0], np.r_[T[0], Y[:, 0]], 1e-6)
    assert st == 0 and nsub >= 1
    _, st2, nsub2, nrej2 = om_h2.rodas4(p[0], np.r_[T[0], Y[:, 0]], 1e-6)
    assert (nsub, nrej) == (nsub2, nrej2)
    assert counts["exp"] > 0 and counts["add"] > 0 and counts["mul"] > 0
