"""Oracle: constant-pressure, constant-enthalpy (HP) chemical equilibrium by Gibbs minimisation.

TEST INFRASTRUCTURE ONLY.  Independent of the kinetics: it shares only the NASA-7 evaluation
(``OracleMech.thermo``) with the rest of the oracle and never evaluates a rate.

Method (element potentials, the textbook dual of ideal-gas Gibbs minimisation): at fixed T
and p the minimiser of G = sum_k n_k (g_k/RT + ln(n_k/N) + ln(p/p_atm)) subject to the element
balances A n = b has mole fractions x_k = exp(sum_e a_ek lam_e - g_k/RT - ln(p/p_atm)).  The
element potentials lam and the total moles N solve  N sum_k a_ek x_k = b_e,  sum_k x_k = 1
(Newton).  An outer root-find on T matches the mixture enthalpy of the initial state.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import brentq


def element_moles(om, Y):
    """Moles of each element per gram of mixture: b_e = sum_k a_ek Y_k / W_k."""
    comp = np.asarray(om.mech.comp, np.float64)
    return comp.T @ (np.asarray(Y, np.float64) / om.W)


def equilibrate_tp(om, T, p, b, lam0=None, tol=1e-14, max_iter=200):
    """Equilibrium mass fractions at fixed T, p for element moles b (per gram).

    Elements with b_e == 0 are removed together with every species that contains them.
    Returns (Y, lam, info).
    """
    comp = np.asarray(om.mech.comp, np.float64)
    present = b > 0
    keep = np.all(comp[:, ~present] == 0, axis=1)
    A = comp[keep][:, present]                 # [nk, ne']
    bb = b[present]
    cp, h_RT, s_R, _ = om.thermo(T)
    g = (h_RT - s_R)[keep] + np.log(p / om.PATM)
    ne = A.shape[1]
    if lam0 is None:
        # initial guess: potentials reproducing a uniform-ish mixture of the species
        lam, *_ = np.linalg.lstsq(A, g - np.log(1.0 / A.shape[0]), rcond=None)
        lnN = np.log(bb.sum() / max(A.sum(axis=1).mean(), 1.0))
    else:
        lam, lnN = lam0[0].copy(), lam0[1]
    info = {"iters": 0, "resid": np.inf}
    for it in range(max_iter):
        z = A @ lam - g
        z = np.minimum(z, 700.0)
        x = np.exp(z)
        N = np.exp(lnN)
        n = N * x
        r = np.r_[(A.T @ n) / bb - 1.0, x.sum() - 1.0]
        info["resid"] = float(np.max(np.abs(r)))
        info["iters"] = it
        if info["resid"] < tol:
            break
        Jm = np.zeros((ne + 1, ne + 1))
        Jm[:ne, :ne] = (A.T * n) @ A / bb[:, None]
        Jm[:ne, ne] = (A.T @ n) / bb
        Jm[ne, :ne] = A.T @ x
        Jm[ne, ne] = 0.0
        d = np.linalg.solve(Jm, -r)
        step = np.max(np.abs(d))
        if step > 2.0:
            d *= 2.0 / step
        lam = lam + d[:ne]
        lnN = lnN + d[ne]
    x_full = np.zeros(om.ns)
    x_full[keep] = np.exp(np.minimum(A @ lam - g, 700.0))
    Y = x_full * om.W
    Y /= Y.sum()
    return Y, (lam, lnN), info


def equilibrate_hp(om, T0, p, Y0, Tmax=5000.0, Tmin=300.0, dT=50.0):
    """Adiabatic constant-pressure equilibrium of the state (T0, p, Y0): returns (T, Y).

    The element potentials are continued downward in T from Tmax (where every species is
    abundant and Newton converges from a crude start) until h_eq(T) - h0 changes sign; the
    bracket is then refined with Brent's method from warm starts.
    """
    Y0 = np.asarray(Y0, np.float64)
    b = element_moles(om, Y0)
    h0 = om.enthalpy_mass(T0, Y0)
    lam = None
    prev = None
    bracket = None
    for T in np.arange(Tmax, Tmin - 1e-9, -dT):
        Y, lam, info = equilibrate_tp(om, T, p, b, lam)
        if info["resid"] > 1e-10:
            raise RuntimeError(f"element-potential Newton failed at T={T}: {info}")
        r = om.enthalpy_mass(T, Y) - h0
        if prev is not None and np.sign(r) != np.sign(prev[1]):
            bracket = (T, prev[0], lam)
            break
        prev = (T, r, lam)
    if bracket is None:
        raise RuntimeError("no adiabatic equilibrium temperature in range")
    lam_w = bracket[2]

    def resid(T):
        Y, _, info = equilibrate_tp(om, T, p, b, lam_w)
        return om.enthalpy_mass(T, Y) - h0

    T = brentq(resid, bracket[0], bracket[1], xtol=1e-12, rtol=1e-15, maxiter=200)
    Y, _, info = equilibrate_tp(om, T, p, b, lam_w)
    return T, Y
