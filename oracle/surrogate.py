"""Oracle: the surrogate's transforms and physics post-processing, written out plainly.

TEST INFRASTRUCTURE ONLY.

* Box-Cox transform of mass fractions, lambda = 0.1: BC(y) = (y^lam - 1) / lam for y >= 0
  (negative y clipped to 0 first) and its inverse y = max(0, 1 + lam z)^(1/lam).
* Features x = [T, ln p, BC(Y_1..Y_ns)]; network outputs are z-scored increments of BC(Y).
* Element-conservation projection: with A_ek = a_ek M_e / W_k (mass of element e per mass of
  species k) and b = A Y0, the corrected composition is the D^{-1}-weighted least-squares
  projection Y'' = Y' - D A^T (A D A^T)^{-1} (A Y' - b), D = diag(Y' + 1e-12), then clipped at 0.
* Temperature from enthalpy conservation at constant p: Newton on h(T, Y'') = h(T0, Y0), the
  operation the paper's Thermo class performs (§3.1).
* Heat-release rate of a step: q = -rho0 sum_k h_k(T0) dY_k / (W_k dt), h_k molar.
"""
from __future__ import annotations

import numpy as np

LAMBDA = 0.1


def boxcox(y, lam=LAMBDA):
    y = np.maximum(np.asarray(y, np.float64), 0.0)
    return (np.power(y, lam) - 1.0) / lam


def boxcox_inv(z, lam=LAMBDA):
    base = np.maximum(1.0 + lam * np.asarray(z, np.float64), 0.0)
    return np.power(base, 1.0 / lam)


def features(T, p, Y):
    """x [n, ns + 2] from T [n], p [n], Y [ns, n]."""
    return np.concatenate([np.asarray(T)[:, None], np.log(np.asarray(p))[:, None],
                           boxcox(np.asarray(Y)).T], axis=1)


def element_mass_matrix(mech):
    comp = np.asarray(mech.comp, np.float64)       # [ns, ne]
    W = comp @ np.asarray(mech.elem_mass, np.float64)
    return (comp * np.asarray(mech.elem_mass)[None, :] / W[:, None]).T   # [ne, ns]


def project(mech, Y0, Yp):
    """Element-conservation projection of one cell's composition (vectors of length ns)."""
    A = element_mass_matrix(mech)
    b = A @ Y0
    D = np.asarray(Yp, np.float64) + 1e-12
    r = A @ Yp - b
    G = (A * D[None, :]) @ A.T
    lam = np.linalg.solve(G, r)
    Ypp = Yp - D * (A.T @ lam)
    Ypp = np.maximum(Ypp, 0.0)
    ok = (np.max(np.abs(A @ Ypp - b)) <= 1e-9) and (abs(Ypp.sum() - np.sum(Y0)) <= 1e-9)
    return Ypp, bool(ok)


def temperature_from_enthalpy(om, h0, Y, T_guess, tol=1e-9, max_iter=50):
    """Newton iteration T <- T - (h(T, Y) - h0) / cp(T, Y).  Returns (T, ok)."""
    T = float(T_guess)
    for _ in range(max_iter):
        dT = (om.enthalpy_mass(T, Y) - h0) / om.cp_mass(T, Y)
        T -= dT
        if not (200.0 <= T <= 6000.0):
            return T, False
        if abs(dT) < tol * T:
            return T, True
    return T, False


def heat_release(om, T0, p, Y0, Y1, dt):
    """q = -rho0 sum_k h_k(T0) (Y1_k - Y0_k) / (W_k dt)  (erg / cm^3 / s) for one cell."""
    _, h_RT, _, _ = om.thermo(T0)
    rho0 = om.density(T0, p, Y0)
    hk = om.RU * T0 * h_RT
    return -rho0 * float(np.sum(hk * (np.asarray(Y1) - np.asarray(Y0)) / om.W)) / dt


def hrr_error(q_sur, q_ref):
    """Field L1-relative heat-release error: sum |q_sur - q_ref| / sum |q_ref|."""
    q_sur = np.asarray(q_sur); q_ref = np.asarray(q_ref)
    return float(np.sum(np.abs(q_sur - q_ref)) / np.sum(np.abs(q_ref)))
