"""Write the flamelet tables that the synthetic quasi-DNS and LES fields interpolate.

Calls only the oracle.  There is no transport solver, so a premixed-flame profile is taken from
an adiabatic constant-pressure reactor that starts at the unburnt mixture's enthalpy
("ignition by product recirculation"):
  1. unburnt fuel/air mixture Y_u at 300 K and its HP equilibrium (T_ad, Y_ad) (Gibbs oracle);
  2. the reactor starts from the mixing state Y_e = (1 - e) Y_u + e Y_ad at the same enthalpy
     (T_e by Newton on h), with the smallest e in {0.02, 0.05, 0.1, 0.2, 0.3, 0.5} that
     ignites (T rises by >= 50 K by t_end), and is sampled at log-spaced times;
  3. progress c = (T - 300 K) / (T_end - 300 K): c in [0, c_e] is the mixing line between the
     unburnt state and Y_e, c in [c_e, 1] the reactor trajectory (made monotone);
  4. Y(c) on a uniform c grid and T(c) from h(T, Y(c)) = h(300 K, Y_u) by Newton, which the
     adiabatic reactor satisfies along its trajectory.
A mixture that never ignites is tabulated along the mixing line to its equilibrium; one without
an equilibrium temperature in range stays unburnt.
H2: stoichiometric, 257 c points.  CH4: 64 mixture fractions (Z = s^2, s uniform), 25 c points.

    python -m oracle.make_flamelet_tables
"""
import os

import numpy as np

import oracle
from oracle.equilibrium import equilibrate_hp
from oracle.surrogate import temperature_from_enthalpy
from synth.mechanism import ch4_mechanism, h2_mechanism
from synth.states import DATA_DIR, PATM, fuel_air

T_U = 300.0
MIX_SHARES = (0.02, 0.05, 0.1, 0.2, 0.3, 0.5)


def _reactor(om, T0, Y0, t_end, n_out=200):
    times = np.r_[0.0, np.logspace(-9, np.log10(t_end), n_out)]
    T = np.array([T0]); Y = Y0[:, None].copy()
    Ts, Ys = [T0], [Y0.copy()]
    for i in range(1, times.size):
        T, Y, st, _ = om.advance(T, np.array([PATM]), Y, times[i] - times[i - 1], 1e-8, 1e-12, 1)
        if st[0] != 0:
            raise RuntimeError(f"reactor failed with status {st[0]}")
        Ts.append(T[0]); Ys.append(Y[:, 0].copy())
    return np.array(Ts), np.array(Ys)


def flamelet(om, Y_u, c_grid, t_end=0.05):
    """(T(c), Y(c) [ns, nc]) for one unburnt mixture."""
    ns = Y_u.size
    h_u = om.enthalpy_mass(T_U, Y_u)
    try:
        T_ad, Y_ad = equilibrate_hp(om, T_U, PATM, Y_u, Tmin=200.0)
    except RuntimeError:
        Yc = np.repeat(Y_u[:, None], c_grid.size, axis=1)
        return np.full(c_grid.size, T_U), Yc
    traj = None
    for e in MIX_SHARES:
        Y_e = (1.0 - e) * Y_u + e * Y_ad
        T_e, ok = temperature_from_enthalpy(om, h_u, Y_e, T_U + e * (T_ad - T_U))
        if not ok:
            continue
        Ts, Ys = _reactor(om, T_e, Y_e, t_end)
        if Ts[-1] - T_e >= 50.0:
            traj = (e, Ts, Ys)
            break
    if traj is None or abs(T_ad - T_U) < 1.0:
        # mixing line from the unburnt state to its equilibrium
        c_pts = np.array([0.0, 1.0])
        Y_pts = np.stack([Y_u, Y_ad])
    else:
        e, Ts, Ys = traj
        c_tr = np.maximum.accumulate((Ts - T_U) / (Ts[-1] - T_U))
        c_tr = np.clip(c_tr, c_tr[0], 1.0)
        c_tr[-1] = 1.0
        keep = np.r_[True, np.diff(c_tr) > 0]
        c_pts = np.r_[0.0, c_tr[keep]]
        Y_pts = np.vstack([Y_u[None, :], Ys[keep]])
    Yc = np.stack([np.interp(c_grid, c_pts, Y_pts[:, k]) for k in range(ns)])
    T_c = np.zeros(c_grid.size)
    guess = T_U
    for i in range(c_grid.size):
        T_c[i], ok = temperature_from_enthalpy(om, h_u, Yc[:, i], guess)
        if not ok:
            raise RuntimeError("Newton for T(h) failed")
        guess = T_c[i]
    return T_c, Yc


def main():
    os.makedirs(DATA_DIR, exist_ok=True)
    m = h2_mechanism()
    om = oracle.OracleMech(m)
    c_grid = np.linspace(0.0, 1.0, 257)
    T_c, Y_c = flamelet(om, fuel_air(m, "H2", np.array([0.0285]))[:, 0], c_grid)
    np.savez_compressed(os.path.join(DATA_DIR, "h2_flamelet.npz"), c=c_grid, T=T_c, Y=Y_c)
    print("h2: T(c) from %.1f to %.1f K" % (T_c[0], T_c[-1]))

    m = ch4_mechanism()
    om = oracle.OracleMech(m)
    Z_grid = np.linspace(0.0, 1.0, 64) ** 2
    c_grid = np.linspace(0.0, 1.0, 25)
    TT = np.zeros((Z_grid.size, c_grid.size))
    YY = np.zeros((Z_grid.size, c_grid.size, m.ns))
    Y_u = fuel_air(m, "CH4", Z_grid)
    for i in range(Z_grid.size):
        T_c, Y_c = flamelet(om, Y_u[:, i], c_grid)
        TT[i] = T_c
        YY[i] = Y_c.T
    np.savez_compressed(os.path.join(DATA_DIR, "ch4_flamelet.npz"), Z=Z_grid, c=c_grid,
                        T=TT.astype(np.float32), Y=YY.astype(np.float32))
    print("ch4: T range %.1f .. %.1f K; max T per Z:" % (TT.min(), TT.max()),
          np.round(TT[:, -1]).astype(int).tolist())


if __name__ == "__main__":
    main()
