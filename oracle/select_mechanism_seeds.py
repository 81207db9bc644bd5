"""Pick the mechanism seeds used by the synthetic workloads (calls only the oracle).

A seed is accepted when the stoichiometric fuel/air mixture
  * has an adiabatic, constant-pressure equilibrium temperature from 300 K in [1950, 2800] K
    (HP Gibbs minimisation, oracle/equilibrium.py) with N2 mass fraction >= 0.6,
  * (CH4 only) has CO2 mass fraction >= 0.05 at that equilibrium,
  * ignites in the oracle reactor: T rises by >= 400 K within 1 ms from 1000 K (H2) / 1200 K (CH4).
The first accepted seed from 12345 upward is printed for each kind.

    python -m oracle.select_mechanism_seeds
"""
import numpy as np

import oracle
from oracle.equilibrium import equilibrate_hp
from synth.mechanism import generate_mechanism
from synth.states import PATM, fuel_air


def accept(kind, seed):
    m = generate_mechanism(kind, seed)
    om = oracle.OracleMech(m)
    fuel = "H2" if kind == "h2" else "CH4"
    Zst = 0.0285 if kind == "h2" else 0.0552
    Y = fuel_air(m, fuel, np.array([Zst]))[:, 0]
    try:
        Tad, Yeq = equilibrate_hp(om, 300.0, PATM, Y)
    except RuntimeError:
        return False
    if not (1950.0 <= Tad <= 2800.0 and Yeq[m.index("N2")] >= 0.6):
        return False
    if kind == "ch4" and Yeq[m.index("CO2")] < 0.05:
        return False
    T0 = 1000.0 if kind == "h2" else 1200.0
    y1, st, _, _ = om.rodas4(PATM, np.r_[T0, Y], 1e-3)
    return st == 0 and y1[0] - T0 >= 400.0


if __name__ == "__main__":
    for kind in ("h2", "ch4"):
        seed = 12345
        while not accept(kind, seed):
            seed += 1
        print(kind, seed)
