"""Shared test helpers: seeded state sets built from the generators and the oracle."""
import numpy as np

from synth.states import PATM, fuel_air, mixing_states


def random_states(mech, n, seed, fuel, Tlo=900.0, Thi=2200.0, radicals=1e-3):
    """Seeded mixtures with some radicals sprinkled in (exercises every reaction)."""
    rng = np.random.default_rng(seed)
    Z = rng.uniform(0.0, 0.3 if fuel == "CH4" else 0.6, n)
    Y = fuel_air(mech, fuel, Z)
    Y += radicals * rng.uniform(0.0, 1.0, Y.shape)
    Y /= Y.sum(axis=0, keepdims=True)
    T = rng.uniform(Tlo, Thi, n)
    return T, np.full(n, PATM), Y


def prereacted_mixing_states(om, mech, n, seed):
    """The small H2 parity workload: mixing states, half partially reacted by the oracle."""
    st = mixing_states(mech, n, seed)
    T, p, Y = st["T"].copy(), st["p"], st["Y"].copy()
    idx = np.nonzero(st["react"])[0]
    T1, Y1, status = om.advance_dt(T[idx], p[idx], Y[:, idx], st["t_react"][idx], 1e-8, 1e-14)
    assert np.all(status == 0)
    T[idx] = T1
    Y[:, idx] = Y1
    return T, p, Y
