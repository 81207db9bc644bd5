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


def with_inert_argon(mech):
    """The mechanism with an inert argon appended (one more species and one more element): a
    species and element count the fixed-size kernel instances do not cover, so the runtime-width
    paths run.  Argon's NASA-7 polynomial is the monatomic ideal gas: cp/R = 5/2 in both ranges,
    h(298.15 K) = 0 (a6 = -5/2 * 298.15) and a7 = 4.366 (its standard entropy); third-body
    efficiency 1."""
    m = mech.copy()
    m.name = mech.name + "+AR"
    m.elements = list(mech.elements) + ["AR"]
    m.elem_mass = np.append(mech.elem_mass, 39.948)
    comp = np.zeros((mech.ns + 1, mech.ne + 1), mech.comp.dtype)
    comp[:mech.ns, :mech.ne] = mech.comp
    comp[mech.ns, mech.ne] = 1
    m.comp = comp
    m.species = list(mech.species) + ["AR"]
    m.W = np.append(mech.W, 39.948)
    ar = np.array([2.5, 0.0, 0.0, 0.0, 0.0, -2.5 * 298.15, 4.366])
    m.nasa_lo = np.vstack([mech.nasa_lo, ar])
    m.nasa_hi = np.vstack([mech.nasa_hi, ar])
    m.eff = np.hstack([mech.eff, np.ones((mech.nr, 1))])
    if mech.hf_R is not None:
        m.hf_R = np.append(mech.hf_R, 0.0)
    if mech.s0_R is not None:
        m.s0_R = np.append(mech.s0_R, 2.5 * np.log(298.15) + 4.366)
    return m


def with_inert_species(mech, k):
    """The mechanism with k inert species appended, AR_1 .. AR_k made of 1 .. k argon atoms (one
    more element; molar masses 39.948 i, so no two columns of the Jacobian coincide), each with
    argon's monatomic NASA-7 polynomial and third-body efficiency 1.  CH4 with 11 of them has
    N = 65 unknowns, beyond the 64 rows of the register-held triangular solves and the panel LU,
    so the shared-memory LU and sweeps run."""
    m = mech.copy()
    m.name = f"{mech.name}+{k}inert"
    m.elements = list(mech.elements) + ["AR"]
    m.elem_mass = np.append(mech.elem_mass, 39.948)
    comp = np.zeros((mech.ns + k, mech.ne + 1), mech.comp.dtype)
    comp[:mech.ns, :mech.ne] = mech.comp
    comp[mech.ns:, mech.ne] = np.arange(1, k + 1)
    m.comp = comp
    m.species = list(mech.species) + [f"AR_{i}" for i in range(1, k + 1)]
    m.W = np.append(mech.W, 39.948 * np.arange(1, k + 1))
    ar = np.array([2.5, 0.0, 0.0, 0.0, 0.0, -2.5 * 298.15, 4.366])
    m.nasa_lo = np.vstack([mech.nasa_lo] + [ar] * k)
    m.nasa_hi = np.vstack([mech.nasa_hi] + [ar] * k)
    m.eff = np.hstack([mech.eff, np.ones((mech.nr, k))])
    if mech.hf_R is not None:
        m.hf_R = np.append(mech.hf_R, np.zeros(k))
    if mech.s0_R is not None:
        m.s0_R = np.append(mech.s0_R, np.full(k, 2.5 * np.log(298.15) + 4.366))
    return m
