"""Seeded synthetic reactor states shaped like the paper's two flames (input generation only).

The paper's fields (the 3D reactive Taylor-Green vortex quasi-DNS of §4.1 and the Cambridge
stratified burner LES of §4.2) are not available; these generators stand in for them:

* ``mixing_states``: H2/air mixture fraction Z ~ U[0, 1], T ~ U[900, 2200] K, p = 1 atm, with a
  seeded half of the cells flagged for partial reaction over t ~ logU[1e-7, 1e-3] s (the
  caller advances those cells with a reactor of its choice).
* ``quasi_dns_field``: a 128^3 grid (x fastest; 128 x 128 x nz for more than 2^21 cells)
  carrying a train of planar premixed fronts,
  c(x) = (1 + tanh(s(x)/delta))/2 with two fronts per 32-cell period and delta = 2 cells,
  mapped through a tabulated flamelet (T(c), Y(c)), then multiplied by seeded Gaussian random
  fields (correlation length 8 cells): T by (1 + 0.05 g), each Y_k by (1 + 0.10 g_k), and Y
  renormalised to sum 1.
* ``les_field``: mixture fraction Z ~ Beta(mean 0.3, var 0.05), progress c ~ U[0, 1], mapped
  through a flamelet table over (Z, c), then 5 % multiplicative T noise clipped to [300, 2200] K.

The flamelet tables are data files written by oracle/make_flamelet_tables.py.  This module only
interpolates and perturbs; it evaluates no thermodynamics or kinetics.
"""
from __future__ import annotations

import os

import numpy as np

PATM = 1.01325e6
AIR_O2 = 0.233
AIR_N2 = 0.767
DATA_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")


def fuel_air(mech, fuel, Z):
    """Mass fractions [ns, n] of a fuel/air mixture with mixture fraction Z (fuel mass share)."""
    Z = np.asarray(Z, np.float64)
    Y = np.zeros((mech.ns, Z.shape[0]))
    Y[mech.index(fuel)] = Z
    Y[mech.index("O2")] = AIR_O2 * (1.0 - Z)
    Y[mech.index("N2")] = AIR_N2 * (1.0 - Z)
    return Y


def mixing_states(mech, n, seed, fuel="H2"):
    """Random mixing states (the small H2 parity workload).

    Returns dict(T [n], p [n], Y [ns, n], react [n] bool, t_react [n]).
    """
    rng = np.random.default_rng(seed)
    Z = rng.uniform(0.0, 1.0, n)
    T = rng.uniform(900.0, 2200.0, n)
    p = np.full(n, PATM)
    Y = fuel_air(mech, fuel, Z)
    react = np.zeros(n, bool)
    react[rng.permutation(n)[: n // 2]] = True
    t_react = 10.0 ** rng.uniform(-7.0, -3.0, n)
    return {"T": T, "p": p, "Y": Y, "react": react, "t_react": t_react}


def gaussian_random_field(shape, corr_len, rng):
    """Unit-variance periodic Gaussian random field by spectral filtering of white noise."""
    noise = rng.standard_normal(shape)
    k = [np.fft.fftfreq(n) * 2.0 * np.pi for n in shape]
    kk = np.zeros(shape)
    for ax, kv in enumerate(k):
        sh = [1] * len(shape)
        sh[ax] = -1
        kk = kk + kv.reshape(sh) ** 2
    filt = np.exp(-0.5 * kk * corr_len ** 2)
    g = np.real(np.fft.ifftn(np.fft.fftn(noise) * filt))
    g -= g.mean()
    return g / g.std()


def load_table(name):
    with np.load(os.path.join(DATA_DIR, name)) as d:
        return {k: d[k].astype(np.float64) for k in d.files}


def _interp_profile(c_grid, vals, c):
    """vals [m, nc] tabulated on c_grid -> [m, n] at c."""
    return np.stack([np.interp(c, c_grid, v) for v in vals])


def quasi_dns_field(table, n=1 << 20, seed=12346, grid=128, period=32, delta=2.0, corr_len=8.0):
    """Quasi-DNS-shaped H2 field: the first n cells (x fastest) of a grid^3 box."""
    rng = np.random.default_rng(seed)
    nz = -(-n // (grid * grid))
    shape = (max(grid, nz), grid, grid)  # indexed [z, y, x]; taller than grid^3 beyond 2^21 cells
    x = np.arange(grid)
    s = period / 4.0 - np.abs((x % period) - period / 2.0)
    c_x = 0.5 * (1.0 + np.tanh(s / delta))
    c = np.broadcast_to(c_x[None, None, :], (nz, grid, grid)).reshape(-1)[:n]
    T = np.interp(c, table["c"], table["T"])
    Y = _interp_profile(table["c"], table["Y"], c)
    gT = gaussian_random_field(shape, corr_len, rng)[:nz].reshape(-1)[:n]
    T = T * (1.0 + 0.05 * gT)
    for k in range(Y.shape[0]):
        gk = gaussian_random_field(shape, corr_len, rng)[:nz].reshape(-1)[:n]
        Y[k] = np.maximum(Y[k] * (1.0 + 0.10 * gk), 0.0)
    Y /= Y.sum(axis=0, keepdims=True)
    return {"T": T, "p": np.full(n, PATM), "Y": Y, "c": c}


def flamelet_samples(table, n, seed, front_fraction=0.0, delta=2.0, half_width=8.0):
    """Independent samples of the quasi-DNS state distribution (no spatial structure) with the
    same T and Y perturbation amplitudes.  Used for training data.  Progress variable: c ~ U[0, 1]
    for a share 1 - front_fraction of the samples; the rest sample c across a resolved front,
    c = (1 + tanh(s / delta)) / 2 with s ~ U[-half_width, half_width] cells, the density of c in
    the quasi-DNS field (concentrated near the unburnt and burnt ends)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.0, 1.0, n)
    nf = int(round(front_fraction * n))
    if nf > 0:
        s = rng.uniform(-half_width, half_width, nf)
        c[rng.permutation(n)[:nf]] = 0.5 * (1.0 + np.tanh(s / delta))
    T = np.interp(c, table["c"], table["T"]) * (1.0 + 0.05 * rng.standard_normal(n))
    Y = _interp_profile(table["c"], table["Y"], c)
    Y = np.maximum(Y * (1.0 + 0.10 * rng.standard_normal(Y.shape)), 0.0)
    Y /= Y.sum(axis=0, keepdims=True)
    return {"T": T, "p": np.full(n, PATM), "Y": Y, "c": c}


def beta_params(mean, var):
    f = mean * (1.0 - mean) / var - 1.0
    return mean * f, (1.0 - mean) * f


def les_field(table, n=262144, seed=12347, z_mean=0.3, z_var=0.05, t_noise=0.05):
    """LES-shaped CH4 field from a (Z, c) flamelet table."""
    rng = np.random.default_rng(seed)
    a, b = beta_params(z_mean, z_var)
    Z = rng.beta(a, b, n)
    c = rng.uniform(0.0, 1.0, n)
    zg, cg = table["Z"], table["c"]
    TT, YY = table["T"], table["Y"]        # [nZ, nc], [nZ, nc, ns]
    iz = np.clip(np.searchsorted(zg, Z) - 1, 0, zg.size - 2)
    ic = np.clip(np.searchsorted(cg, c) - 1, 0, cg.size - 2)
    wz = np.clip((Z - zg[iz]) / (zg[iz + 1] - zg[iz]), 0.0, 1.0)
    wc = np.clip((c - cg[ic]) / (cg[ic + 1] - cg[ic]), 0.0, 1.0)

    def bil(F):
        f00 = F[iz, ic]; f01 = F[iz, ic + 1]; f10 = F[iz + 1, ic]; f11 = F[iz + 1, ic + 1]
        wz_ = wz.reshape((-1,) + (1,) * (F.ndim - 2)); wc_ = wc.reshape((-1,) + (1,) * (F.ndim - 2))
        return (1 - wz_) * ((1 - wc_) * f00 + wc_ * f01) + wz_ * ((1 - wc_) * f10 + wc_ * f11)

    T = bil(TT)
    Y = np.maximum(bil(YY), 0.0).T         # [ns, n]
    Y /= Y.sum(axis=0, keepdims=True)
    T = np.clip(T * (1.0 + t_noise * rng.standard_normal(n)), 300.0, 2200.0)
    return {"T": T, "p": np.full(n, PATM), "Y": Y, "Z": Z, "c": c}
