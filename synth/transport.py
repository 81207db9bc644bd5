"""Seeded synthetic transport data for the synthetic mechanisms (input generation only).

The paper's Thermo class evaluates the transport properties of every cell from temperature
polynomials (§3.1); the real mechanisms and their transport data are not available.  This module
draws a Lennard-Jones-like diameter sigma_k and well depth eps_k for every species (seeded; both
grow with the molar mass), evaluates the Chapman-Enskog pure-species viscosity and binary
diffusion coefficients (Hirschfelder, Curtiss & Bird) with the reduced collision integrals of
Neufeld, Janzen & Aziz (J. Chem. Phys. 57, 1100, 1972), and a modified-Eucken conductivity
lambda_k = mu_k / W_k (cp_k + 1.25 R), and fits ln mu_k, ln lambda_k and ln D_jk (at 1 atm) as
cubic polynomials in ln T on [300, 3000] K.  The fitted coefficients are the transport data:
the GPU kernels and the oracle both start from them and nothing else.

Units: mu g/(cm s), lambda erg/(cm s K), D cm^2/s at p_atm (D scales as p_atm / p).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

RU = 8.314462618e7            # erg / (mol K)
T_FIT = np.linspace(300.0, 3000.0, 60)


@dataclass
class TransportData:
    mu_poly: np.ndarray       # [ns, 4]: ln mu = sum_n c_n (ln T)^n
    lambda_poly: np.ndarray   # [ns, 4]
    diff_poly: np.ndarray     # [ns, ns, 4] symmetric: ln D_jk(p_atm)

    @property
    def ns(self):
        return self.mu_poly.shape[0]


def omega22(ts):
    return 1.16145 * ts ** -0.14874 + 0.52487 * np.exp(-0.77320 * ts) + 2.16178 * np.exp(-2.43787 * ts)


def omega11(ts):
    return (1.06036 * ts ** -0.15610 + 0.19300 * np.exp(-0.47635 * ts) + 1.03587 * np.exp(-1.52996 * ts)
            + 1.76474 * np.exp(-3.89411 * ts))


def _cp_R(mech, T):
    """cp/R of every species from the NASA-7 fits, [ns, nT]."""
    out = np.empty((mech.ns, T.size))
    for k in range(mech.ns):
        for i, t in enumerate(T):
            a = mech.nasa_lo[k] if t < 1000.0 else mech.nasa_hi[k]
            out[k, i] = a[0] + t * (a[1] + t * (a[2] + t * (a[3] + t * a[4])))
    return out


def _fit(lnT, values_ln):
    V = np.stack([np.ones_like(lnT), lnT, lnT ** 2, lnT ** 3], axis=1)
    c, *_ = np.linalg.lstsq(V, values_ln, rcond=None)
    return c


def generate_transport(mech, seed=2024):
    rng = np.random.default_rng(seed)
    W = np.asarray(mech.W, np.float64)
    ns = mech.ns
    # sigma in Angstrom and eps/k_B in K, growing with molar mass, with seeded scatter
    sigma = 2.5 + 1.1 * np.log1p(W / 4.0) * rng.uniform(0.85, 1.15, ns)
    eps = 60.0 + 55.0 * np.log1p(W / 4.0) ** 1.5 * rng.uniform(0.8, 1.25, ns)
    T = T_FIT
    lnT = np.log(T)
    mu = np.empty((ns, T.size))
    for k in range(ns):
        mu[k] = 2.6693e-5 * np.sqrt(W[k] * T) / (sigma[k] ** 2 * omega22(T / eps[k]))
    lam = mu / W[:, None] * RU * (_cp_R(mech, T) + 1.25)
    mu_poly = np.stack([_fit(lnT, np.log(mu[k])) for k in range(ns)])
    lambda_poly = np.stack([_fit(lnT, np.log(lam[k])) for k in range(ns)])
    diff_poly = np.empty((ns, ns, 4))
    for j in range(ns):
        for k in range(j, ns):
            s = 0.5 * (sigma[j] + sigma[k])
            e = np.sqrt(eps[j] * eps[k])
            D = 0.0018583 * np.sqrt(T ** 3 * (1.0 / W[j] + 1.0 / W[k])) / (s ** 2 * omega11(T / e))
            c = _fit(lnT, np.log(D))
            diff_poly[j, k] = c
            diff_poly[k, j] = c
    return TransportData(mu_poly=mu_poly, lambda_poly=lambda_poly, diff_poly=diff_poly)
