"""Oracle: mixture-averaged transport properties of a cell, written out plainly.

TEST INFRASTRUCTURE ONLY.

The paper's Thermo class (§3.1) evaluates thermophysical and transport properties from
temperature polynomials; it prints no formula.  The standard mixture-averaged model is restated
here, per cell, in FP64:

* pure species (fits from the transport data): ln mu_k = sum_n a_kn (ln T)^n, same for lambda_k,
  ln D_jk(p_atm) = sum_n d_jkn (ln T)^n, and D_jk(p) = D_jk(p_atm) p_atm / p;
* mole fractions X_k = (Y_k / W_k) / sum_j Y_j / W_j;
* viscosity, Wilke's rule: mu = sum_k X_k mu_k / sum_j X_j Phi_kj with
  Phi_kj = (1 + (mu_k / mu_j)^(1/2) (W_j / W_k)^(1/4))^2 / (8 (1 + W_k / W_j))^(1/2);
* conductivity, the Mathur-Saxena average: lambda = (sum_k X_k lambda_k + 1 / sum_k X_k / lambda_k) / 2;
* mixture-averaged diffusion coefficients D_km = (1 - Y_k) / sum_{j != k} X_j / D_jk; for a cell
  that holds species k alone (the sum vanishes) D_km is the self-diffusion fit D_kk.
"""
from __future__ import annotations

import numpy as np

PATM = 1.01325e6


def _poly(c, lnT):
    return c[..., 0] + lnT * (c[..., 1] + lnT * (c[..., 2] + lnT * c[..., 3]))


def pure_species(tr, T, p):
    """(mu_k [ns], lambda_k [ns], D_jk [ns, ns]) at one state."""
    lnT = np.log(T)
    mu = np.exp(_poly(tr.mu_poly, lnT))
    lam = np.exp(_poly(tr.lambda_poly, lnT))
    D = np.exp(_poly(tr.diff_poly, lnT)) * (PATM / p)
    return mu, lam, D


def mixture(tr, W, T, p, Y):
    """(mu, lambda, D_km [ns]) of one cell (T K, p dyn/cm^2, mass fractions Y [ns])."""
    W = np.asarray(W, np.float64)
    Y = np.asarray(Y, np.float64)
    ns = W.size
    mu_k, lam_k, D = pure_species(tr, T, p)
    X = (Y / W) / np.sum(Y / W)
    mu_den = np.zeros(ns)
    for k in range(ns):
        for j in range(ns):
            phi = (1.0 + np.sqrt(mu_k[k] / mu_k[j]) * (W[j] / W[k]) ** 0.25) ** 2 / np.sqrt(8.0 * (1.0 + W[k] / W[j]))
            mu_den[k] += X[j] * phi
    mu = float(np.sum(X * mu_k / mu_den))
    lam = 0.5 * (float(np.sum(X * lam_k)) + 1.0 / float(np.sum(X / lam_k)))
    Dm = np.empty(ns)
    for k in range(ns):
        s = 0.0
        for j in range(ns):
            if j != k:
                s += X[j] / D[j, k]
        Dm[k] = (1.0 - Y[k]) / s if s > 0.0 else D[k, k]
    return mu, lam, Dm


def mixture_cells(tr, W, T, p, Y):
    """Vectorised over cells by a plain loop: T [n], p [n], Y [ns, n] -> mu [n], lambda [n], D [ns, n]."""
    n = np.asarray(T).size
    mu = np.empty(n)
    lam = np.empty(n)
    D = np.empty((np.asarray(W).size, n))
    for i in range(n):
        mu[i], lam[i], D[:, i] = mixture(tr, W, T[i], p[i], Y[:, i])
    return mu, lam, D
