"""Oracle: implicit finite-volume assembly of a species equation and the PaSR factor, written out
plainly (dense matrices, loops over faces and cells).

TEST INFRASTRUCTURE ONLY.

Species equation of one species over one step dt (the paper's species PDE, §3.1; implicit Euler
in time, upwind convection, the Laplacian term of Alg. 1), for the new value Y of every cell P:

  (rho_P Y_P - rho_P^old Y_P^old) V_P / dt                    (time derivative)
  + sum over the faces f of P of F_f(Y)                        (convection, upwind)
  - sum over internal faces f of P of a_f (Y_N - Y_P)         (diffusion, Alg. 1)
  - sum over fixed-value boundary faces b of P of a_b (Y_b - Y_P)
  = V_P kappa_P S_P                                            (chemistry source, PaSR-scaled)

with, on an internal face f between owner o and neighbour n:
  gamma_f = w_f gamma_o + (1 - w_f) gamma_n      (Alg. 1: linear interpolation of gamma = rho D)
  a_f = gamma_f |S_f| delta_f                     (Alg. 1: the upper and lower entry magnitude)
  mass flux phi_f from o to n; the flux out of o is phi_f, out of n is -phi_f; the convected value
  is the upwind cell's: Y_o if phi_f >= 0, else Y_n;
on a boundary face b of cell P: a_b = gamma_b |S_b| delta_b on fixed-value faces (zero-gradient
faces carry no diffusive flux); outward mass flux phi_b convects Y_P if phi_b >= 0 (outflow) and
the boundary value Y_b otherwise (inflow).

As a linear system A Y = s in the paper's ldu form (lower/upper per internal face, diag per cell,
source per cell): upper_f = A[o, n], lower_f = A[n, o].

PaSR (§2: the LES closes sub-grid turbulence-chemistry interaction with a partially stirred
reactor; the paper only cites its formula): kappa = tau_c / (tau_c + tau_mix) with
tau_mix = C_mix sqrt(mu_eff / (rho eps)), the Smagorinsky sub-grid viscosity
nu_sgs = (C_s Delta)^2 |S|, mu_eff = mu + rho nu_sgs and eps = nu_sgs |S|^2 (the sub-grid
dissipation that balances production).  tau_c is the caller's chemical time scale.
"""
from __future__ import annotations

import numpy as np


def species_matrix(mesh, dt=0.0, rho=None, rho_old=None, Y_old=None, phi=None, phi_b=None,
                   gamma=None, gamma_b=None, Y_b=None, S=None, kappa=None):
    """Dense A [n, n] and right-hand side s [n]; a term is left out when its inputs are None
    (dt <= 0: no time derivative)."""
    n = mesh.n_cells
    A = np.zeros((n, n))
    s = np.zeros(n)
    V = mesh.volume
    if dt > 0.0:
        for P in range(n):
            A[P, P] += rho[P] * V[P] / dt
            s[P] += rho_old[P] * Y_old[P] * V[P] / dt
    for f in range(mesh.owner.size):
        o, nb = int(mesh.owner[f]), int(mesh.neighbour[f])
        if phi is not None:
            F = phi[f]
            # row o: flux out of o is F; row n: flux out of n is -F
            up = o if F >= 0.0 else nb
            A[o, up] += F
            A[nb, up] -= F
        if gamma is not None:
            g = mesh.weight[f] * gamma[o] + (1.0 - mesh.weight[f]) * gamma[nb]
            a = g * mesh.mag_sf[f] * mesh.delta[f]
            A[o, o] += a
            A[o, nb] -= a
            A[nb, nb] += a
            A[nb, o] -= a
    for b in range(mesh.b_cell.size):
        P = int(mesh.b_cell[b])
        if phi_b is not None:
            if phi_b[b] >= 0.0:
                A[P, P] += phi_b[b]
            else:
                s[P] -= phi_b[b] * Y_b[b]
        if gamma is not None and mesh.b_type[b] == 1:
            a = gamma_b[b] * mesh.b_mag_sf[b] * mesh.b_delta[b]
            A[P, P] += a
            s[P] += a * Y_b[b]
    if S is not None:
        k = np.ones(n) if kappa is None else kappa
        s += V * k * S
    return A, s


def species_rows(mesh, cells, dt=0.0, rho=None, rho_old=None, Y_old=None, phi=None, phi_b=None,
                 gamma=None, gamma_b=None, Y_b=None, S=None, kappa=None):
    """The same equation for selected cells only (large meshes): {cell: ({column: value}, s)}."""
    out = {}
    V = mesh.volume
    for P in cells:
        P = int(P)
        row = {P: 0.0}
        s = 0.0
        if dt > 0.0:
            row[P] += rho[P] * V[P] / dt
            s += rho_old[P] * Y_old[P] * V[P] / dt
        for f in np.nonzero((mesh.owner == P) | (mesh.neighbour == P))[0]:
            o, nb = int(mesh.owner[f]), int(mesh.neighbour[f])
            other = nb if o == P else o
            row.setdefault(other, 0.0)
            if phi is not None:
                Fout = phi[f] if o == P else -phi[f]
                if Fout >= 0.0:
                    row[P] += Fout
                else:
                    row[other] += Fout
            if gamma is not None:
                g = mesh.weight[f] * gamma[o] + (1.0 - mesh.weight[f]) * gamma[nb]
                a = g * mesh.mag_sf[f] * mesh.delta[f]
                row[P] += a
                row[other] -= a
        for b in np.nonzero(mesh.b_cell == P)[0]:
            if phi_b is not None:
                if phi_b[b] >= 0.0:
                    row[P] += phi_b[b]
                else:
                    s -= phi_b[b] * Y_b[b]
            if gamma is not None and mesh.b_type[b] == 1:
                a = gamma_b[b] * mesh.b_mag_sf[b] * mesh.b_delta[b]
                row[P] += a
                s += a * Y_b[b]
        if S is not None:
            s += V[P] * (1.0 if kappa is None else kappa[P]) * S[P]
        out[P] = (row, s)
    return out


def ldu(mesh, A):
    """(lower, upper, diag) of a dense matrix on the mesh's addressing."""
    o, nb = mesh.owner.astype(np.int64), mesh.neighbour.astype(np.int64)
    return A[nb, o].copy(), A[o, nb].copy(), np.diag(A).copy()


def pasr_kappa(tau_c, rho, mu, strain, delta, c_s, c_mix):
    tau_c = np.asarray(tau_c, np.float64)
    nu_sgs = (c_s * np.asarray(delta)) ** 2 * np.asarray(strain)
    mu_eff = np.asarray(mu) + np.asarray(rho) * nu_sgs
    eps = nu_sgs * np.asarray(strain) ** 2
    kappa = np.empty_like(tau_c)
    for i in range(tau_c.size):
        if eps[i] > 0.0:
            tmix = c_mix * np.sqrt(mu_eff[i] / (rho[i] * eps[i]))
            kappa[i] = tau_c[i] / (tau_c[i] + tmix)
        else:
            kappa[i] = 1.0            # no sub-grid turbulence: the cell is a perfectly stirred reactor
    return kappa
