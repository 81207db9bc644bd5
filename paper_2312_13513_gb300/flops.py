"""Algorithmic FP64 operation counts of one integrator sub-step (roofline numerator).

The counts follow the formulation the kernels evaluate (sparse production lists, the sparse
Jacobian-assembly program, dense LU with partial pivoting), one cell at a time, counting each
useful arithmetic operation once (add/sub/mul/div/sqrt = 1 flop, fused multiply-add = 2 flops),
not the lanes or the redundant per-thread copies the GPU executes.  Transcendentals (exp, log,
log10, pow) are counted separately and folded in at TRANSCENDENTAL_FLOPS each.

Per cell:  flops = n_accepted * (rhs + jac) + n_attempts * attempt, where jac is the extra work of
the analytic Jacobian at a state whose right-hand side is also evaluated, and attempt is one
Rodas4 attempt (iteration matrix, LU, six stages with five right-hand sides, error norm).
"""
from __future__ import annotations

import numpy as np

TRANSCENDENTAL_FLOPS = 20


def _rxn_sides(mech):
    nre = (np.asarray(mech.reac) >= 0).sum(axis=1)
    npr = (np.asarray(mech.prod) >= 0).sum(axis=1)
    return nre, npr


def lu_flops(N):
    """Dense LU with partial pivoting of an N x N matrix: per column k, N-k-1 multipliers and a
    rank-one update of (N-k-1)^2 multiply-adds, plus the N pivot reciprocals."""
    return sum((N - k - 1) + 2 * (N - k - 1) ** 2 for k in range(N)) + N


def solve_flops(N):
    """Forward (unit lower) and backward substitution with the factors: 2 N^2 - N."""
    return 2 * N * N - N


def counts(mech):
    """dict of per-event (flops, transcendentals) for one cell of this mechanism."""
    ns, nr = mech.ns, mech.nr
    N = ns + 1
    rtype = np.asarray(mech.rtype)
    nre, npr = _rxn_sides(mech)
    eff = np.asarray(mech.eff)
    neff = int(sum(np.count_nonzero(eff[j] != 1.0) for j in range(nr) if rtype[j] != 0))
    nprod = 0
    for j in range(nr):
        nu = {}
        for k in mech.reac[j]:
            if k >= 0:
                nu[k] = nu.get(k, 0) - 1
        for k in mech.prod[j]:
            if k >= 0:
                nu[k] = nu.get(k, 0) + 1
        nprod += sum(1 for v in nu.values() if v != 0)
    ntb = int(np.count_nonzero(rtype != 0))
    ntroe = int(np.count_nonzero(rtype == 2))
    nt2 = int(np.count_nonzero((rtype == 2) & (np.asarray(mech.has_t2) != 0)))

    # ---- right-hand side ---------------------------------------------------------------
    rhs = 1                                   # 1/T
    rhs += ns * (10 + 11 + 8 + 1 + 1 + 3)     # h/RT, s/R, cp/R Horner; g; Y/W; two partial sums
    rhs += 3 + 1 + 2 * ns                     # rho, 1/rho, concentrations
    per_rxn = 4 + (nre - 1) + (npr - 1) + nre + npr + 2 + 1 + 2 + 1   # kf arg, products, dG, lnKc, kr, fwd/rev, q
    rhs += int(per_rxn.sum()) + ntb * 2 + 2 * neff + int(np.count_nonzero(rtype == 1))
    rhs += ntroe * 30 + nt2 * 3               # fall-off blending
    rhs += 2 * nprod + ns * (1 + 2 + 2) + 3   # production, h_k, Q, f
    rhs_tr = 1 + nr * 2 + ntroe * 6 + nt2     # lnT; exp(kf), exp(1/Kc); Troe exps/logs

    # ---- analytic Jacobian (extra over the right-hand side at the same state) ------------
    jac = ns * (6 + 2)                        # d(cp/R)/dT and its sum
    jac += int((4 + (nre + npr) + 2 + 5 + 2 * (nre + npr) + 2).sum())
    jac += ntroe * 45                         # fall-off derivatives
    jac += 2 * nprod + 4 * ns                 # d(wdot)/dT, partial sums
    nterm = 0
    for j in range(nr):
        nu_nz = 0
        nu = {}
        for k in mech.reac[j]:
            if k >= 0:
                nu[k] = nu.get(k, 0) - 1
        for k in mech.prod[j]:
            if k >= 0:
                nu[k] = nu.get(k, 0) + 1
        nu_nz = sum(1 for v in nu.values() if v != 0)
        nterm += nu_nz * (nre[j] + npr[j])
        if rtype[j] != 0:
            nterm += nu_nz * int(np.count_nonzero(eff[j] != 0.0))
    jac += 2 * nterm                          # assembly program
    jac += 2 * ns * ns + (2 * ns * ns + ns)   # r_k and H_m
    jac += 3 * ns + 2                         # R_h
    jac += 6 * ns * ns + 6 * ns + 10 * ns + 20
    jac_tr = ntroe * 2

    # ---- one Rodas4 attempt ----------------------------------------------------------------
    lu = lu_flops(N)
    solve = solve_flops(N)
    att = 3 + N * N + lu + 6 * solve
    att += sum(N * 2 * s for s in range(1, 6))            # stage arguments
    att += sum(N * 2 * s + s for s in range(1, 6))        # stage right-hand sides
    att += 12 * N + 5 * N + 3                             # y_new, error norm
    att += 5 * rhs
    att_tr = 5 * rhs_tr + 1                               # five RHS, pow in the step control
    return {"rhs": (rhs, rhs_tr), "jac": (jac, jac_tr), "attempt": (att, att_tr),
            "nterm": nterm, "nprod": nprod, "neff": neff}


def launch_flops(mech, n_accepted_total, n_attempts_total):
    """(flops, transcendentals, folded flops) of a launch with the given sub-step totals."""
    c = counts(mech)
    fl = n_accepted_total * (c["rhs"][0] + c["jac"][0]) + n_attempts_total * c["attempt"][0]
    tr = n_accepted_total * (c["rhs"][1] + c["jac"][1]) + n_attempts_total * c["attempt"][1]
    return float(fl), float(tr), float(fl + TRANSCENDENTAL_FLOPS * tr)


def transport_counts(ns):
    """(flops, transcendentals) of one cell's mixture-averaged properties (chem_transport_eval),
    counting the diffusion fits once per unordered species pair, as the definition needs."""
    per_species = 2 * 6 + 2 + 6 + 4          # two cubic fits, X_k, Mathur sums, D_km division
    pairs = ns * (ns - 1) // 2
    fl = ns * per_species + pairs * (6 + 2 * 2) + ns * ns * 6 + 8
    tr = 4 * ns + pairs + 1                   # sqrt(mu), 1/sqrt(mu), lambda, 1/lambda; D fits; ln T
    return fl, tr
