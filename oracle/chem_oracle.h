/*
 * Oracle: a plain, slow, FP64 CPU implementation of the per-cell chemistry advance.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library.  It shares no code with the CUDA path.
 *
 * The paper (§2) delegates kinetics to Cantera and integrates it with CVODE on the CPU; it
 * prints none of the formulas.  This file restates the standard definitions that such a
 * library computes (NASA-7 thermo, Arrhenius / third-body / Troe rates, reverse rates from
 * equilibrium constants, the constant-pressure adiabatic reactor ODE) and integrates them with
 * the L-stable Rosenbrock method Rodas4 (Hairer & Wanner, Solving ODEs II, §IV.7).
 *
 * Units are CHEMKIN cgs: concentrations mol/cm^3, pressure dyn/cm^2, Ea in cal/mol.
 * State vector y = (T, Y_1 .. Y_ns), N = ns + 1.  Matrices are row-major, J[i*N + j] = df_i/dy_j.
 */
#ifndef CHEM_ORACLE_H
#define CHEM_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_mech or_mech;

enum { OR_OK = 0, OR_MAX_STEPS = 1, OR_H_UNDERFLOW = 2, OR_NONFINITE = 3, OR_SINGULAR_LU = 4 };

or_mech* or_mech_new(int ns, int ne, int nr, const double* elem_mass, const int* comp,
                     const double* nasa_lo, const double* nasa_hi, const int* rtype,
                     const int* reac, const int* prod, const double* A, const double* b,
                     const double* Ea, const double* troe, const int* has_t2, const double* eff);
void or_mech_free(or_mech* m);

/* per-species cp/R, h/RT, s/R and d(cp/R)/dT at temperature T (any pointer may be NULL) */
void or_species_thermo(const or_mech* m, double T, double* cp_R, double* h_RT, double* s_R,
                       double* dcpR_dT);
/* molar production rates wdot[ns] (mol/cm^3/s); q, kf, kr per reaction (may be NULL) */
void or_rates(const or_mech* m, double T, double p, const double* Y, double* wdot, double* q,
              double* kf, double* kr);
void or_rhs(const or_mech* m, double p, const double* y, double* f);
void or_rhs_complex(const or_mech* m, double p, const double* y_re, const double* y_im,
                    double* f_re, double* f_im);
void or_jacobian(const or_mech* m, double p, const double* y, double* J);
void or_jacobian_complex_step(const or_mech* m, double p, const double* y, double* J);

/* One CFD step of length dt for one cell, in place.  Returns an OR_* status. */
int or_rodas4(const or_mech* m, double p, double* y, double dt, double rtol, double atol,
              int max_steps, int* nsub, int* nrej);
/* Batch over cells with OpenMP.  Y is species-major: Y[k*ld + i].  status/nsub may be NULL. */
void or_advance(const or_mech* m, int64_t n, double* T, const double* p, double* Y, int64_t ld,
                double dt, double rtol, double atol, int8_t* status, int32_t* nsub, int nthreads);
/* Same with a per-cell step length dt[n] (status may be NULL). */
void or_advance_dt(const or_mech* m, int64_t n, double* T, const double* p, double* Y, int64_t ld,
                   const double* dt, double rtol, double atol, int8_t* status, int nthreads);
/* Classical RK4 with nsteps equal steps over dt (brute-force reference). */
void or_rk4(const or_mech* m, double p, double* y, double dt, int64_t nsteps);

/* Rodas4 coefficients in the transformed form: gamma, A[6*6], C[6*6], M[6], E[6] */
void or_rodas4_tableau(double* gamma, double* A, double* C, double* M, double* E);
/* Rodas4 on the linear system y' = L y (N x N), nsteps fixed steps of size h (order tests) */
void or_rodas4_linear(int N, const double* L, double* y, double h, int nsteps, double* err_last);

/* Operation counts of one cell advance (counted scalar type).  counts[] =
 * {add, mul, div, exp, log, pow, sqrt, cmp}; returns status, nsub/nrej filled. */
int or_count_ops(const or_mech* m, double p, const double* y, double dt, double rtol, double atol,
                 double* counts, int* nsub, int* nrej);

#ifdef __cplusplus
}
#endif
#endif
