// Oracle: plain FP64 CPU kinetics, Jacobian and Rosenbrock integrator.
//
// TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the benchmark).
// Shares no code with the CUDA path.  Every routine favours a direct transcription of the
// definition over speed: dense loops over all reactions and species, no sparsity, no fusion.
//
// Sources of the definitions (the paper, §2, names Cantera and CVODE but prints no formula):
//   * NASA-7 polynomials: cp/R, h/RT, s/R with two temperature ranges split at 1000 K.
//   * Mass-action kinetics: kf = A T^b exp(-Ea/(Rc T)); third-body [M] = sum eff_k C_k;
//     Troe fall-off (Gilbert, Luther & Troe 1983); Kc from the standard Gibbs energy change;
//     kr = kf / Kc.
//   * Constant-pressure adiabatic reactor: dY_k/dt = W_k wdot_k / rho,
//     dT/dt = -sum_k h_k wdot_k / (rho cp).
//   * Rodas4 (Hairer & Wanner, Solving ODEs II, §IV.7), transformed stage form.
#include "chem_oracle.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

const double RU = 8.314462618e7;       // erg / (mol K)
const double RC = RU / 4.184e7;        // cal / (mol K)
const double PATM = 1.01325e6;         // dyn / cm^2
const double TMID = 1000.0;

// ---------------------------------------------------------------------------------------
// scalar helpers: plain double, complex (complex-step derivative) and an op-counting double
// ---------------------------------------------------------------------------------------
inline double re(double x) { return x; }
inline double re(const std::complex<double>& x) { return x.real(); }

struct OpCounts { double add, mul, div, exp, log, pow, sqrt, cmp; };
thread_local OpCounts g_ops;

struct CD {   // counted double
  double v;
  CD() : v(0) {}
  CD(double x) : v(x) {}
};
inline double re(const CD& x) { return x.v; }
inline CD operator+(CD a, CD b) { g_ops.add++; return CD(a.v + b.v); }
inline CD operator-(CD a, CD b) { g_ops.add++; return CD(a.v - b.v); }
inline CD operator-(CD a) { return CD(-a.v); }
inline CD operator*(CD a, CD b) { g_ops.mul++; return CD(a.v * b.v); }
inline CD operator/(CD a, CD b) { g_ops.div++; return CD(a.v / b.v); }
inline CD& operator+=(CD& a, CD b) { a = a + b; return a; }
inline CD& operator-=(CD& a, CD b) { a = a - b; return a; }
inline CD& operator*=(CD& a, CD b) { a = a * b; return a; }
inline CD& operator/=(CD& a, CD b) { a = a / b; return a; }
inline bool operator<(CD a, CD b) { g_ops.cmp++; return a.v < b.v; }
inline bool operator>(CD a, CD b) { g_ops.cmp++; return a.v > b.v; }
inline bool operator<=(CD a, CD b) { g_ops.cmp++; return a.v <= b.v; }
inline bool operator>=(CD a, CD b) { g_ops.cmp++; return a.v >= b.v; }
inline CD exp(CD a) { g_ops.exp++; return CD(std::exp(a.v)); }
inline CD log(CD a) { g_ops.log++; return CD(std::log(a.v)); }
inline CD log10(CD a) { g_ops.log++; return CD(std::log10(a.v)); }
inline CD pow(CD a, CD b) { g_ops.pow++; return CD(std::pow(a.v, b.v)); }
inline CD sqrt(CD a) { g_ops.sqrt++; return CD(std::sqrt(a.v)); }
inline CD fabs(CD a) { return CD(std::fabs(a.v)); }

using std::exp;
using std::log;
using std::log10;
using std::pow;
using std::sqrt;
using std::fabs;

template <class S> S sq(const S& x) { return x * x; }

}  // namespace

struct or_mech {
  int ns, ne, nr;
  std::vector<double> elem_mass, W, lo, hi, A, b, Ea, troe, eff;
  std::vector<int> comp, rtype, reac, prod, has_t2;
};

namespace {

// ---------------------------------------------------------------------------------------
// NASA-7 thermo (per species, dimensionless)
// ---------------------------------------------------------------------------------------
template <class S>
void thermo(const or_mech& m, const S& T, S* cp_R, S* h_RT, S* s_R, S* dcp) {
  for (int k = 0; k < m.ns; ++k) {
    const double* a = (re(T) < TMID) ? &m.lo[7 * k] : &m.hi[7 * k];
    S T2 = T * T, T3 = T2 * T, T4 = T3 * T;
    if (cp_R) cp_R[k] = S(a[0]) + S(a[1]) * T + S(a[2]) * T2 + S(a[3]) * T3 + S(a[4]) * T4;
    if (h_RT)
      h_RT[k] = S(a[0]) + S(a[1]) * T / S(2.0) + S(a[2]) * T2 / S(3.0) + S(a[3]) * T3 / S(4.0) +
                S(a[4]) * T4 / S(5.0) + S(a[5]) / T;
    if (s_R)
      s_R[k] = S(a[0]) * log(T) + S(a[1]) * T + S(a[2]) * T2 / S(2.0) + S(a[3]) * T3 / S(3.0) +
               S(a[4]) * T4 / S(4.0) + S(a[6]);
    if (dcp) dcp[k] = S(a[1]) + S(2.0) * S(a[2]) * T + S(3.0) * S(a[3]) * T2 + S(4.0) * S(a[4]) * T3;
  }
}

// ---------------------------------------------------------------------------------------
// Rates of progress and molar production rates
// ---------------------------------------------------------------------------------------
template <class S>
struct RxnEval {   // per-reaction quantities needed by the analytic Jacobian
  S kf, kr, Kc, fwd, rev, M, q;
};

template <class S>
void rates(const or_mech& m, const S& T, const S& p, const S* Y, S* wdot, RxnEval<S>* ev) {
  const int ns = m.ns;
  std::vector<S> h_RT(ns), s_R(ns), C(ns);
  thermo<S>(m, T, nullptr, h_RT.data(), s_R.data(), nullptr);
  S sumYW(0.0);
  for (int k = 0; k < ns; ++k) sumYW += Y[k] / S(m.W[k]);
  S rho = p / (S(RU) * T * sumYW);
  for (int k = 0; k < ns; ++k) C[k] = rho * Y[k] / S(m.W[k]);
  for (int k = 0; k < ns; ++k) wdot[k] = S(0.0);
  for (int j = 0; j < m.nr; ++j) {
    S kf = S(m.A[j]) * pow(T, S(m.b[j])) * exp(-S(m.Ea[j]) / (S(RC) * T));
    S M(0.0);
    if (m.rtype[j] != 0)
      for (int k = 0; k < ns; ++k) M += S(m.eff[(size_t)j * ns + k]) * C[k];
    if (m.rtype[j] == 2) {
      // Troe fall-off; k = kinf Pr/(1+Pr) F vanishes when kinf or k0 [M] does (Pr = 0)
      const double* tr = &m.troe[7 * j];
      S k0 = S(tr[0]) * pow(T, S(tr[1])) * exp(-S(tr[2]) / (S(RC) * T));
      if (re(kf) == 0.0 || re(k0 * M) == 0.0) {
        kf = S(0.0);
      } else {
        S Pr = k0 * M / kf;
        S Fcent = (S(1.0) - S(tr[3])) * exp(-T / S(tr[4])) + S(tr[3]) * exp(-T / S(tr[5]));
        if (m.has_t2[j]) Fcent += exp(-S(tr[6]) / T);
        S L = log10(Fcent);
        S c = S(-0.4) - S(0.67) * L;
        S n = S(0.75) - S(1.27) * L;
        S u = log10(Pr) + c;
        S f1 = u / (n - S(0.14) * u);
        S logF = L / (S(1.0) + f1 * f1);
        kf = kf * (Pr / (S(1.0) + Pr)) * pow(S(10.0), logF);
      }
    }
    // standard-state Gibbs change and net mole change of the reaction
    S dG(0.0);
    int dnu = 0;
    for (int i = 0; i < 3; ++i) {
      int kp = m.prod[3 * j + i], kr_ = m.reac[3 * j + i];
      if (kp >= 0) { dG += h_RT[kp] - s_R[kp]; dnu += 1; }
      if (kr_ >= 0) { dG -= h_RT[kr_] - s_R[kr_]; dnu -= 1; }
    }
    S Kc = exp(-dG) * pow(S(PATM) / (S(RU) * T), S((double)dnu));
    S kr = kf / Kc;
    S fwd = kf, rev = kr;
    for (int i = 0; i < 3; ++i) {
      if (m.reac[3 * j + i] >= 0) fwd = fwd * C[m.reac[3 * j + i]];
      if (m.prod[3 * j + i] >= 0) rev = rev * C[m.prod[3 * j + i]];
    }
    S q = fwd - rev;
    if (m.rtype[j] == 1) q = q * M;
    for (int i = 0; i < 3; ++i) {
      if (m.reac[3 * j + i] >= 0) wdot[m.reac[3 * j + i]] -= q;
      if (m.prod[3 * j + i] >= 0) wdot[m.prod[3 * j + i]] += q;
    }
    if (ev) {
      ev[j].kf = kf; ev[j].kr = kr; ev[j].Kc = Kc; ev[j].fwd = fwd; ev[j].rev = rev;
      ev[j].M = M; ev[j].q = q;
    }
  }
}

// Right-hand side of the constant-pressure adiabatic reactor, y = (T, Y)
template <class S>
void rhs(const or_mech& m, const S& p, const S* y, S* f) {
  const int ns = m.ns;
  const S T = y[0];
  const S* Y = y + 1;
  std::vector<S> wdot(ns), cp_R(ns), h_RT(ns);
  rates<S>(m, T, p, Y, wdot.data(), nullptr);
  thermo<S>(m, T, cp_R.data(), h_RT.data(), nullptr, nullptr);
  S sumYW(0.0);
  for (int k = 0; k < ns; ++k) sumYW += Y[k] / S(m.W[k]);
  S rho = p / (S(RU) * T * sumYW);
  S cp(0.0), Q(0.0);
  for (int k = 0; k < ns; ++k) {
    cp += Y[k] * S(RU) * cp_R[k] / S(m.W[k]);
    Q += S(RU) * T * h_RT[k] * wdot[k];
  }
  f[0] = -Q / (rho * cp);
  for (int k = 0; k < ns; ++k) f[k + 1] = S(m.W[k]) * wdot[k] / rho;
}

// ---------------------------------------------------------------------------------------
// Analytic Jacobian of rhs: dense chain rule through C(T, Y) and rho(T, Y)
// ---------------------------------------------------------------------------------------
template <class S>
void jacobian(const or_mech& m, const S& p, const S* y, S* J) {
  const int ns = m.ns, N = ns + 1, nr = m.nr;
  const S T = y[0];
  const S* Y = y + 1;
  std::vector<S> wdot(ns), cp_R(ns), h_RT(ns), s_R(ns), dcp(ns), C(ns);
  std::vector<RxnEval<S>> ev(nr);
  rates<S>(m, T, p, Y, wdot.data(), ev.data());
  thermo<S>(m, T, cp_R.data(), h_RT.data(), s_R.data(), dcp.data());
  S sumYW(0.0);
  for (int k = 0; k < ns; ++k) sumYW += Y[k] / S(m.W[k]);
  S rho = p / (S(RU) * T * sumYW);
  for (int k = 0; k < ns; ++k) C[k] = rho * Y[k] / S(m.W[k]);

  // dwdot/dC (ns x ns) and dwdot/dT at fixed C
  std::vector<S> dWdC((size_t)ns * ns, S(0.0)), dWdT(ns, S(0.0)), dqdC(ns);
  for (int j = 0; j < nr; ++j) {
    const RxnEval<S>& e = ev[j];
    const int* rs = &m.reac[3 * j];
    const int* ps = &m.prod[3 * j];
    // d(prod_i C_{r_i})/dC_m summed over list positions holding m
    std::vector<S> dPf(ns, S(0.0)), dPr(ns, S(0.0));
    for (int i = 0; i < 3; ++i) {
      if (rs[i] >= 0) {
        S prod(1.0);
        for (int l = 0; l < 3; ++l) if (l != i && rs[l] >= 0) prod = prod * C[rs[l]];
        dPf[rs[i]] += prod;
      }
      if (ps[i] >= 0) {
        S prod(1.0);
        for (int l = 0; l < 3; ++l) if (l != i && ps[l] >= 0) prod = prod * C[ps[l]];
        dPr[ps[i]] += prod;
      }
    }
    // products of concentrations without the rate constants
    S Pf(1.0), Pr_(1.0);
    for (int i = 0; i < 3; ++i) {
      if (rs[i] >= 0) Pf = Pf * C[rs[i]];
      if (ps[i] >= 0) Pr_ = Pr_ * C[ps[i]];
    }
    int dnu = 0;
    S dH_RT(0.0);
    for (int i = 0; i < 3; ++i) {
      if (ps[i] >= 0) { dnu++; dH_RT += h_RT[ps[i]]; }
      if (rs[i] >= 0) { dnu--; dH_RT -= h_RT[rs[i]]; }
    }
    // d ln Kc / dT = (sum nu h/RT - dnu) / T
    S dlnKc = (dH_RT - S((double)dnu)) / T;
    const double Ta = m.Ea[j] / RC;
    S dlnkinf = S(m.b[j]) / T + S(Ta) / (T * T);
    S dlnkf = dlnkinf;     // d ln kf / dT at fixed C
    S dkfdM(0.0);          // d kf / d[M] (Troe only)
    if (m.rtype[j] == 2) {
      const double* tr = &m.troe[7 * j];
      S kinf = S(m.A[j]) * pow(T, S(m.b[j])) * exp(-S(Ta) / T);
      S k0 = S(tr[0]) * pow(T, S(tr[1])) * exp(-S(tr[2] / RC) / T);
      if (re(kinf) == 0.0 || re(k0) == 0.0) {
        dlnkf = S(0.0);     // kf vanishes identically: no T or [M] dependence
        dkfdM = S(0.0);
        goto troe_done;
      }
      if (re(e.M) == 0.0) {
        // [M] -> 0: kf -> 0 and dkf/d[M] -> k0 F(Pr -> 0), F(0) = Fcent^(1/(1 + (1/0.14)^2))
        S e3 = exp(-T / S(tr[4])), e1 = exp(-T / S(tr[5]));
        S Fc = (S(1.0) - S(tr[3])) * e3 + S(tr[3]) * e1;
        if (m.has_t2[j]) Fc += exp(-S(tr[6]) / T);
        dkfdM = k0 * pow(Fc, S(1.0 / (1.0 + 1.0 / (0.14 * 0.14))));
        dlnkf = S(0.0);
        goto troe_done;
      }
    }
    if (m.rtype[j] == 2) {
      const double* tr = &m.troe[7 * j];
      S kinf = S(m.A[j]) * pow(T, S(m.b[j])) * exp(-S(Ta) / T);
      S k0 = S(tr[0]) * pow(T, S(tr[1])) * exp(-S(tr[2] / RC) / T);
      S Pr = k0 * e.M / kinf;
      S e3 = exp(-T / S(tr[4])), e1 = exp(-T / S(tr[5]));
      S Fc = (S(1.0) - S(tr[3])) * e3 + S(tr[3]) * e1;
      S dFc = -(S(1.0) - S(tr[3])) / S(tr[4]) * e3 - S(tr[3]) / S(tr[5]) * e1;
      if (m.has_t2[j]) {
        S e2 = exp(-S(tr[6]) / T);
        Fc += e2;
        dFc += S(tr[6]) / (T * T) * e2;
      }
      S L = log10(Fc);
      S c = S(-0.4) - S(0.67) * L;
      S n = S(0.75) - S(1.27) * L;
      S u = log10(Pr) + c;
      S d = n - S(0.14) * u;
      S f1 = u / d;
      S den = S(1.0) + f1 * f1;
      S logF = L / den;
      S F = pow(S(10.0), logF);
      S dG_dlogPr = -S(2.0) * L * f1 / (den * den) * (n / (d * d));
      S df1_dL = (S(-0.67) * d - u * S(-1.27 + 0.14 * 0.67)) / (d * d);
      S dG_dL = S(1.0) / den - S(2.0) * L * f1 / (den * den) * df1_dL;
      S dL_dT = dFc / (Fc * S(std::log(10.0)));
      S dlnk0 = S(tr[1]) / T + S(tr[2] / RC) / (T * T);
      S dlnPr = dlnk0 - dlnkinf;
      dlnkf = dlnkinf + dlnPr * (S(1.0) / (S(1.0) + Pr) + dG_dlogPr) +
              S(std::log(10.0)) * dG_dL * dL_dT;
      dkfdM = k0 * F / (S(1.0) + Pr) * (S(1.0) / (S(1.0) + Pr) + dG_dlogPr);
    }
  troe_done:
    S dlnkr = dlnkf - dlnKc;
    // dq/dC_m and dq/dT
    for (int k = 0; k < ns; ++k) {
      S v = e.kf * dPf[k] - e.kr * dPr[k];
      if (m.rtype[j] == 1) v = e.M * v + S(m.eff[(size_t)j * ns + k]) * (e.fwd - e.rev);
      if (m.rtype[j] == 2) v = v + dkfdM * S(m.eff[(size_t)j * ns + k]) * (Pf - Pr_ / e.Kc);
      dqdC[k] = v;
    }
    S dqdT = e.fwd * dlnkf - e.rev * dlnkr;
    if (m.rtype[j] == 1) dqdT = e.M * dqdT;
    for (int i = 0; i < 3; ++i) {
      for (int side = 0; side < 2; ++side) {
        int k = side == 0 ? rs[i] : ps[i];
        if (k < 0) continue;
        S sgn = side == 0 ? S(-1.0) : S(1.0);
        dWdT[k] += sgn * dqdT;
        for (int l = 0; l < ns; ++l) dWdC[(size_t)k * ns + l] += sgn * dqdC[l];
      }
    }
  }
  // dC_n/dY_m = rho/W_n delta_nm - C_n/(sumYW W_m);  dC_n/dT = -C_n / T
  std::vector<S> dWdY((size_t)ns * ns), dWdTY(ns);
  for (int k = 0; k < ns; ++k) {
    for (int mm = 0; mm < ns; ++mm) {
      S acc(0.0);
      for (int n = 0; n < ns; ++n) {
        S dCn = -C[n] / (sumYW * S(m.W[mm]));
        if (n == mm) dCn = dCn + rho / S(m.W[n]);
        acc += dWdC[(size_t)k * ns + n] * dCn;
      }
      dWdY[(size_t)k * ns + mm] = acc;
    }
    S acc = dWdT[k];
    for (int n = 0; n < ns; ++n) acc += dWdC[(size_t)k * ns + n] * (-C[n] / T);
    dWdTY[k] = acc;
  }
  S cp(0.0), Q(0.0), dcpdT(0.0);
  std::vector<S> h(ns);
  for (int k = 0; k < ns; ++k) {
    h[k] = S(RU) * T * h_RT[k];
    cp += Y[k] * S(RU) * cp_R[k] / S(m.W[k]);
    dcpdT += Y[k] * S(RU) * dcp[k] / S(m.W[k]);
    Q += h[k] * wdot[k];
  }
  S rcp = rho * cp;
  // species rows
  for (int k = 0; k < ns; ++k) {
    S fk = S(m.W[k]) * wdot[k] / rho;
    // d rho/dT = -rho/T ; d rho/dY_m = -rho/(sumYW W_m)
    J[(size_t)(k + 1) * N + 0] = S(m.W[k]) / rho * dWdTY[k] + fk / T;
    for (int mm = 0; mm < ns; ++mm)
      J[(size_t)(k + 1) * N + mm + 1] =
          S(m.W[k]) / rho * dWdY[(size_t)k * ns + mm] + fk / (sumYW * S(m.W[mm]));
  }
  // temperature row
  {
    S num(0.0);
    for (int k = 0; k < ns; ++k) num += S(RU) * cp_R[k] * wdot[k] + h[k] * dWdTY[k];
    S drcp_dT = -rho / T * cp + rho * dcpdT;
    J[0] = -num / rcp + Q / (rcp * rcp) * drcp_dT;
    for (int mm = 0; mm < ns; ++mm) {
      S s(0.0);
      for (int k = 0; k < ns; ++k) s += h[k] * dWdY[(size_t)k * ns + mm];
      S drcp = -rho / (sumYW * S(m.W[mm])) * cp + rho * S(RU) * cp_R[mm] / S(m.W[mm]);
      J[mm + 1] = -s / rcp + Q / (rcp * rcp) * drcp;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Dense LU with partial pivoting (Doolittle; ties resolved to the lowest row index)
// ---------------------------------------------------------------------------------------
template <class S>
bool lu_factor(int N, S* a, int* piv) {
  for (int k = 0; k < N; ++k) {
    int pr = k;
    double best = std::fabs(re(a[(size_t)k * N + k]));
    for (int i = k + 1; i < N; ++i) {
      double v = std::fabs(re(a[(size_t)i * N + k]));
      if (v > best) { best = v; pr = i; }
    }
    piv[k] = pr;
    if (best == 0.0) return false;
    if (pr != k)
      for (int j = 0; j < N; ++j) std::swap(a[(size_t)k * N + j], a[(size_t)pr * N + j]);
    for (int i = k + 1; i < N; ++i) {
      S l = a[(size_t)i * N + k] / a[(size_t)k * N + k];
      a[(size_t)i * N + k] = l;
      for (int j = k + 1; j < N; ++j) a[(size_t)i * N + j] -= l * a[(size_t)k * N + j];
    }
  }
  return true;
}

template <class S>
void lu_solve(int N, const S* a, const int* piv, S* x) {
  for (int k = 0; k < N; ++k)
    if (piv[k] != k) std::swap(x[k], x[piv[k]]);
  for (int i = 1; i < N; ++i)
    for (int j = 0; j < i; ++j) x[i] -= a[(size_t)i * N + j] * x[j];
  for (int i = N - 1; i >= 0; --i) {
    for (int j = i + 1; j < N; ++j) x[i] -= a[(size_t)i * N + j] * x[j];
    x[i] = x[i] / a[(size_t)i * N + i];
  }
}

// ---------------------------------------------------------------------------------------
// Rodas4 coefficients, transformed form (u-variables): stage i solves
//   (I/(gamma h) - J) u_i = f(y + sum_j A_ij u_j) + sum_j (C_ij / h) u_j,
//   y1 = y + sum_i M_i u_i,  error estimate = sum_i E_i u_i.
// ---------------------------------------------------------------------------------------
const double RD_GAMMA = 0.25;
const double RD_A[6][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.544, 0, 0, 0, 0, 0},
    {0.9466785280815826, 0.2557011698983284, 0, 0, 0, 0},
    {3.314825187068521, 2.896124015972201, 0.9986419139977817, 0, 0, 0},
    {1.221224509226641, 6.019134481288629, 12.53708332932087, -0.6878860361058950, 0, 0},
    {1.221224509226641, 6.019134481288629, 12.53708332932087, -0.6878860361058950, 1.0, 0}};
const double RD_C[6][6] = {
    {0, 0, 0, 0, 0, 0},
    {-5.6688, 0, 0, 0, 0, 0},
    {-2.430093356833875, -0.2063599157091915, 0, 0, 0, 0},
    {-0.1073529058151375, -9.594562251023355, -20.47028614809616, 0, 0, 0},
    {7.496443313967647, -10.24680431464352, -33.99990352819905, 11.70890893206160, 0, 0},
    {8.083246795921522, -7.981132988064893, -31.52159432874371, 16.31930543123136,
     -6.058818238834054, 0}};
const double RD_M[6] = {1.221224509226641, 6.019134481288629, 12.53708332932087,
                        -0.6878860361058950, 1.0, 1.0};
const double RD_E[6] = {0, 0, 0, 0, 0, 1.0};

// One Rodas4 attempt from y with step h given f0 = f(y) and J = df/dy.
// Returns false if the iteration matrix is singular.  ynew and the error vector are filled.
template <class S, class RHS>
bool rodas4_attempt(int N, RHS&& fun, const S* y, const S* f0, const S* J, S h, S* ynew, S* err) {
  std::vector<S> Mx((size_t)N * N), u((size_t)6 * N), ys(N), fs(N);
  std::vector<int> piv(N);
  S ig = S(1.0) / (S(RD_GAMMA) * h);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) Mx[(size_t)i * N + j] = (i == j ? ig : S(0.0)) - J[(size_t)i * N + j];
  if (!lu_factor<S>(N, Mx.data(), piv.data())) return false;
  for (int s = 0; s < 6; ++s) {
    if (s == 0) {
      for (int i = 0; i < N; ++i) fs[i] = f0[i];
    } else {
      for (int i = 0; i < N; ++i) {
        S v = y[i];
        for (int j = 0; j < s; ++j) v += S(RD_A[s][j]) * u[(size_t)j * N + i];
        ys[i] = v;
      }
      fun(ys.data(), fs.data());
    }
    S* us = &u[(size_t)s * N];
    for (int i = 0; i < N; ++i) {
      S v = fs[i];
      for (int j = 0; j < s; ++j) v += S(RD_C[s][j]) / h * u[(size_t)j * N + i];
      us[i] = v;
    }
    lu_solve<S>(N, Mx.data(), piv.data(), us);
  }
  for (int i = 0; i < N; ++i) {
    S v = y[i], e(0.0);
    for (int s = 0; s < 6; ++s) {
      v += S(RD_M[s]) * u[(size_t)s * N + i];
      e += S(RD_E[s]) * u[(size_t)s * N + i];
    }
    ynew[i] = v;
    err[i] = e;
  }
  return true;
}

inline bool finite_state(int N, const double* y, double p) {
  if (!std::isfinite(p) || !(p > 0.0)) return false;
  if (!std::isfinite(y[0]) || !(y[0] > 0.0)) return false;
  for (int i = 1; i < N; ++i)
    if (!std::isfinite(y[i])) return false;
  return true;
}

// Adaptive Rodas4 over [0, dt]; y is updated in place with the last accepted state.
template <class S>
int rodas4_integrate(const or_mech& m, const S& p, S* y, double dt, double rtol, double atol,
                     int max_steps, int* nsub_out, int* nrej_out) {
  const int N = m.ns + 1;
  std::vector<S> f0(N), J((size_t)N * N), ynew(N), err(N);
  auto fun = [&](const S* yy, S* ff) { rhs<S>(m, p, yy, ff); };
  S t(0.0);
  S h(dt);
  S facmax(6.0);
  int nsub = 0, nrej = 0, attempts = 0, status = OR_OK;
  bool have_fj = false;
  for (;;) {
    if (attempts >= max_steps) { status = OR_MAX_STEPS; break; }
    bool last = false;
    if (re(h) >= dt - re(t)) { h = S(dt) - t; last = true; }
    if (re(h) < 1e-12 * dt) { status = OR_H_UNDERFLOW; break; }
    if (!have_fj) {
      fun(y, f0.data());
      jacobian<S>(m, p, y, J.data());
      have_fj = true;
    }
    ++attempts;
    if (!rodas4_attempt<S>(N, fun, y, f0.data(), J.data(), h, ynew.data(), err.data())) {
      status = OR_SINGULAR_LU;
      break;
    }
    S acc(0.0);
    for (int i = 0; i < N; ++i) {
      double ay = std::fabs(re(y[i])), an = std::fabs(re(ynew[i]));
      S sc = S(atol) + S(rtol) * S(ay > an ? ay : an);
      acc += sq(err[i] / sc);
    }
    S en = sqrt(acc / S((double)N));
    double env = re(en);
    if (env <= 1.0) {
      for (int i = 0; i < N; ++i) y[i] = ynew[i];
      have_fj = false;
      ++nsub;
      if (last) break;
      t += h;
      S fac = S(0.9) * pow(en, S(-0.25));
      if (re(fac) < 0.2) fac = S(0.2);
      if (re(fac) > re(facmax)) fac = facmax;
      h = h * fac;
      facmax = S(6.0);
    } else {
      ++nrej;
      S fac(0.2);
      if (std::isfinite(env)) {
        fac = S(0.9) * pow(en, S(-0.25));
        if (re(fac) < 0.2) fac = S(0.2);
      }
      h = h * fac;
      facmax = S(1.0);
    }
  }
  if (nsub_out) *nsub_out = nsub;
  if (nrej_out) *nrej_out = nrej;
  return status;
}

}  // namespace

// =========================================================================================
// extern "C" API
// =========================================================================================
extern "C" {

or_mech* or_mech_new(int ns, int ne, int nr, const double* elem_mass, const int* comp,
                     const double* nasa_lo, const double* nasa_hi, const int* rtype,
                     const int* reac, const int* prod, const double* A, const double* b,
                     const double* Ea, const double* troe, const int* has_t2, const double* eff) {
  or_mech* m = new or_mech();
  m->ns = ns; m->ne = ne; m->nr = nr;
  m->elem_mass.assign(elem_mass, elem_mass + ne);
  m->comp.assign(comp, comp + (size_t)ns * ne);
  m->W.assign(ns, 0.0);
  for (int k = 0; k < ns; ++k)
    for (int e = 0; e < ne; ++e) m->W[k] += comp[(size_t)k * ne + e] * elem_mass[e];
  m->lo.assign(nasa_lo, nasa_lo + 7 * ns);
  m->hi.assign(nasa_hi, nasa_hi + 7 * ns);
  m->rtype.assign(rtype, rtype + nr);
  m->reac.assign(reac, reac + 3 * nr);
  m->prod.assign(prod, prod + 3 * nr);
  m->A.assign(A, A + nr);
  m->b.assign(b, b + nr);
  m->Ea.assign(Ea, Ea + nr);
  m->troe.assign(troe, troe + 7 * nr);
  m->has_t2.assign(has_t2, has_t2 + nr);
  m->eff.assign(eff, eff + (size_t)nr * ns);
  return m;
}

void or_mech_free(or_mech* m) { delete m; }

void or_species_thermo(const or_mech* m, double T, double* cp_R, double* h_RT, double* s_R,
                       double* dcpR_dT) {
  thermo<double>(*m, T, cp_R, h_RT, s_R, dcpR_dT);
}

void or_rates(const or_mech* m, double T, double p, const double* Y, double* wdot, double* q,
              double* kf, double* kr) {
  std::vector<RxnEval<double>> ev(m->nr);
  std::vector<double> w(m->ns);
  rates<double>(*m, T, p, Y, w.data(), ev.data());
  for (int k = 0; k < m->ns; ++k) if (wdot) wdot[k] = w[k];
  for (int j = 0; j < m->nr; ++j) {
    if (q) q[j] = ev[j].q;
    if (kf) kf[j] = ev[j].kf;
    if (kr) kr[j] = ev[j].kr;
  }
}

void or_rhs(const or_mech* m, double p, const double* y, double* f) { rhs<double>(*m, p, y, f); }

void or_rhs_complex(const or_mech* m, double p, const double* y_re, const double* y_im,
                    double* f_re, double* f_im) {
  const int N = m->ns + 1;
  std::vector<std::complex<double>> y(N), f(N);
  for (int i = 0; i < N; ++i) y[i] = std::complex<double>(y_re[i], y_im[i]);
  rhs<std::complex<double>>(*m, std::complex<double>(p, 0.0), y.data(), f.data());
  for (int i = 0; i < N; ++i) { f_re[i] = f[i].real(); f_im[i] = f[i].imag(); }
}

void or_jacobian(const or_mech* m, double p, const double* y, double* J) {
  jacobian<double>(*m, p, y, J);
}

// Complex-step derivative: df/dy_j = Im f(y + i h e_j) / h, exact to rounding for analytic f.
void or_jacobian_complex_step(const or_mech* m, double p, const double* y, double* J) {
  const int N = m->ns + 1;
  std::vector<std::complex<double>> yc(N), fc(N);
  for (int j = 0; j < N; ++j) {
    double h = 1e-30 * std::max(1.0, std::fabs(y[j]));
    for (int i = 0; i < N; ++i) yc[i] = std::complex<double>(y[i], i == j ? h : 0.0);
    rhs<std::complex<double>>(*m, std::complex<double>(p, 0.0), yc.data(), fc.data());
    for (int i = 0; i < N; ++i) J[(size_t)i * N + j] = fc[i].imag() / h;
  }
}

int or_rodas4(const or_mech* m, double p, double* y, double dt, double rtol, double atol,
              int max_steps, int* nsub, int* nrej) {
  const int N = m->ns + 1;
  if (!finite_state(N, y, p)) {
    if (nsub) *nsub = 0;
    if (nrej) *nrej = 0;
    return OR_NONFINITE;
  }
  return rodas4_integrate<double>(*m, p, y, dt, rtol, atol, max_steps, nsub, nrej);
}

void or_advance(const or_mech* m, int64_t n, double* T, const double* p, double* Y, int64_t ld,
                double dt, double rtol, double atol, int8_t* status, int32_t* nsub, int nthreads) {
  const int ns = m->ns, N = ns + 1;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
  for (int64_t i = 0; i < n; ++i) {
    std::vector<double> y(N);
    y[0] = T[i];
    for (int k = 0; k < ns; ++k) y[k + 1] = Y[(size_t)k * ld + i];
    int ns_ = 0, nr_ = 0;
    int st = or_rodas4(m, p[i], y.data(), dt, rtol, atol, 100000, &ns_, &nr_);
    if (st != OR_NONFINITE) {
      T[i] = y[0];
      for (int k = 0; k < ns; ++k) Y[(size_t)k * ld + i] = y[k + 1];
    }
    if (status) status[i] = (int8_t)st;
    if (nsub) nsub[i] = ns_;
  }
}

void or_advance_dt(const or_mech* m, int64_t n, double* T, const double* p, double* Y, int64_t ld,
                   const double* dt, double rtol, double atol, int8_t* status, int nthreads) {
  const int ns = m->ns, N = ns + 1;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
  for (int64_t i = 0; i < n; ++i) {
    std::vector<double> y(N);
    y[0] = T[i];
    for (int k = 0; k < ns; ++k) y[k + 1] = Y[(size_t)k * ld + i];
    int st = or_rodas4(m, p[i], y.data(), dt[i], rtol, atol, 100000, nullptr, nullptr);
    if (st != OR_NONFINITE) {
      T[i] = y[0];
      for (int k = 0; k < ns; ++k) Y[(size_t)k * ld + i] = y[k + 1];
    }
    if (status) status[i] = (int8_t)st;
  }
}

void or_rk4(const or_mech* m, double p, double* y, double dt, int64_t nsteps) {
  const int N = m->ns + 1;
  std::vector<double> k1(N), k2(N), k3(N), k4(N), yt(N);
  double h = dt / (double)nsteps;
  for (int64_t s = 0; s < nsteps; ++s) {
    rhs<double>(*m, p, y, k1.data());
    for (int i = 0; i < N; ++i) yt[i] = y[i] + 0.5 * h * k1[i];
    rhs<double>(*m, p, yt.data(), k2.data());
    for (int i = 0; i < N; ++i) yt[i] = y[i] + 0.5 * h * k2[i];
    rhs<double>(*m, p, yt.data(), k3.data());
    for (int i = 0; i < N; ++i) yt[i] = y[i] + h * k3[i];
    rhs<double>(*m, p, yt.data(), k4.data());
    for (int i = 0; i < N; ++i) y[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  }
}

void or_rodas4_tableau(double* gamma, double* A, double* C, double* M, double* E) {
  *gamma = RD_GAMMA;
  for (int i = 0; i < 6; ++i) {
    for (int j = 0; j < 6; ++j) { A[6 * i + j] = RD_A[i][j]; C[6 * i + j] = RD_C[i][j]; }
    M[i] = RD_M[i];
    E[i] = RD_E[i];
  }
}

void or_rodas4_linear(int N, const double* L, double* y, double h, int nsteps, double* err_last) {
  auto fun = [&](const double* yy, double* ff) {
    for (int i = 0; i < N; ++i) {
      double v = 0.0;
      for (int j = 0; j < N; ++j) v += L[(size_t)i * N + j] * yy[j];
      ff[i] = v;
    }
  };
  std::vector<double> f0(N), ynew(N), err(N);
  for (int s = 0; s < nsteps; ++s) {
    fun(y, f0.data());
    rodas4_attempt<double>(N, fun, y, f0.data(), L, h, ynew.data(), err.data());
    for (int i = 0; i < N; ++i) y[i] = ynew[i];
  }
  if (err_last)
    for (int i = 0; i < N; ++i) err_last[i] = err[i];
}

int or_count_ops(const or_mech* m, double p, const double* y, double dt, double rtol, double atol,
                 double* counts, int* nsub, int* nrej) {
  const int N = m->ns + 1;
  std::vector<CD> yc(N);
  for (int i = 0; i < N; ++i) yc[i] = CD(y[i]);
  g_ops = OpCounts{0, 0, 0, 0, 0, 0, 0, 0};
  int st = rodas4_integrate<CD>(*m, CD(p), yc.data(), dt, rtol, atol, 100000, nsub, nrej);
  counts[0] = g_ops.add; counts[1] = g_ops.mul; counts[2] = g_ops.div; counts[3] = g_ops.exp;
  counts[4] = g_ops.log; counts[5] = g_ops.pow; counts[6] = g_ops.sqrt; counts[7] = g_ops.cmp;
  return st;
}

}  // extern "C"
