// Mixture thermodynamics of one cell from the NASA-7 coefficients of the mechanism blob (device
// code shared by the surrogate's post-processing and the thermo kernels).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "chem_internal.h"

namespace chem {

// Mass-specific enthalpy h (erg/g, formation included) and cp (erg/(g K)) at temperature T of
// the composition Yloc[k] (if given) or Y[k * ld + cell].
__device__ __forceinline__ void h_cp_mass(const unsigned char* blob, const MechLayout& L, double T,
                                          const double* Y, int64_t ld, int64_t cell, const double* Yloc,
                                          double* h, double* cp) {
  const int ns = L.ns;
  const int rg = T < TMID ? 0 : 1;
  const double* hc = (const double*)(blob + L.o_hc);
  const double* cc = (const double*)(blob + L.o_cpc);
  const double* invW = (const double*)(blob + L.o_invW);
  const double invT = 1.0 / T;
  double hs = 0.0, cs = 0.0;
  for (int k = 0; k < ns; ++k) {
    const double* a = hc + (rg * ns + k) * 6;
    const double* c = cc + (rg * ns + k) * 5;
    const double hRT = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4]))) + a[5] * invT;
    const double cpR = c[0] + T * (c[1] + T * (c[2] + T * (c[3] + T * c[4])));
    const double yk = Yloc ? Yloc[k] : Y[k * ld + cell];
    hs += yk * hRT * __ldg(invW + k);
    cs += yk * cpR * __ldg(invW + k);
  }
  *h = RU * T * hs;
  *cp = RU * cs;
}

// Mass-specific enthalpy alone (erg/g, formation included) of the composition Yloc at T, as the
// polynomial h / R = a5 + a0 T + a1 T^2 + ... + a4 T^5 per species (no division by T).
__device__ __forceinline__ double h_mass(const unsigned char* blob, const MechLayout& L, double T,
                                         const double* Yloc) {
  const int ns = L.ns;
  const int rg = T < TMID ? 0 : 1;
  const double* hc = (const double*)(blob + L.o_hc);
  const double* invW = (const double*)(blob + L.o_invW);
  double hs = 0.0;
  for (int k = 0; k < ns; ++k) {
    const double* a = hc + (rg * ns + k) * 6;
    const double hR = a[5] + T * (a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4]))));
    hs += Yloc[k] * hR * __ldg(invW + k);
  }
  return RU * hs;
}

// The mixture's NASA-7 polynomials for one temperature range: for mass fractions Yloc,
// Ah[i] = sum_k Y_k / W_k a_ik (the h/RT coefficients, a6 included) and Ac[i] likewise for cp/R,
// so that h = R T (Ah0 + Ah1 T + ... + Ah4 T^4 + Ah5 / T) and cp = R (Ac0 + ... + Ac4 T^4): a
// Newton iteration on T at fixed composition then costs one polynomial instead of one per
// species (the same sums, reordered).
__device__ __forceinline__ void mixture_nasa(const unsigned char* blob, const MechLayout& L, int rg,
                                             const double* Yloc, double Ah[6], double Ac[5]) {
  const int ns = L.ns;
  const double* hc = (const double*)(blob + L.o_hc);
  const double* cc = (const double*)(blob + L.o_cpc);
  const double* invW = (const double*)(blob + L.o_invW);
  for (int i = 0; i < 6; ++i) Ah[i] = 0.0;
  for (int i = 0; i < 5; ++i) Ac[i] = 0.0;
  for (int k = 0; k < ns; ++k) {
    const double yw = Yloc[k] * __ldg(invW + k);
    const double* a = hc + (rg * ns + k) * 6;
    const double* c = cc + (rg * ns + k) * 5;
    for (int i = 0; i < 6; ++i) Ah[i] = fma(yw, a[i], Ah[i]);
    for (int i = 0; i < 5; ++i) Ac[i] = fma(yw, c[i], Ac[i]);
  }
}

// h and cp of a mixture polynomial at T; h = R (Ah5 + Ah0 T + ... + Ah4 T^5), no division by T
__device__ __forceinline__ void h_cp_from_mixture(const double Ah[6], const double Ac[5], double T, double* h,
                                                  double* cp) {
  *h = RU * (Ah[5] + T * (Ah[0] + T * (Ah[1] + T * (Ah[2] + T * (Ah[3] + T * Ah[4])))));
  *cp = RU * (Ac[0] + T * (Ac[1] + T * (Ac[2] + T * (Ac[3] + T * Ac[4]))));
}

}  // namespace chem
