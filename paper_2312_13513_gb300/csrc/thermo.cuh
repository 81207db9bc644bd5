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

}  // namespace chem
