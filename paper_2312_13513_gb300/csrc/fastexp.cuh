// Table-driven FP64 exponential for the FP64-pipe-bound kernels (rates, fits).
//
// Method (Tang, "Table-driven implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15(2):144-157, 1989), restated:
//   n = round(64 x / ln 2), r = x - n ln 2 / 64 (|r| <= ln 2 / 128, ln 2 / 64 as a double-double),
//   exp(x) = 2^(n >> 6) * 2^((n & 63) / 64) * exp(r),
// with 2^(j / 64) from a 64-entry table and exp(r) from its degree-5 Taylor polynomial (the
// truncation, r^6 / 720, stays below 4e-17 relative).  The rounding of 64 x / ln 2 uses the
// 1.5 * 2^52 shifter: after one FMA the integer n sits in the low mantissa bits, so no
// float-to-integer conversion is needed, and 2^(n >> 6) is added to the table entry's exponent
// field with integer arithmetic.  Ten FP64 instructions in all.  Arguments with |x| >= 700 (and
// NaN) take the library exp, so overflow, underflow and subnormal results keep their usual
// meaning.  The table lives in shared memory (indices differ across lanes).
#pragma once
#include <stdint.h>

#include "exp_table.h"

namespace chem {

// device copy of the table, for kernels that stage it into shared memory themselves
static __constant__ double c_exp_table[64] = {CHEM_EXP_TABLE_VALUES};

__device__ __forceinline__ void stage_exp_table(double* dst) {
  for (int i = threadIdx.x; i < 64; i += blockDim.x) dst[i] = c_exp_table[i];
}

__device__ __forceinline__ double exp_tab(double x, const double* __restrict__ tab) {
  const int hx = __double2hiint(x) & 0x7fffffff;
  if (hx >= 0x4085e000) return exp(x);                       // |x| >= 700, inf, NaN
  const double kShift = 6755399441055744.0;                  // 1.5 * 2^52
  const double t = fma(x, kExpInvStep, kShift);
  const int n = __double2loint(t);                           // round(64 x / ln 2)
  const double nd = t - kShift;
  double r = fma(-nd, kExpStepHi, x);
  r = fma(-nd, kExpStepLo, r);
  double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  q = fma(q, r, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  q = fma(q, r, 1.0);
  q = fma(q, r, 1.0);
  const double tj = tab[n & 63];
  const int escale = (int)((unsigned)(n >> 6) << 20);         // 2^(n >> 6) in the exponent field
  const double s = __hiloint2double(__double2hiint(tj) + escale, __double2loint(tj));
  return s * q;
}

}  // namespace chem
