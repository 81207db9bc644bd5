// GELU for the BF16 network epilogues (the single network's fused kernel and the per-species
// networks' GEMM epilogue).
#pragma once

namespace chem {

// GELU(v) = v Phi(v) = v (1 + erf(v / sqrt 2)) / 2, the exact (erf) form, with erf from
// Abramowitz & Stegun, Handbook of Mathematical Functions, 7.1.28:
//   erf(x) = 1 - (1 + a1 x + a2 x^2 + ... + a6 x^6)^-16 for x >= 0 (|error| <= 3e-7), odd in x.
// With r = (1 + a1 x + ...)^-16 at x = |v| / sqrt 2, GELU(v) = max(v, 0) - |v| r / 2 for either
// sign; the coefficients below are a_i / sqrt(2)^i, so the polynomial takes |v| directly.  One
// polynomial, four squarings and one approximate reciprocal (rcp.approx, relative error below
// 2^-22): GELU is within 5e-7 of the exact value, and the activation is rounded to BF16
// (relative step 2^-8) right after.
__device__ __forceinline__ float rcp_approx(float q) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(q));
  return r;
}

__device__ __forceinline__ float gelu_f(float v) {
  const float x = fabsf(v);
  float q = fmaf(x, 5.3829750000e-06f, 4.8890635643e-05f);
  q = fmaf(q, x, 3.8003575000e-05f);
  q = fmaf(q, x, 3.2776263241e-03f);
  q = fmaf(q, x, 2.1141006150e-02f);
  q = fmaf(q, x, 4.9867346967e-02f);
  q = fmaf(q, x, 1.0f);
  q = q * q;
  q = q * q;
  q = q * q;
  q = q * q;                                         // (...)^16; overflow to inf gives r = 0
  return fmaf(-0.5f * x, rcp_approx(q), fmaxf(v, 0.0f));
}

}  // namespace chem
