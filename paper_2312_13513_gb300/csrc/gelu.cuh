// GELU for the BF16 network epilogues (the single network's fused kernel and the per-species
// networks' GEMM epilogue).
#pragma once

namespace chem {

// GELU(v) = v Phi(v) = v (1 + erf(v / sqrt 2)) / 2, the exact (erf) form, with erf from
// Abramowitz & Stegun, Handbook of Mathematical Functions, 7.1.28:
//   erf(x) = 1 - (1 + a1 x + a2 x^2 + ... + a6 x^6)^-16 for x >= 0 (|error| <= 3e-7), odd in x.
// With r = (1 + a1 x + ...)^-16 at x = |v| / sqrt 2, GELU(v) = max(v, 0) - |v| r / 2 for either
// sign.  The coefficients below are c a_i / sqrt(2)^i with the constant term c = 2^(1/16): the
// polynomial takes |v| directly, and its 16th power is 2 (1 + a1 x + ...)^16, so its reciprocal
// is already r / 2 and the last step is one FMA.  One polynomial, four squarings and one
// approximate reciprocal (rcp.approx, relative error below 2^-22): GELU is within 5e-7 of the
// exact value, and the activation is rounded to BF16 (relative step 2^-8) right after.
__device__ __forceinline__ float rcp_approx(float q) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(q));
  return r;
}

__device__ __forceinline__ float gelu_f(float v) {
  const float x = fabsf(v);
  float q = fmaf(x, 5.6212998061e-06f, 5.1055209042e-05f);
  q = fmaf(q, x, 3.9686136006e-05f);
  q = fmaf(q, x, 3.4227392171e-03f);
  q = fmaf(q, x, 2.2076997906e-02f);
  q = fmaf(q, x, 5.2075162530e-02f);
  q = fmaf(q, x, 1.0442737341e+00f);
  q = q * q;
  q = q * q;
  q = q * q;
  q = q * q;                                         // (...)^16; overflow to inf gives r = 0
  return fmaf(x, rcp_approx(-q), fmaxf(v, 0.0f));
}

// Two GELUs at once with the packed FP32 instructions (fma/mul .f32x2: each half rounds exactly
// like the scalar instruction, so gelu2 gives bitwise the values of two gelu_f calls) at half the
// instruction count of the polynomial and the squarings; v0, v1 are updated in place.
__device__ __forceinline__ unsigned long long f32x2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}

__device__ __forceinline__ void f32x2_split(unsigned long long r, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}

__device__ __forceinline__ unsigned long long fma_x2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__device__ __forceinline__ unsigned long long mul_x2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

__device__ __forceinline__ unsigned long long add_x2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

__device__ __forceinline__ void gelu2(float& v0, float& v1) {
  const float x0 = fabsf(v0), x1 = fabsf(v1);
  const unsigned long long x = f32x2(x0, x1);
  unsigned long long q = fma_x2(x, f32x2(5.6212998061e-06f, 5.6212998061e-06f),
                                f32x2(5.1055209042e-05f, 5.1055209042e-05f));
  q = fma_x2(q, x, f32x2(3.9686136006e-05f, 3.9686136006e-05f));
  q = fma_x2(q, x, f32x2(3.4227392171e-03f, 3.4227392171e-03f));
  q = fma_x2(q, x, f32x2(2.2076997906e-02f, 2.2076997906e-02f));
  q = fma_x2(q, x, f32x2(5.2075162530e-02f, 5.2075162530e-02f));
  q = fma_x2(q, x, f32x2(1.0442737341e+00f, 1.0442737341e+00f));
  q = mul_x2(q, q);
  q = mul_x2(q, q);
  q = mul_x2(q, q);
  q = mul_x2(q, q);                                  // (...)^16
  float q0, q1;
  f32x2_split(q, q0, q1);
  const unsigned long long r = f32x2(rcp_approx(-q0), rcp_approx(-q1));
  const unsigned long long out = fma_x2(x, r, f32x2(fmaxf(v0, 0.0f), fmaxf(v1, 0.0f)));
  f32x2_split(out, v0, v1);
}

}  // namespace chem
