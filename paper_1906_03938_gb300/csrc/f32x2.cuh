// Packed FP32 pairs and the polynomial sine / cosine of the fused kernel's evaluation.
//
// The evaluation handles two entries of a row at once (its two columns of the 16-wide
// K-block), so their identical arithmetic goes through the paired FP32 instructions (one
// instruction per two lanes' worth of work; same rounding as the scalar operations).
#pragma once

#include "trig_poly.cuh"

namespace bem {

typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2(float a, float b) {
  f2_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2split(f2_t v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2_t mul2(f2_t a, f2_t b) {
  f2_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2_t add2(f2_t a, f2_t b) {
  f2_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2_t sub2(f2_t a, f2_t b) {
  f2_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2_t fma2(f2_t a, f2_t b, f2_t c) {
  f2_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ f2_t f2dup(float a) { return f2(a, a); }

// e^{i phi} of two phases on the FMA pipe (the polynomials of trig_poly.cuh): with
// t = phi / pi, n = rint(t), f = t - n,  e^{i phi} = (-1)^n (cos(pi f) + i sin(pi f)).
// Returns cos(pi f) and sin(pi f) of both lanes, and (-1)^n of both lanes as a mask of
// their sign bits: XOR it into the bits of the factor that multiplies them.
__device__ __forceinline__ void sincos_poly2(f2_t ph, f2_t& c, f2_t& s, f2_t& sign) {
  using namespace trig;
  const f2_t t = mul2(ph, f2dup(kInvPi));
  const f2_t tb = add2(t, f2dup(kRoundShift));   // n in the low bits of both lanes
  const f2_t f = sub2(t, sub2(tb, f2dup(kRoundShift)));
  const f2_t u = mul2(f, f);
  f2_t ps = fma2(f2dup(kS4), u, f2dup(kS3));
  ps = fma2(ps, u, f2dup(kS2));
  ps = fma2(ps, u, f2dup(kS1));
  ps = fma2(ps, u, f2dup(kS0));
  s = mul2(f, ps);
  f2_t pc = fma2(f2dup(kC4), u, f2dup(kC3));
  pc = fma2(pc, u, f2dup(kC2));
  pc = fma2(pc, u, f2dup(kC1));
  c = fma2(pc, u, f2dup(kC0));
  unsigned lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(tb));
  lo <<= 31;
  hi <<= 31;
  asm("mov.b64 %0, {%1, %2};" : "=l"(sign) : "r"(lo), "r"(hi));
}

}  // namespace bem
