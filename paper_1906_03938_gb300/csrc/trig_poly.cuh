// Polynomial sine and cosine on the FP32 FMA pipe (generated by trig_poly_fit.py:
// minimax fits of cos(pi f) and sin(pi f) / f in u = f^2 over |f| <= 1/2, FP32
// coefficients). The phase is reduced in half revolutions: t = phi / pi, n = rint(t)
// (by the 1.5 * 2^23 shift, which leaves n in the low bits of t + shift), f = t - n,
// e^{i phi} = (-1)^n e^{i pi f}; phi may be any FP32 value below ~1e6.
#pragma once

namespace bem {
namespace trig {

constexpr float kInvPi = 0.318309886f;
constexpr float kRoundShift = 12582912.0f;   // 1.5 * 2^23: x + s - s = rint(x)
constexpr float kS0 = 3.141592503e+00f;
constexpr float kS1 = -5.167703629e+00f;
constexpr float kS2 = 2.549984932e+00f;
constexpr float kS3 = -5.977979898e-01f;
constexpr float kS4 = 7.678086311e-02f;
constexpr float kC0 = 9.999999404e-01f;
constexpr float kC1 = -4.934792995e+00f;
constexpr float kC2 = 4.058412075e+00f;
constexpr float kC3 = -1.331880212e+00f;
constexpr float kC4 = 2.196968049e-01f;

}  // namespace trig
}  // namespace bem
