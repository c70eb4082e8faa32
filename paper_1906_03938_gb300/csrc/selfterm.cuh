// FP64 device helpers shared by the kernels that evaluate the singular self term
// A_ll(k) = integral over triangle l of exp(i k r) / (4 pi r) about its centroid.
//
// Polar coordinates about the centroid x in the plane of the triangle: the radial
// integral is R h(i k R) with h(w) = (e^w - 1) / w; along each edge (d the distance from
// x to the edge's line, s the position along the edge from the foot of the perpendicular)
// the angle is traded for u = asinh(s / d), so R = d cosh(u), d(phi) = du / cosh(u) and
// the integrand d h(i k d cosh u) is entire in u; 16-point Gauss-Legendre on each side of
// u = 0.
#pragma once

#include <math.h>

namespace bem {

constexpr double kPiD = 3.141592653589793238462643383279502884;

struct GL16 {
  double x[16];
  double w[16];
};

// Gauss-Legendre nodes as the roots of P_16 by Newton's method (three-term recurrence).
inline GL16 make_gl16() {
  GL16 g;
  const int n = 16;
  for (int i = 0; i < n; ++i) {
    double x = cos(kPiD * (4.0 * i + 3.0) / (4.0 * n + 2.0));
    double dp = 1.0;
    for (int it = 0; it < 60; ++it) {
      double pm = 1.0, p = x;
      for (int k = 1; k < n; ++k) {
        const double pn = ((2 * k + 1) * x * p - k * pm) / (k + 1);
        pm = p;
        p = pn;
      }
      dp = n * (pm - x * p) / (1.0 - x * x);
      const double step = p / dp;
      x -= step;
      if (fabs(step) <= 4e-17) break;
    }
    double pm = 1.0, p = x;
    for (int k = 1; k < n; ++k) {
      const double pn = ((2 * k + 1) * x * p - k * pm) / (k + 1);
      pm = p;
      p = pn;
    }
    dp = n * (pm - x * p) / (1.0 - x * x);
    g.x[i] = x;
    g.w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  return g;
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// h(w) = (e^w - 1) / w; Taylor series sum_m w^m / (m + 1)! for |w| < 1/2.
__device__ inline double2 h_fun(double2 w) {
  if (w.x * w.x + w.y * w.y < 0.25) {
    double2 s = make_double2(0.0, 0.0), t = make_double2(1.0, 0.0);
    for (int m = 0; m < 24; ++m) {
      s.x += t.x;
      s.y += t.y;
      t = zmul(t, w);
      t.x /= (m + 2.0);
      t.y /= (m + 2.0);
    }
    return s;
  }
  double sn, cs;
  sincos(w.y, &sn, &cs);
  const double e = exp(w.x);
  const double2 num = make_double2(e * cs - 1.0, e * sn);
  const double d = w.x * w.x + w.y * w.y;
  return make_double2((num.x * w.x + num.y * w.y) / d, (num.y * w.x - num.x * w.y) / d);
}

// h'(w) = (w e^w - e^w + 1) / w^2; Taylor series sum_{m>=1} m w^{m-1} / (m + 1)! near 0.
__device__ inline double2 hprime_fun(double2 w) {
  if (w.x * w.x + w.y * w.y < 0.25) {
    double2 s = make_double2(0.0, 0.0), p = make_double2(1.0, 0.0);   // p = w^{m-1}
    double fact = 2.0;                                                // (m + 1)!
    for (int m = 1; m < 26; ++m) {
      s.x += m * p.x / fact;
      s.y += m * p.y / fact;
      p = zmul(p, w);
      fact *= (m + 2.0);
    }
    return s;
  }
  double sn, cs;
  sincos(w.y, &sn, &cs);
  const double e = exp(w.x);
  const double2 ew = make_double2(e * cs, e * sn);
  const double2 num = make_double2(zmul(w, ew).x - ew.x + 1.0, zmul(w, ew).y - ew.y);
  const double2 w2 = zmul(w, w);
  const double d = w2.x * w2.x + w2.y * w2.y;
  return make_double2((num.x * w2.x + num.y * w2.y) / d, (num.y * w2.x - num.x * w2.y) / d);
}

// Self term of the triangle with vertices v[0..2] about the point x, at wavenumber k.
// (deriv = true: its derivative in k, the integral of i R^2 h'(i k R) d(phi), i.e.
// i d^2 cosh(u) h'(i k d cosh u) du along each edge.)
__device__ inline double2 self_term(const double v[3][3], const double x[3], double2 k,
                                    const GL16& gl, bool deriv = false) {
  double2 total = make_double2(0.0, 0.0);
  for (int e = 0; e < 3; ++e) {
    const double* p = v[e];
    const double* q = v[(e + 1) % 3];
    double tx = q[0] - p[0], ty = q[1] - p[1], tz = q[2] - p[2];
    const double len = sqrt(tx * tx + ty * ty + tz * tz);
    tx /= len;
    ty /= len;
    tz /= len;
    const double px = p[0] - x[0], py = p[1] - x[1], pz = p[2] - x[2];
    const double qx = q[0] - x[0], qy = q[1] - x[1], qz = q[2] - x[2];
    const double sp = px * tx + py * ty + pz * tz;
    const double sq = qx * tx + qy * ty + qz * tz;
    const double ox = px - sp * tx, oy = py - sp * ty, oz = pz - sp * tz;
    const double d = sqrt(ox * ox + oy * oy + oz * oz);
    const double up = asinh(sp / d), uq = asinh(sq / d);
    const bool split = up < 0.0 && uq > 0.0;
    for (int s = 0; s < (split ? 2 : 1); ++s) {
      const double lo = split ? (s == 0 ? up : 0.0) : up;
      const double hi = split ? (s == 0 ? 0.0 : uq) : uq;
      const double half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
      for (int gi = 0; gi < 16; ++gi) {
        const double R = d * cosh(mid + half * gl.x[gi]);
        const double2 wv = make_double2(-k.y * R, k.x * R);   // i k R
        if (deriv) {
          const double2 hp = hprime_fun(wv);
          const double f = half * gl.w[gi] * d * R;         // d^2 cosh(u) = d R
          total.x += -f * hp.y;                               // i * hp
          total.y += f * hp.x;
        } else {
          const double2 h = h_fun(wv);
          const double f = half * gl.w[gi] * d;
          total.x += f * h.x;
          total.y += f * h.y;
        }
      }
    }
  }
  return make_double2(total.x / (4.0 * kPiD), total.y / (4.0 * kPiD));
}

// Edge data of the self term, FP64: for edge e = (v[e], v[e+1]) about the point x, the
// distance d from x to the edge's line and the u = asinh(s / d) range of the edge.
__device__ inline void self_edge(const double v[3][3], const double x[3], int e, double& d,
                                 double& up, double& uq) {
  const double* p = v[e];
  const double* q = v[(e + 1) % 3];
  double tx = q[0] - p[0], ty = q[1] - p[1], tz = q[2] - p[2];
  const double len = sqrt(tx * tx + ty * ty + tz * tz);
  tx /= len;
  ty /= len;
  tz /= len;
  const double px = p[0] - x[0], py = p[1] - x[1], pz = p[2] - x[2];
  const double qx = q[0] - x[0], qy = q[1] - x[1], qz = q[2] - x[2];
  const double sp = px * tx + py * ty + pz * tz;
  const double sq = qx * tx + qy * ty + qz * tz;
  const double ox = px - sp * tx, oy = py - sp * ty, oz = pz - sp * tz;
  d = sqrt(ox * ox + oy * oy + oz * oz);
  up = asinh(sp / d);
  uq = asinh(sq / d);
}

// FP32 version for the mixed path: given the edge data (d, u range per edge, computed in
// FP64), the angular quadrature and h(i k R) in FP32 (relative accuracy ~1e-6, the level
// of the mixed path). Returns the part of the sum over the angular nodes t = part,
// part + nparts, ... of the 96 = 3 edges x 2 sides x 16 nodes.
__device__ inline float2 self_term32_part(const float d3[3], const float up3[3],
                                          const float uq3[3], float kr, float ki,
                                          const GL16& gl, int part, int nparts) {
  float tr = 0.f, ti = 0.f;
  for (int t = part; t < 96; t += nparts) {
    const int e = t / 32, side = (t / 16) % 2, gi = t % 16;
    const float d = d3[e], up = up3[e], uq = uq3[e];
    // the two sides of u = 0 when the foot lies inside the edge, else the whole range once
    const bool split = up < 0.f && uq > 0.f;
    float lo, hi;
    if (split) {
      lo = side == 0 ? up : 0.f;
      hi = side == 0 ? 0.f : uq;
    } else {
      if (side == 1) continue;
      lo = up;
      hi = uq;
    }
    const float half = 0.5f * (hi - lo), mid = 0.5f * (hi + lo);
    const float R = d * coshf(mid + half * (float)gl.x[gi]);
    const float wr = -ki * R, wi = kr * R;   // w = i k R
    float hr, hi2;
    if (wr * wr + wi * wi < 0.25f) {
      // sum_m w^m / (m + 1)!, 10 terms
      float sr = 0.f, si = 0.f, cr = 1.f, ci = 0.f;
      for (int m = 0; m < 10; ++m) {
        sr += cr;
        si += ci;
        const float nr = (cr * wr - ci * wi) / (m + 2.0f);
        const float ni = (cr * wi + ci * wr) / (m + 2.0f);
        cr = nr;
        ci = ni;
      }
      hr = sr;
      hi2 = si;
    } else {
      float sn, cs;
      sincosf(wi, &sn, &cs);
      const float ex = expf(wr);
      const float nr = ex * cs - 1.f, ni = ex * sn;
      const float dd = wr * wr + wi * wi;
      hr = (nr * wr + ni * wi) / dd;
      hi2 = (ni * wr - nr * wi) / dd;
    }
    const float f = half * (float)gl.w[gi] * d;
    tr += f * hr;
    ti += f * hi2;
  }
  const float inv4pi = (float)(1.0 / (4.0 * kPiD));
  return make_float2(tr * inv4pi, ti * inv4pi);
}

}  // namespace bem
