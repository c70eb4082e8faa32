// Geometry, contour and self-term kernels (FP64).
//
// * Panel geometry (the constant-element discretisation of Section 1): centroid x_l,
//   area |T_l| and Radon's 7-point degree-5 rule mapped onto each triangle. Weights are
//   stored as W_lq / (4 pi) so that an off-diagonal entry is sum_q qw * exp(i k r) / r.
// * Contour (Section 2, Eq. Tz, Eq. TzApp): trapezoid nodes theta_j = 2 pi (j + 1/2) / N;
//   or the Chebyshev points of a real interval (Eq. Chebyshev) with unit weights.
// * Self terms A_ll(z_j) for every panel and node (see selfterm.cuh), in FP64 for the plain
//   path and in FP32 for the mixed path.
#include <math.h>

#include "internal.h"
#include "selfterm.cuh"

namespace bem {
namespace {

struct Rule7 {
  double bary[7][3];
  double w[7];
};

// Radon's rule from its closed-form constants: the centroid with weight 9/40 and two
// orbits of three points (alpha, alpha, 1 - 2 alpha), alpha = (6 -+ sqrt 15) / 21, with
// weights (155 -+ sqrt 15) / 1200.
Rule7 make_rule7() {
  Rule7 r;
  const double s = sqrt(15.0);
  const double al[2] = {(6.0 - s) / 21.0, (6.0 + s) / 21.0};
  const double wt[2] = {(155.0 - s) / 1200.0, (155.0 + s) / 1200.0};
  r.bary[0][0] = r.bary[0][1] = r.bary[0][2] = 1.0 / 3.0;
  r.w[0] = 9.0 / 40.0;
  for (int o = 0; o < 2; ++o) {
    for (int p = 0; p < 3; ++p) {
      const int q = 1 + 3 * o + p;
      for (int c = 0; c < 3; ++c) r.bary[q][c] = (c == p) ? 1.0 - 2.0 * al[o] : al[o];
      r.w[q] = wt[o];
    }
  }
  return r;
}

__global__ void geometry_kernel(Geometry g, Rule7 rule, int* status) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g.pack32 && l >= g.n && l < (g.n + 15) / 16 * 16) {
    // padding panels of the packed array: finite placeholders, zero weights
    for (int t = 0; t < 64; ++t) g.pack32[l * 64 + t] = (t < 28 && t % 4 != 3) ? 1.0f : 0.0f;
    return;
  }
  if (l >= g.n) return;
  const int32_t i0 = g.tri[3 * l], i1 = g.tri[3 * l + 1], i2 = g.tri[3 * l + 2];
  if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= g.nv || i1 >= g.nv || i2 >= g.nv) {
    atomicOr(status, kStatusBadIndex);
    return;
  }
  double v[3][3];
  for (int c = 0; c < 3; ++c) {
    v[0][c] = g.xyz[3 * (int64_t)i0 + c];
    v[1][c] = g.xyz[3 * (int64_t)i1 + c];
    v[2][c] = g.xyz[3 * (int64_t)i2 + c];
  }
  const double e1[3] = {v[1][0] - v[0][0], v[1][1] - v[0][1], v[1][2] - v[0][2]};
  const double e2[3] = {v[2][0] - v[0][0], v[2][1] - v[0][1], v[2][2] - v[0][2]};
  const double nx = e1[1] * e2[2] - e1[2] * e2[1];
  const double ny = e1[2] * e2[0] - e1[0] * e2[2];
  const double nz = e1[0] * e2[1] - e1[1] * e2[0];
  const double area = 0.5 * sqrt(nx * nx + ny * ny + nz * nz);
  // degenerate: area below 1e-12 of the squared longest edge (an exact zero can come out
  // of the cross product as a rounding residue once products are fused)
  const double e3[3] = {v[2][0] - v[1][0], v[2][1] - v[1][1], v[2][2] - v[1][2]};
  const double l2 = fmax(fmax(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2],
                              e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]),
                         e3[0] * e3[0] + e3[1] * e3[1] + e3[2] * e3[2]);
  if (!(area > 1e-12 * l2) || !isfinite(area)) atomicOr(status, kStatusZeroArea);
  if (g.diam) {
    // panel diameter for the near-field criterion, rounded step by step (no fused
    // operations) so that the criterion is decided exactly as written
    double len2[3];
    const double* ed[3] = {e1, e2, e3};
    for (int t = 0; t < 3; ++t)
      len2[t] = __dadd_rn(__dadd_rn(__dmul_rn(ed[t][0], ed[t][0]), __dmul_rn(ed[t][1], ed[t][1])),
                          __dmul_rn(ed[t][2], ed[t][2]));
    g.diam[l] = fmax(fmax(sqrt(len2[0]), sqrt(len2[1])), sqrt(len2[2]));
  }
  const int64_t n = g.n;
  for (int c = 0; c < 3; ++c) {
    const double x = (v[0][c] + v[1][c] + v[2][c]) / 3.0;
    g.cx[c * n + l] = x;
    g.cx32[c * n + l] = (float)x;
  }
  {
    // unit normal in the vertex order (the double-layer kernel's n_y)
    const double inv = 1.0 / (2.0 * area);
    const double un[3] = {nx * inv, ny * inv, nz * inv};
    for (int c = 0; c < 3; ++c) {
      if (g.nrm) g.nrm[c * n + l] = un[c];
      if (g.pack32) g.pack32[(int64_t)l * 64 + 56 + c] = (float)un[c];
    }
  }
  for (int q = 0; q < 7; ++q) {
    for (int c = 0; c < 3; ++c) {
      const double p = rule.bary[q][0] * v[0][c] + rule.bary[q][1] * v[1][c] +
                       rule.bary[q][2] * v[2][c];
      g.qp[(7 * c + q) * n + l] = p;
      g.qp32[(7 * c + q) * n + l] = (float)p;
    }
    const double w = rule.w[q] * area / (4.0 * kPiD);
    g.qw[q * n + l] = w;
    g.qw32[q * n + l] = (float)w;
    if (g.pack32) {
      float* pk = g.pack32 + (int64_t)l * 64;
      for (int c = 0; c < 3; ++c) {
        const double pt = rule.bary[q][0] * v[0][c] + rule.bary[q][1] * v[1][c] +
                          rule.bary[q][2] * v[2][c];
        const float hi = (float)pt;
        pk[4 * q + c] = hi;
        pk[28 + 4 * q + c] = (float)(pt - (double)hi);
      }
      pk[4 * q + 3] = (float)w;
      pk[28 + 4 * q + 3] = 0.f;
    }
  }
  if (g.edge32) {
    // node-independent edge data of the FP32 self term, once per panel: the vertex offsets
    // from the centroid are formed in FP64, the rest in FP32 (the FP32 table needs no more)
    double x[3];
    for (int c = 0; c < 3; ++c) x[c] = (v[0][c] + v[1][c] + v[2][c]) / 3.0;
    float o[3][3];
    for (int e = 0; e < 3; ++e)
      for (int c = 0; c < 3; ++c) o[e][c] = (float)(v[e][c] - x[c]);
    for (int e = 0; e < 3; ++e) {
      const float* p = o[e];
      const float* q = o[(e + 1) % 3];
      float tx = q[0] - p[0], ty = q[1] - p[1], tz = q[2] - p[2];
      const float il = rsqrtf(tx * tx + ty * ty + tz * tz);
      tx *= il;
      ty *= il;
      tz *= il;
      const float sp = p[0] * tx + p[1] * ty + p[2] * tz;
      const float sq = q[0] * tx + q[1] * ty + q[2] * tz;
      const float fx = p[0] - sp * tx, fy = p[1] - sp * ty, fz = p[2] - sp * tz;
      const float d = sqrtf(fx * fx + fy * fy + fz * fz);
      g.edge32[(3 * e + 0) * n + l] = d;
      g.edge32[(3 * e + 1) * n + l] = asinhf(sp / d);
      g.edge32[(3 * e + 2) * n + l] = asinhf(sq / d);
    }
  }
}

__global__ void contour_kernel(int N, int kind, double c_re, double c_im, double a, double b,
                               double* z, double* w) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  if (kind == BEM_CONTOUR_CHEBYSHEV) {   // Chebyshev points of [c - a, c + a], unit weights
    z[2 * j] = c_re + a * cospi((j + 0.5) / N);
    z[2 * j + 1] = c_im;
    w[2 * j] = 1.0;
    w[2 * j + 1] = 0.0;
    return;
  }
  if (kind == BEM_CONTOUR_CIRCLE) b = a;
  // theta_j = pi (2 j + 1) / N; the lower half mirrors the upper (theta_{N-1-j} = 2 pi -
  // theta_j) exactly, so conjugate nodes have bit-equal real parts
  const int m = 2 * j + 1 > N ? N - 1 - j : j;
  double s, c;
  sincospi((2.0 * m + 1.0) / N, &s, &c);
  if (m != j) s = -s;
  z[2 * j] = c_re + a * c;
  z[2 * j + 1] = c_im + b * s;
  w[2 * j] = b * c / N;
  w[2 * j + 1] = a * s / N;
}

// One thread per (panel l, node j).
// T's self entry: c_G times the single-layer self integral plus c_H / 2 (the jump of H).
__global__ void self_term_kernel(Geometry g, int N, const double* z, GL16 gl, OpCoef op,
                                 double* self) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= g.n * (int64_t)N) return;
  const int64_t l = t % g.n;
  const int j = (int)(t / g.n);
  double v[3][3], x[3];
  for (int e = 0; e < 3; ++e) {
    const int32_t vi = g.tri[3 * l + e];
    for (int c = 0; c < 3; ++c) v[e][c] = g.xyz[3 * (int64_t)vi + c];
  }
  for (int c = 0; c < 3; ++c) x[c] = g.cx[c * g.n + l];
  const double2 a = self_term(v, x, make_double2(z[2 * j], z[2 * j + 1]), gl);
  self[2 * (j * g.n + l)] = op.cgr * a.x - op.cgi * a.y + 0.5 * op.chr;
  self[2 * (j * g.n + l) + 1] = op.cgr * a.y + op.cgi * a.x + 0.5 * op.chi;
}

// Moments of the FP32 self term. With f_g = half * w_g * d the angular weight of node g and
// R_g = d cosh(u_g) its radius, A_ll(k) = (1/4 pi) sum_g f_g h(i k R_g) and
// h(w) = sum_m w^m / (m + 1)!, so A_ll(k) = sum_m (i k rho)^m c_m with
// c_m = (1/4 pi) sum_g f_g (R_g / rho)^m / (m + 1)!, rho the panel's largest centroid-to-
// vertex distance (so R_g / rho <= 1 and c_m <= c_0 / (m + 1)!). The moments depend on the
// panel only; each node then costs one polynomial evaluation. One warp per panel; lane L
// takes the angular nodes L, L + 32, L + 64 and the sums are combined by a fixed shuffle tree.
__global__ void self_moments32_kernel(Geometry g, GL16 gl) {
  const int64_t l = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (l >= g.n) return;
  float d3[3], up3[3], uq3[3];
  float rho = 0.f;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    d3[e] = g.edge32[(3 * e + 0) * g.n + l];
    up3[e] = g.edge32[(3 * e + 1) * g.n + l];
    uq3[e] = g.edge32[(3 * e + 2) * g.n + l];
    rho = fmaxf(rho, d3[e] * coshf(fmaxf(fabsf(up3[e]), fabsf(uq3[e]))));
  }
  const float irho = 1.f / rho;
  float c[kSelfMoments];
#pragma unroll
  for (int m = 0; m < kSelfMoments; ++m) c[m] = 0.f;
  for (int t = lane; t < 96; t += 32) {
    const int e = t / 32, side = (t / 16) % 2, gi = t % 16;
    const float d = d3[e], up = up3[e], uq = uq3[e];
    const bool split = up < 0.f && uq > 0.f;   // the foot of the perpendicular inside the edge
    if (!split && side == 1) continue;
    const float lo = split ? (side == 0 ? up : 0.f) : up;
    const float hi = split ? (side == 0 ? 0.f : uq) : uq;
    const float half = 0.5f * (hi - lo), mid = 0.5f * (hi + lo);
    const float r = d * coshf(mid + half * (float)gl.x[gi]) * irho;
    float term = half * (float)gl.w[gi] * d;   // f_g (R / rho)^m / (m + 1)! at m = 0
#pragma unroll
    for (int m = 0; m < kSelfMoments; ++m) {
      c[m] += term;
      term *= r * (1.f / (float)(m + 2));
    }
  }
  const float inv4pi = (float)(1.0 / (4.0 * kPiD));
#pragma unroll
  for (int m = 0; m < kSelfMoments; ++m) {
    float v = c[m];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == m) g.mom32[(int64_t)m * g.n + l] = v * inv4pi;
  }
  if (lane == 0) g.rho32[l] = rho;
}

// |i k rho| up to which the FP32 self term is summed from the moments: the terms of the
// series grow to about e^x / x before they decay, so at x = 3.5 the sum loses about one
// decimal digit to cancellation, still far below the mixed path's ~1e-5 level. Beyond it
// (panels large against the wavelength) the angular quadrature is summed directly.
constexpr float kMomentReach = 3.5f;

// FP32 table for the mixed path, one thread per (panel l, node j): the moment series in
// i k rho by Horner's rule, truncated where x^M / (M + 1)! < 1.5e-8 (x = |k| rho), or the
// 96-node angular quadrature directly when x > kMomentReach or no moments exist.
__global__ void self_term32_kernel(Geometry g, int N, const double* z, GL16 gl, OpCoef op,
                                   float* self32) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= g.n * (int64_t)N) return;
  const int64_t l = t % g.n;
  const int j = (int)(t / g.n);
  const float kr = (float)z[2 * j], ki = (float)z[2 * j + 1];
  float2 out;
  const float rho = g.mom32 ? g.rho32[l] : 0.f;
  const float wr = -ki * rho, wi = kr * rho;   // i k rho
  const float x = sqrtf(wr * wr + wi * wi);
  if (g.mom32 && x <= kMomentReach) {
    int M = 1;
    float bound = 0.5f * x;   // x^M / (M + 1)!
    while (M < kSelfMoments && bound > 1.5e-8f) {
      ++M;
      bound *= x / (float)(M + 1);
    }
    float sr = g.mom32[(int64_t)(M - 1) * g.n + l], si = 0.f;
    for (int m = M - 2; m >= 0; --m) {
      const float nr = sr * wr - si * wi + g.mom32[(int64_t)m * g.n + l];
      si = sr * wi + si * wr;
      sr = nr;
    }
    out = make_float2(sr, si);
  } else {
    float d3[3], up3[3], uq3[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      d3[e] = g.edge32[(3 * e + 0) * g.n + l];
      up3[e] = g.edge32[(3 * e + 1) * g.n + l];
      uq3[e] = g.edge32[(3 * e + 2) * g.n + l];
    }
    out = self_term32_part(d3, up3, uq3, kr, ki, gl, 0, 1);
  }
  if (!op_single(op))   // T's self entry: c_G A_ll + c_H / 2
    out = make_float2((float)op.cgr * out.x - (float)op.cgi * out.y + 0.5f * (float)op.chr,
                      (float)op.cgr * out.y + (float)op.cgi * out.x + 0.5f * (float)op.chi);
  reinterpret_cast<float2*>(self32)[(int64_t)j * g.n + l] = out;
}

}  // namespace

cudaError_t launch_geometry(bem_ctx* ctx, cudaStream_t s) {
  static const Rule7 rule = make_rule7();
  const int64_t n = (ctx->geo.n + 15) / 16 * 16;   // padding panels of the packed array too
  // one thread per panel in 32-thread blocks: the FP64 work per panel is long and FP64
  // issue is slow, so the panels are spread over as many SMs as possible
  geometry_kernel<<<(unsigned)((n + 31) / 32), 32, 0, s>>>(ctx->geo, rule, ctx->d_status);
  ctx->launches++;
  if (ctx->geo.mom32) {
    static const GL16 gl = make_gl16();
    self_moments32_kernel<<<(unsigned)((32 * ctx->geo.n + 255) / 256), 256, 0, s>>>(ctx->geo, gl);
    ctx->launches++;
  }
  return cudaGetLastError();
}

cudaError_t launch_contour(bem_ctx* ctx, cudaStream_t s) {
  const Contour& c = ctx->con;
  contour_kernel<<<(c.N + 127) / 128, 128, 0, s>>>(c.N, c.kind, c.c_re, c.c_im, c.a, c.b, c.z,
                                                   c.w);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t launch_self_terms32(bem_ctx* ctx, cudaStream_t s) {
  static const GL16 gl = make_gl16();
  const int64_t total = ctx->geo.n * (int64_t)ctx->con.N;
  self_term32_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(ctx->geo, ctx->con.N,
                                                                     ctx->con.z, gl, ctx->op,
                                                                     ctx->con.self32);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t launch_self32(bem_ctx* ctx, int nk, const double* kz, float* out, cudaStream_t s) {
  static const GL16 gl = make_gl16();
  const int64_t total = ctx->geo.n * (int64_t)nk;
  self_term32_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(ctx->geo, nk, kz, gl, ctx->op,
                                                                     out);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t launch_self_terms(bem_ctx* ctx, cudaStream_t s) {
  static const GL16 gl = make_gl16();
  const int64_t total = ctx->geo.n * (int64_t)ctx->con.N;
  self_term_kernel<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(ctx->geo, ctx->con.N,
                                                                   ctx->con.z, gl, ctx->op,
                                                                   ctx->con.self);
  ctx->launches++;
  return cudaGetLastError();
}

}  // namespace bem
