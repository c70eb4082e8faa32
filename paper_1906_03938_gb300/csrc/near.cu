// Near field: a finer rule on panel pairs close to each other.
//
// The 7-point rule (Section 1's Gauss quadrature of the regular integrals) loses accuracy
// when the collocation point x_i is close to panel l. A pair (i, l), i != l, is near when
// the centroid distance is below twice the larger panel diameter (longest edge); its entry
// is then the 8 x 8 conical-product rule: the triangle (a, b, c) is the image of the unit
// square under y = a + s (b - a) + s t (c - b) (Jacobian 2 |T| s), with Gauss-Legendre in s
// and t, collapsed at the vertex nearest x_i (the first in the triangle's order on a tie).
// The matrix-free kernels keep the 7-point rule everywhere; the near pairs are corrected by
// (A_near - A_7) applied as a sparse matrix, which is what this file provides:
//   * the pair list (CSR, columns increasing within a row), decided in FP64 with the
//     criterion rounded step by step exactly as written, after an FP32 prefilter;
//   * Y_j += C(z_j) V for the FP64 projection, the same in FP32 into a slice of the mixed
//     path's partial products, and R[:, c] += C(lam_c) X[:, c] (values or k-derivatives)
//     for residuals and refinement.
// FP64 and residual paths: one warp per (row, node) or (row, column), whose lanes evaluate
// the row's pair corrections and then sweep the basis columns with them. FP32 path: the
// values of every (pair, node) first, by the 8 x 8 rule (a thread per pair and 8 nodes) or
// by the surrogate network on the tensor core (128-sample tiles), then one warp per (row,
// node) sweeps the basis columns with them. Every sum runs in a fixed order, so the results
// are deterministic.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "sm100.cuh"
#include "surrogate.cuh"

namespace bem {
namespace {

using namespace sm100;

constexpr double kPi = 3.141592653589793238462643383279502884;

struct GL8 {
  double x[8];   // nodes on [0, 1]
  double w[8];
};

// Gauss-Legendre nodes as the roots of P_8 (Newton's method on the three-term recurrence),
// mapped to [0, 1].
GL8 make_gl8() {
  GL8 g;
  const int n = 8;
  for (int i = 0; i < n; ++i) {
    double x = cos(kPi * (4.0 * i + 3.0) / (4.0 * n + 2.0));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double pm = 1.0, p = x;
      for (int k = 1; k < n; ++k) {
        const double pn = ((2 * k + 1) * x * p - k * pm) / (k + 1);
        pm = p;
        p = pn;
      }
      dp = n * (pm - x * p) / (1.0 - x * x);
      const double step = p / dp;
      x -= step;
      if (fabs(step) <= 1e-17) break;
    }
    double pm = 1.0, p = x;
    for (int k = 1; k < n; ++k) {
      const double pn = ((2 * k + 1) * x * p - k * pm) / (k + 1);
      pm = p;
      p = pn;
    }
    dp = n * (pm - x * p) / (1.0 - x * x);
    g.x[i] = 0.5 * (x + 1.0);
    g.w[i] = 0.5 * 2.0 / ((1.0 - x * x) * dp * dp);
  }
  return g;
}

// |a - b| rounded step by step (no fused operations)
__device__ __forceinline__ double dist_rn(const double a[3], const double b[3]) {
  const double dx = __dsub_rn(a[0], b[0]), dy = __dsub_rn(a[1], b[1]), dz = __dsub_rn(a[2], b[2]);
  return sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}

constexpr int kScanTile = 256;

// Near pairs of every row: counts (cols == nullptr) or the columns themselves at
// row_ptr[i] in increasing order. One thread per row; the columns' centroids and
// diameters are staged through shared memory, first tested in FP32 with a margin, then
// exactly in FP64.
__global__ void __launch_bounds__(kScanTile)
near_scan_kernel(Geometry g, int32_t* __restrict__ counts, const int32_t* __restrict__ row_ptr,
                 int32_t* __restrict__ cols) {
  __shared__ float4 sc[kScanTile];
  const int64_t n = g.n;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double xi[3] = {0.0, 0.0, 0.0};
  double hi = 0.0;
  if (i < n) {
    for (int c = 0; c < 3; ++c) xi[c] = g.cx[c * n + i];
    hi = g.diam[i];
  }
  const float fx = (float)xi[0], fy = (float)xi[1], fz = (float)xi[2], fh = (float)hi;
  int32_t cnt = 0;
  const int64_t base = (cols && i < n) ? row_ptr[i] : 0;
  for (int64_t l0 = 0; l0 < n; l0 += kScanTile) {
    __syncthreads();
    const int64_t lt = l0 + threadIdx.x;
    sc[threadIdx.x] = lt < n ? make_float4((float)g.cx[lt], (float)g.cx[n + lt],
                                           (float)g.cx[2 * n + lt], (float)g.diam[lt])
                             : make_float4(3e30f, 3e30f, 3e30f, 0.f);
    __syncthreads();
    if (i >= n) continue;
    const int lim = (int)(n - l0 < kScanTile ? n - l0 : kScanTile);
    for (int t = 0; t < lim; ++t) {
      const float4 c = sc[t];
      const float dx = fx - c.x, dy = fy - c.y, dz = fz - c.z;
      const float hm = fmaxf(fh, c.w);
      if (dx * dx + dy * dy + dz * dz > 4.02f * hm * hm + 1e-30f) continue;
      const int64_t l = l0 + t;
      if (l == i) continue;
      const double xl[3] = {g.cx[l], g.cx[n + l], g.cx[2 * n + l]};
      if (dist_rn(xi, xl) < 2.0 * fmax(hi, g.diam[l])) {
        if (cols) cols[base + cnt] = (int32_t)l;
        ++cnt;
      }
    }
  }
  if (i < n && !cols) counts[i] = cnt;
}

// The 8 x 8 rule's frame for panel l seen from x: collapsed vertex a (nearest x), the two
// edge vectors and 2 |T| / (4 pi).
struct NearFrame {
  double a[3], ab[3], bc[3];
  double scale;
};

__device__ void near_frame(const Geometry& g, int64_t l, const double x[3], NearFrame& F) {
  double v[3][3];
  for (int e = 0; e < 3; ++e) {
    const int32_t vi = g.tri[3 * l + e];
    for (int c = 0; c < 3; ++c) v[e][c] = g.xyz[3 * (int64_t)vi + c];
  }
  int a = 0;
  double best = dist_rn(v[0], x);
  for (int q = 1; q < 3; ++q) {
    const double r = dist_rn(v[q], x);
    if (r < best) {
      best = r;
      a = q;
    }
  }
  const double* A = v[a];
  const double* B = v[(a + 1) % 3];
  const double* C = v[(a + 2) % 3];
  for (int c = 0; c < 3; ++c) {
    F.a[c] = A[c];
    F.ab[c] = B[c] - A[c];
    F.bc[c] = C[c] - B[c];
  }
  const double nx = F.ab[1] * F.bc[2] - F.ab[2] * F.bc[1];
  const double ny = F.ab[2] * F.bc[0] - F.ab[0] * F.bc[2];
  const double nz = F.ab[0] * F.bc[1] - F.ab[1] * F.bc[0];
  F.scale = sqrt(nx * nx + ny * ny + nz * nz) / (4.0 * kPi);
}

// kernel value e^{ikr}/r (deriv: i e^{ikr}) times w, added to acc
__device__ __forceinline__ void add_kernel64(double2& acc, double w, double r, double kr,
                                             double ki, bool deriv) {
  double s, c;
  sincos(kr * r, &s, &c);
  const double amp = deriv ? w * exp(-ki * r) : w * exp(-ki * r) / r;
  if (deriv) {
    acc.x -= amp * s;
    acc.y += amp * c;
  } else {
    acc.x += amp * c;
    acc.y += amp * s;
  }
}

// (T_near - T_7)(k) of the pair (x, l), FP64; deriv: its k-derivative.
__device__ double2 near_corr64(const Geometry& g, int64_t l, const double x[3], double kr,
                               double ki, bool deriv, const GL8& gl, const OpCoef& op) {
  NearFrame F;
  near_frame(g, l, x, F);
  double2 acc = make_double2(0.0, 0.0);
  if (!op_single(op)) {   // the general operator: both kernels at every point
    const int64_t n = g.n;
    const double nx = g.nrm[l], ny = g.nrm[n + l], nz = g.nrm[2 * n + l];
    for (int p = 0; p < 8; ++p) {
      const double sp = gl.x[p];
      for (int q = 0; q < 8; ++q) {
        const double st = sp * gl.x[q];
        const double y0 = F.a[0] + sp * F.ab[0] + st * F.bc[0];
        const double y1 = F.a[1] + sp * F.ab[1] + st * F.bc[1];
        const double y2 = F.a[2] + sp * F.ab[2] + st * F.bc[2];
        op_point64(acc, op, gl.w[p] * gl.w[q] * sp * F.scale, y0 - x[0], y1 - x[1], y2 - x[2],
                   nx, ny, nz, kr, ki, deriv);
      }
    }
    for (int q = 0; q < 7; ++q)
      op_point64(acc, op, -g.qw[q * n + l], g.qp[q * n + l] - x[0],
                 g.qp[(7 + q) * n + l] - x[1], g.qp[(14 + q) * n + l] - x[2], nx, ny, nz, kr,
                 ki, deriv);
    return acc;
  }
  for (int p = 0; p < 8; ++p) {
    const double sp = gl.x[p];
    for (int q = 0; q < 8; ++q) {
      const double st = sp * gl.x[q];
      const double y0 = F.a[0] + sp * F.ab[0] + st * F.bc[0];
      const double y1 = F.a[1] + sp * F.ab[1] + st * F.bc[1];
      const double y2 = F.a[2] + sp * F.ab[2] + st * F.bc[2];
      const double dx = x[0] - y0, dy = x[1] - y1, dz = x[2] - y2;
      add_kernel64(acc, gl.w[p] * gl.w[q] * sp * F.scale, sqrt(dx * dx + dy * dy + dz * dz), kr,
                   ki, deriv);
    }
  }
  const int64_t n = g.n;
  for (int q = 0; q < 7; ++q) {
    const double dx = x[0] - g.qp[q * n + l], dy = x[1] - g.qp[(7 + q) * n + l],
                 dz = x[2] - g.qp[(14 + q) * n + l];
    add_kernel64(acc, -g.qw[q * n + l], sqrt(dx * dx + dy * dy + dz * dz), kr, ki, deriv);
  }
  return acc;
}

// Canonical features of the pair for the surrogate network: the frame has its origin at
// x, e1 along (b - a), e3 along the normal (b - a) x (c - b) flipped so that a lies on its
// non-negative side, e2 = e3 x e1; the three vertices in that frame divided by the
// panel's diameter h, then Re(k h), Im(k h).
__device__ void near_features32(const Geometry& g, int64_t l, const NearFrame& F, const double x[3],
                                float kr, float ki, float feat[kNetIn]) {
  const double h = g.diam[l];
  double e1[3] = {F.ab[0], F.ab[1], F.ab[2]};
  double n1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  for (int c = 0; c < 3; ++c) e1[c] /= n1;
  double e3[3] = {F.ab[1] * F.bc[2] - F.ab[2] * F.bc[1], F.ab[2] * F.bc[0] - F.ab[0] * F.bc[2],
                  F.ab[0] * F.bc[1] - F.ab[1] * F.bc[0]};
  double n3 = sqrt(e3[0] * e3[0] + e3[1] * e3[1] + e3[2] * e3[2]);
  for (int c = 0; c < 3; ++c) e3[c] /= n3;
  const double ax[3] = {F.a[0] - x[0], F.a[1] - x[1], F.a[2] - x[2]};
  if (ax[0] * e3[0] + ax[1] * e3[1] + ax[2] * e3[2] < 0.0)
    for (int c = 0; c < 3; ++c) e3[c] = -e3[c];
  const double e2[3] = {e3[1] * e1[2] - e3[2] * e1[1], e3[2] * e1[0] - e3[0] * e1[2],
                        e3[0] * e1[1] - e3[1] * e1[0]};
  double p[3][3];
  for (int c = 0; c < 3; ++c) {
    p[0][c] = ax[c];
    p[1][c] = ax[c] + F.ab[c];
    p[2][c] = ax[c] + F.ab[c] + F.bc[c];
  }
  for (int v = 0; v < 3; ++v) {
    feat[3 * v + 0] = (float)((p[v][0] * e1[0] + p[v][1] * e1[1] + p[v][2] * e1[2]) / h);
    feat[3 * v + 1] = (float)((p[v][0] * e2[0] + p[v][1] * e2[1] + p[v][2] * e2[2]) / h);
    feat[3 * v + 2] = (float)((p[v][0] * e3[0] + p[v][1] * e3[1] + p[v][2] * e3[2]) / h);
  }
  feat[9] = (float)(kr * h);
  feat[10] = (float)(ki * h);
}

// (A_near - A_7)(k) of the pair by the 8 x 8 rule, FP32 with coordinates relative to x
// (formed in FP64): the surrogate's value for pairs outside its training box.
__device__ float2 near_corr32(const Geometry& g, int64_t l, const double x[3], float kr,
                              float ki, const GL8& gl, const OpCoef& op) {
  NearFrame F;
  near_frame(g, l, x, F);
  if (!op_single(op)) {   // the general operator: the FP64 correction, rounded
    const double2 c = near_corr64(g, l, x, (double)kr, (double)ki, false, gl, op);
    return make_float2((float)c.x, (float)c.y);
  }
  const float ax = (float)(F.a[0] - x[0]), ay = (float)(F.a[1] - x[1]), az = (float)(F.a[2] - x[2]);
  const float abx = (float)F.ab[0], aby = (float)F.ab[1], abz = (float)F.ab[2];
  const float bcx = (float)F.bc[0], bcy = (float)F.bc[1], bcz = (float)F.bc[2];
  const float scale = (float)F.scale;
  float sr = 0.f, si = 0.f;
  for (int p = 0; p < 8; ++p) {
    const float sp = (float)gl.x[p];
    for (int q = 0; q < 8; ++q) {
      const float st = sp * (float)gl.x[q];
      const float dx = ax + sp * abx + st * bcx, dy = ay + sp * aby + st * bcy,
                  dz = az + sp * abz + st * bcz;
      const float r = sqrtf(dx * dx + dy * dy + dz * dz);
      float s, c;
      sincosf(kr * r, &s, &c);
      const float amp = (float)(gl.w[p] * gl.w[q]) * sp * scale * expf(-ki * r) / r;
      sr += amp * c;
      si += amp * s;
    }
  }
  const int64_t n = g.n;
  for (int q = 0; q < 7; ++q) {
    const float dx = (float)(g.qp[q * n + l] - x[0]), dy = (float)(g.qp[(7 + q) * n + l] - x[1]),
                dz = (float)(g.qp[(14 + q) * n + l] - x[2]);
    const float r = sqrtf(dx * dx + dy * dy + dz * dz);
    float s, c;
    sincosf(kr * r, &s, &c);
    const float amp = (float)g.qw[q * n + l] * expf(-ki * r) / r;
    sr -= amp * c;
    si -= amp * s;
  }
  return make_float2(sr, si);
}

constexpr int kMaxColGroups = kMaxNu / 32;

// Y_j += C(z_j) V, FP64: one warp per (row i, node j); Vt is V row-major (nu per row).
__global__ void __launch_bounds__(256)
near_apply64_kernel(Geometry g, const int32_t* __restrict__ ptr, const int32_t* __restrict__ cols,
                    const double* __restrict__ z, int N, const double2* __restrict__ Vt, int nu,
                    double2* __restrict__ Y, GL8 gl, OpCoef op) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  const int64_t n = g.n;
  if (w >= n * (int64_t)N) return;
  const int64_t i = w % n;
  const int node = (int)(w / n);
  const double kr = z[2 * node], ki = z[2 * node + 1];
  const double x[3] = {g.cx[i], g.cx[n + i], g.cx[2 * n + i]};
  double2 acc[kMaxColGroups];
#pragma unroll
  for (int t = 0; t < kMaxColGroups; ++t) acc[t] = make_double2(0.0, 0.0);
  const int32_t e0 = ptr[i], e1 = ptr[i + 1];
  for (int32_t eb = e0; eb < e1; eb += 32) {
    const int32_t e = eb + lane;
    double2 cval = make_double2(0.0, 0.0);
    int32_t l = 0;
    if (e < e1) {
      l = cols[e];
      cval = near_corr64(g, l, x, kr, ki, false, gl, op);
    }
    const int cnt = min(32, e1 - eb);
    for (int t = 0; t < cnt; ++t) {
      const double cx = __shfl_sync(0xffffffffu, cval.x, t);
      const double cy = __shfl_sync(0xffffffffu, cval.y, t);
      const int32_t lt = __shfl_sync(0xffffffffu, l, t);
      const double2* vr = Vt + (int64_t)lt * nu;
#pragma unroll
      for (int cg = 0; cg < kMaxColGroups; ++cg) {
        const int c = lane + 32 * cg;
        if (c < nu) {
          const double2 v = vr[c];
          acc[cg].x += cx * v.x - cy * v.y;
          acc[cg].y += cx * v.y + cy * v.x;
        }
      }
    }
  }
  if (e1 == e0) return;
  double2* Yj = Y + (int64_t)node * n * nu;
#pragma unroll
  for (int cg = 0; cg < kMaxColGroups; ++cg) {
    const int c = lane + 32 * cg;
    if (c < nu) {
      double2 y = Yj[(int64_t)c * n + i];
      y.x += acc[cg].x;
      y.y += acc[cg].y;
      Yj[(int64_t)c * n + i] = y;
    }
  }
}

// Row of every pair of the list (rows[e] = i for e in [ptr[i], ptr[i + 1])).
__global__ void near_rows_kernel(const int32_t* __restrict__ ptr, int64_t n, int32_t* __restrict__ rows) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int32_t e = ptr[i]; e < ptr[i + 1]; ++e) rows[e] = (int32_t)i;
}

constexpr int kNearNodes = 8;   // contour nodes per thread of the value kernel

// C[j][e] = (A_near - A_7)(z_j) of pair e (FP32; with the general operator, T's point
// terms with the factor c_G + c_H s (i k r - 1), s = (d . n) / r^2): one thread per pair and
// group of up to 8 nodes. The pair's frame (FP64, rounded to FP32 relative to x_i) and the
// 71 points' distances are formed once and shared by the group's nodes, whose kernel
// values take one ex2 and one sine / cosine each (MUFU approximations, as the fused
// kernel's; the FP64 path and the residuals keep the exact functions).
template <bool general>
__global__ void __launch_bounds__(256, 3)
near_values32_kernel(Geometry g, const int32_t* __restrict__ rows, const int32_t* __restrict__ cols,
                     int64_t nnz, const double* __restrict__ z, int N, GL8 gl, OpCoef op,
                     float2* __restrict__ Cv) {
  __shared__ float s_x[8], s_w[64];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      s_x[p] = (float)gl.x[p];
#pragma unroll
      for (int q = 0; q < 8; ++q) s_w[8 * p + q] = (float)(gl.w[p] * gl.w[q]);
    }
  }
  __syncthreads();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int groups = (N + kNearNodes - 1) / kNearNodes;
  if (t >= nnz * groups) return;
  const int64_t e = t % nnz;
  const int j0 = (int)(t / nnz) * kNearNodes;
  const int cnt = min(kNearNodes, N - j0);
  const int64_t n = g.n;
  const int64_t i = rows[e], l = cols[e];
  const double x[3] = {g.cx[i], g.cx[n + i], g.cx[2 * n + i]};
  NearFrame F;
  near_frame(g, l, x, F);
  const float ax = (float)(F.a[0] - x[0]), ay = (float)(F.a[1] - x[1]), az = (float)(F.a[2] - x[2]);
  const float abx = (float)F.ab[0], aby = (float)F.ab[1], abz = (float)F.ab[2];
  const float bcx = (float)F.bc[0], bcy = (float)F.bc[1], bcz = (float)F.bc[2];
  const float scale = (float)F.scale;
  float nx = 0.f, ny = 0.f, nz = 0.f;
  if constexpr (general) {
    nx = (float)g.nrm[l];
    ny = (float)g.nrm[n + l];
    nz = (float)g.nrm[2 * n + l];
  }
  float kr[kNearNodes], ki[kNearNodes];
  float2 acc[kNearNodes];
#pragma unroll
  for (int u = 0; u < kNearNodes; ++u) {
    const int j = j0 + (u < cnt ? u : 0);
    kr[u] = (float)z[2 * j];
    ki[u] = (float)z[2 * j + 1];
    acc[u] = make_float2(0.f, 0.f);
  }
  // amp = W / r at distance r (sr = (d . n) / r^2 for the general operator), added for every
  // node of the group
  auto add = [&](float amp, float r, float sr) {
#pragma unroll
    for (int u = 0; u < kNearNodes; ++u) {
      float sn, cs, ex;
      asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(ex) : "f"(-ki[u] * 1.4426950408889634f * r));
      __sincosf(kr[u] * r, &sn, &cs);
      const float a = amp * ex;
      if constexpr (general) {
        float fr, fi;
        op_factor(op, sr, kr[u] * r, ki[u] * r, fr, fi);
        acc[u].x += a * (cs * fr - sn * fi);
        acc[u].y += a * (cs * fi + sn * fr);
      } else {
        acc[u].x = fmaf(a, cs, acc[u].x);
        acc[u].y = fmaf(a, sn, acc[u].y);
      }
    }
  };
#pragma unroll 1
  for (int p = 0; p < 8; ++p) {
    const float sp = s_x[p];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float st = sp * s_x[q];
      const float dx = ax + sp * abx + st * bcx, dy = ay + sp * aby + st * bcy,
                  dz = az + sp * abz + st * bcz;
      const float r2 = dx * dx + dy * dy + dz * dz;
      const float rs = rsqrtf(r2);
      add(s_w[8 * p + q] * sp * scale * rs, r2 * rs, (dx * nx + dy * ny + dz * nz) * rs * rs);
    }
  }
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const float dx = (float)(g.qp[q * n + l] - x[0]), dy = (float)(g.qp[(7 + q) * n + l] - x[1]),
                dz = (float)(g.qp[(14 + q) * n + l] - x[2]);
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float rs = rsqrtf(r2);
    add(-(float)g.qw[q * n + l] * rs, r2 * rs, (dx * nx + dy * ny + dz * nz) * rs * rs);
  }
#pragma unroll
  for (int u = 0; u < kNearNodes; ++u)
    if (u < cnt) Cv[(int64_t)(j0 + u) * nnz + e] = acc[u];
}

// Slice `slice` of the mixed path's partials := C(z_j) V in FP32 (every row < n_pad and
// every column < nu written) from stored pair values Cv (node-major, nnz per node; the 8 x 8
// rule's or the surrogate network's): one warp per (row i, node j); lanes load 32 pairs'
// values and columns, then sweep the basis columns.
__global__ void __launch_bounds__(256)
near_spmm32_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ cols, int64_t n,
                   int64_t nnz, int N, const float2* __restrict__ Cv, const float2* __restrict__ Vt,
                   int nu, int nup, int C, int n_pad, float* __restrict__ Yp, int slice) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (w >= (int64_t)n_pad * N) return;
  const int64_t i = w % n_pad;
  const int node = (int)(w / n_pad);
  float2 acc[kMaxColGroups];
#pragma unroll
  for (int t = 0; t < kMaxColGroups; ++t) acc[t] = make_float2(0.f, 0.f);
  if (i < n) {
    const int32_t e0 = ptr[i], e1 = ptr[i + 1];
    const float2* Cj = Cv + (int64_t)node * nnz;
    for (int32_t eb = e0; eb < e1; eb += 32) {
      const int32_t e = eb + lane;
      float2 cval = make_float2(0.f, 0.f);
      int32_t l = 0;
      if (e < e1) {
        l = cols[e];
        cval = Cj[e];
      }
      const int cnt = min(32, e1 - eb);
      for (int t = 0; t < cnt; ++t) {
        const float cx = __shfl_sync(0xffffffffu, cval.x, t);
        const float cy = __shfl_sync(0xffffffffu, cval.y, t);
        const int32_t lt = __shfl_sync(0xffffffffu, l, t);
        const float2* vr = Vt + (int64_t)lt * nu;
#pragma unroll
        for (int cg = 0; cg < kMaxColGroups; ++cg) {
          const int c = lane + 32 * cg;
          if (c < nu) {
            const float2 v = vr[c];
            acc[cg].x = fmaf(cx, v.x, fmaf(-cy, v.y, acc[cg].x));
            acc[cg].y = fmaf(cx, v.y, fmaf(cy, v.x, acc[cg].y));
          }
        }
      }
    }
  }
  const int acc_cols = 2 * nup;
  float* base = Yp + ((size_t)slice * N + node) * acc_cols * (size_t)n_pad;
#pragma unroll
  for (int cg = 0; cg < kMaxColGroups; ++cg) {
    const int c = lane + 32 * cg;
    if (c < nu) {
      const int colr = (c / C) * 2 * C + (c % C);
      base[(size_t)colr * n_pad + i] = acc[cg].x;
      base[(size_t)(colr + C) * n_pad + i] = acc[cg].y;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Surrogate inference on the tensor core: the network's per-(pair, node) values C_j(e) into
// the same node-major array as the 8 x 8 rule's values, then the same sparse product.
// A CTA takes tiles of 128 samples t = j nnz + e (sample = TMEM lane = thread). The three
// 64-wide layers are tcgen05 kind::f16 MMAs (M = 128, N = 64, K = 16 per instruction): the
// weights, rounded to BF16 for inference, sit in shared memory as the B operands; each
// layer's input activations are split into BF16 hi + lo planes (two MMAs per K step, FP32
// accumulation in 64 TMEM columns), so the products carry ~16 bits of each activation
// against the BF16 weights, as the per-thread FP32 evaluation does to the rounding of its
// sums. Biases, tanh (the MUFU's tanh.approx) and the 64 -> 2 output layer run per thread
// on the accumulator rows read back with tcgen05.ld. Samples whose features leave the
// training box take the plain 8 x 8 rule (near_corr32 without a network).
constexpr int kSurTile = 128;
constexpr int kSurK1 = 16;   // the 11 inputs padded to one MMA K step

// shared memory: A1 (hi/lo planes of 128 x 16), A (hi/lo planes of 128 x 64), W1 (64 x 16),
// W2 and W3 (64 x 64), all BF16 K-major; then the FP32 constants (input shift, scale and
// box, biases, output layer, output scale); then the mbarrier, TMEM slot and abort flag
constexpr uint32_t kSurA1 = 0;
constexpr uint32_t kSurA = kSurA1 + 2u * kSurTile * kSurK1 * 2u;
constexpr uint32_t kSurW1 = kSurA + 2u * kSurTile * kNetHid * 2u;
constexpr uint32_t kSurW2 = kSurW1 + (uint32_t)kNetHid * kSurK1 * 2u;
constexpr uint32_t kSurW3 = kSurW2 + (uint32_t)kNetHid * kNetHid * 2u;
constexpr uint32_t kSurCst = kSurW3 + (uint32_t)kNetHid * kNetHid * 2u;
constexpr int kCShift = 0, kCScale = 11, kCLo = 22, kCHi = 33, kCB1 = 44, kCB2 = 108,
              kCB3 = 172, kCW4 = 236, kCB4 = 364, kCOut = 366, kCFloats = 368;
constexpr uint32_t kSurBar = kSurCst + kCFloats * 4u;
constexpr uint32_t kSurSmem = kSurBar + 16u;

// Byte offset of element (row r, k) in a K-major canonical (no swizzle) BF16 operand with
// K columns: 8-row x 16-byte core matrices, 128 bytes apart along K, 8-row groups
// (K / 8) x 128 bytes apart.
__device__ __forceinline__ uint32_t kmaj_off(int r, int k, int K) {
  return (uint32_t)(r / 8) * (uint32_t)(K / 8) * 128u + (uint32_t)(k / 8) * 128u +
         (uint32_t)(r % 8) * 16u + (uint32_t)(k % 8) * 2u;
}

__device__ __forceinline__ float tanh_mufu(float x) {
  float r;
  asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Per pair: the nine frame features (the triangle's vertices in the pair's frame over h),
// h, and the output factor h / (d / h)^7 (SoA, 11 x nnz floats).
__global__ void __launch_bounds__(256)
surrogate_pair_features_kernel(Geometry g, const int32_t* __restrict__ rows,
                               const int32_t* __restrict__ cols, int64_t nnz,
                               float* __restrict__ pf) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  const int64_t n = g.n;
  const int64_t i = rows[e], l = cols[e];
  const double x[3] = {g.cx[i], g.cx[n + i], g.cx[2 * n + i]};
  NearFrame F;
  near_frame(g, l, x, F);
  float feat[kNetIn];
  near_features32(g, l, F, x, 0.f, 0.f, feat);
  for (int c = 0; c < 9; ++c) pf[c * nnz + e] = feat[c];
  const float h = (float)g.diam[l];
  pf[9 * nnz + e] = h;
  pf[10 * nnz + e] = h / surrogate_decay(feat);
}

__device__ __forceinline__ uint32_t pack_bf16_pair(float lo_elem, float hi_elem) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo_elem, hi_elem);   // .x -> low 16 bits
  return *reinterpret_cast<uint32_t*>(&h);
}

// One row of a layer's input (K values) as BF16 hi and lo planes of a K-major operand.
template <int K>
__device__ __forceinline__ void put_act_row(unsigned char* hi_plane, unsigned char* lo_plane, int r,
                                            const float* v) {
#pragma unroll
  for (int c = 0; c < K / 8; ++c) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float a = v[8 * c + 2 * q], b = v[8 * c + 2 * q + 1];
      h[q] = pack_bf16_pair(a, b);
      l[q] = pack_bf16_pair(a - __uint_as_float(h[q] << 16), b - __uint_as_float(h[q] & 0xFFFF0000u));
    }
    const uint32_t off = kmaj_off(r, 8 * c, K);
    *reinterpret_cast<uint4*>(hi_plane + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(lo_plane + off) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

__global__ void __launch_bounds__(kSurTile)
surrogate_values_tc_kernel(Geometry g, const int32_t* __restrict__ rows,
                           const int32_t* __restrict__ cols, int64_t nnz,
                           const double* __restrict__ z, int N, const float* __restrict__ pf,
                           const float* __restrict__ net, GL8 gl, OpCoef op,
                           float2* __restrict__ Cv, int* status, uint32_t wait_limit,
                           unsigned long long* __restrict__ usage) {
  extern __shared__ __align__(1024) unsigned char smem[];
  float* cst = reinterpret_cast<float*>(smem + kSurCst);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kSurBar);
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + kSurBar + 8);
  const int tid = threadIdx.x, warp = tid / 32;

  // the BF16 weights as K-major B operands (rows = output units), the FP32 constants
  for (int x = tid; x < kNetHid * kSurK1; x += kSurTile) {
    const int o = x / kSurK1, k = x % kSurK1;
    const float w = k < kNetIn ? net[kOffW1 + o * kNetIn + k] : 0.f;
    *reinterpret_cast<__nv_bfloat16*>(smem + kSurW1 + kmaj_off(o, k, kSurK1)) = __float2bfloat16_rn(w);
  }
  for (int x = tid; x < kNetHid * kNetHid; x += kSurTile) {
    const int o = x / kNetHid, k = x % kNetHid;
    *reinterpret_cast<__nv_bfloat16*>(smem + kSurW2 + kmaj_off(o, k, kNetHid)) =
        __float2bfloat16_rn(net[kOffW2 + x]);
    *reinterpret_cast<__nv_bfloat16*>(smem + kSurW3 + kmaj_off(o, k, kNetHid)) =
        __float2bfloat16_rn(net[kOffW3 + x]);
  }
  for (int x = tid; x < kNetIn; x += kSurTile) {
    cst[kCShift + x] = net[kOffInShift + x];
    cst[kCScale + x] = net[kOffInScale + x];
    const float lo = net[kOffFeatLo + x], hi = net[kOffFeatHi + x], m = 0.02f * (hi - lo);
    cst[kCLo + x] = lo - m;   // the training box widened by 2 % of its width
    cst[kCHi + x] = hi + m;
  }
  for (int x = tid; x < kNetHid; x += kSurTile) {
    cst[kCB1 + x] = net[kOffB1 + x];
    cst[kCB2 + x] = net[kOffB2 + x];
    cst[kCB3 + x] = net[kOffB3 + x];
  }
  for (int x = tid; x < kNetOut * kNetHid; x += kSurTile) cst[kCW4 + x] = net[kOffW4 + x];
  if (tid < kNetOut) {
    cst[kCB4 + tid] = net[kOffB4 + tid];
    cst[kCOut + tid] = net[kOffOutScale + tid];
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(slot, kNetHid);
    tmem_relinquish();
  }
  fence_proxy_async_smem();   // the weight planes -> the tensor core
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const uint32_t lanes = tmem + ((uint32_t)(warp * 32) << 16);   // this warp's TMEM lanes
  const uint32_t idesc = idesc_bf16(kSurTile, kNetHid);
  const uint32_t a1 = smem_u32(smem + kSurA1), a = smem_u32(smem + kSurA);
  const uint32_t a1_lo = kSurTile * kSurK1 * 2u, a_lo = kSurTile * kNetHid * 2u;
  const int64_t total = nnz * N;
  const int64_t tiles = (total + kSurTile - 1) / kSurTile;
  uint32_t phase = 0;
  bool ok = true;
  // one layer's MMAs (thread 0) and the wait for them (every thread, bounded; the block
  // agrees on the outcome)
  auto layer = [&](uint32_t a_base, uint32_t a_lo_off, uint32_t w, int K) {
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t sbo = (uint32_t)(K / 8) * 128u;
      for (int kk = 0; kk < K / 16; ++kk) {
        const uint64_t bd = smem_desc(w + kk * 256u, 128, sbo);
        mma_bf16(tmem, smem_desc(a_base + kk * 256u, 128, sbo), bd, idesc, kk > 0 ? 1u : 0u);
        mma_bf16(tmem, smem_desc(a_base + a_lo_off + kk * 256u, 128, sbo), bd, idesc, 1u);
      }
      mma_commit(bar);
    }
    const bool done = mbar_wait(bar, phase, wait_limit);
    phase ^= 1u;
    ok = __syncthreads_and(done) != 0;
    tc_fence_after();
  };
  auto read_act = [&](int boff, float* v) {   // tanh(accumulator row + bias)
#pragma unroll
    for (int c0 = 0; c0 < kNetHid; c0 += 16) {
      float r[16];
      tmem_ld16(lanes + c0, r);
#pragma unroll
      for (int k = 0; k < 16; ++k) v[c0 + k] = tanh_mufu(r[k] + cst[boff + c0 + k]);
    }
  };

  for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
    const int64_t t = tile * kSurTile + tid;
    const bool valid = t < total;
    const int64_t e = valid ? t % nnz : 0;
    const int j = valid ? (int)(t / nnz) : 0;
    const float kr = (float)z[2 * j], ki = (float)z[2 * j + 1];
    const float h = pf[9 * nnz + e], fac = pf[10 * nnz + e];
    float x[kSurK1];
    bool inbox = true;
#pragma unroll
    for (int c = 0; c < kNetIn; ++c) {
      const float f = c < 9 ? pf[c * nnz + e] : (c == 9 ? kr * h : ki * h);
      inbox = inbox && f >= cst[kCLo + c] && f <= cst[kCHi + c];
      x[c] = valid ? (f - cst[kCShift + c]) * cst[kCScale + c] : 0.f;
    }
#pragma unroll
    for (int c = kNetIn; c < kSurK1; ++c) x[c] = 0.f;
    put_act_row<kSurK1>(smem + kSurA1, smem + kSurA1 + a1_lo, tid, x);
    layer(a1, a1_lo, smem_u32(smem + kSurW1), kSurK1);
    if (!ok) break;
    float v[kNetHid];
    read_act(kCB1, v);
    put_act_row<kNetHid>(smem + kSurA, smem + kSurA + a_lo, tid, v);
    layer(a, a_lo, smem_u32(smem + kSurW2), kNetHid);
    if (!ok) break;
    read_act(kCB2, v);
    put_act_row<kNetHid>(smem + kSurA, smem + kSurA + a_lo, tid, v);
    layer(a, a_lo, smem_u32(smem + kSurW3), kNetHid);
    if (!ok) break;
    read_act(kCB3, v);
    float o0 = cst[kCB4], o1 = cst[kCB4 + 1];
#pragma unroll
    for (int k = 0; k < kNetHid; ++k) {
      o0 = fmaf(cst[kCW4 + k], v[k], o0);
      o1 = fmaf(cst[kCW4 + kNetHid + k], v[k], o1);
    }
    float2 val = make_float2(o0 * cst[kCOut] * fac, o1 * cst[kCOut + 1] * fac);
    // samples served by the network and by the plain rule (one atomic per warp)
    const unsigned in_net = __ballot_sync(0xffffffffu, valid && inbox);
    const unsigned in_rule = __ballot_sync(0xffffffffu, valid && !inbox);
    if (tid % 32 == 0) {
      if (in_net) atomicAdd(&usage[0], (unsigned long long)__popc(in_net));
      if (in_rule) atomicAdd(&usage[1], (unsigned long long)__popc(in_rule));
    }
    if (valid && !inbox) {   // outside the training box: the plain 8 x 8 rule
      const int64_t n = g.n, i = rows[e], l = cols[e];
      const double xc[3] = {g.cx[i], g.cx[n + i], g.cx[2 * n + i]};
      val = near_corr32(g, l, xc, kr, ki, gl, op);
    }
    if (valid) Cv[t] = val;
  }
  if (!ok && tid == 0) atomicOr(status, kStatusTimeout);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    // the last commit has completed on the normal path; bounded on an aborted one
    if (tid == 0 && !ok) mbar_wait(bar, phase ^ 1u, kStageWaitDefault);
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, kNetHid);
  }
}

// R[:, c] += C(lam_c) X[:, c] (deriv: k-derivatives); one warp per (row i, column c).
template <bool kDeriv>
__global__ void __launch_bounds__(256)
near_percol64_kernel(Geometry g, const int32_t* __restrict__ ptr, const int32_t* __restrict__ cols,
                     const double* __restrict__ lam, int m, const double2* __restrict__ X,
                     int64_t ldx, double2* __restrict__ R, GL8 gl, OpCoef op) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  const int64_t n = g.n;
  if (w >= n * (int64_t)m) return;
  const int64_t i = w % n;
  const int c = (int)(w / n);
  const double kr = lam[2 * c], ki = lam[2 * c + 1];
  const double x[3] = {g.cx[i], g.cx[n + i], g.cx[2 * n + i]};
  double2 acc = make_double2(0.0, 0.0);
  const int32_t e0 = ptr[i], e1 = ptr[i + 1];
  for (int32_t e = e0 + lane; e < e1; e += 32) {
    const int32_t l = cols[e];
    const double2 cv = near_corr64(g, l, x, kr, ki, kDeriv, gl, op);
    const double2 v = X[(int64_t)c * ldx + l];
    acc.x += cv.x * v.x - cv.y * v.y;
    acc.y += cv.x * v.y + cv.y * v.x;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
  }
  if (lane == 0 && e1 > e0) {
    double2 r = R[(int64_t)c * n + i];
    r.x += acc.x;
    r.y += acc.y;
    R[(int64_t)c * n + i] = r;
  }
}

// Row-major copies of the basis for the near products.
__global__ void transpose64_kernel(const double2* __restrict__ V, int64_t ldv, int64_t n, int nu,
                                   double2* __restrict__ Vt) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * nu) return;
  const int64_t l = t / nu;
  const int c = (int)(t % nu);
  Vt[t] = V[(int64_t)c * ldv + l];
}

__global__ void transpose32_kernel(const float2* __restrict__ V32, int64_t n, int nu,
                                   float2* __restrict__ Vt) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * nu) return;
  const int64_t l = t / nu;
  const int c = (int)(t % nu);
  Vt[t] = V32[(int64_t)c * n + l];
}

__device__ __forceinline__ double u01(uint64_t seed, uint64_t idx) {
  uint64_t z = seed + (idx + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1.0p-53;
}

// Training samples of the surrogate network: sample t takes the near pair
// e = floor(u * nnz) of the current mesh and k uniform in the box, u from SplitMix64 of
// (seed, 3t, 3t+1, 3t+2); features as near_features32, target (A_near - A_7)(k) / h from
// the FP64 8 x 8 rule (the plain quadrature is the network's reference). Optionally the pair
// (row, column) and k of each sample.
__global__ void surrogate_samples_kernel(Geometry g, const int32_t* __restrict__ ptr,
                                         const int32_t* __restrict__ cols, int64_t nnz,
                                         int64_t count, uint64_t seed, double kr_lo, double kr_hi,
                                         double ki_lo, double ki_hi, float* __restrict__ feat,
                                         float* __restrict__ target, int32_t* __restrict__ pairs,
                                         double* __restrict__ ks, GL8 gl) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  int64_t e = (int64_t)(u01(seed, 3 * t) * (double)nnz);
  if (e > nnz - 1) e = nnz - 1;
  const double kr = kr_lo + (kr_hi - kr_lo) * u01(seed, 3 * t + 1);
  const double ki = ki_lo + (ki_hi - ki_lo) * u01(seed, 3 * t + 2);
  int64_t lo = 0, hi = g.n - 1;   // row: the last i with ptr[i] <= e
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (ptr[mid] <= e) lo = mid; else hi = mid - 1;
  }
  const int64_t i = lo, l = cols[e], n = g.n;
  const double x[3] = {g.cx[i], g.cx[n + i], g.cx[2 * n + i]};
  NearFrame F;
  near_frame(g, l, x, F);
  float f[kNetIn];
  near_features32(g, l, F, x, (float)kr, (float)ki, f);
  // the features take k h from the float k; the target uses the same rounded k
  const double2 c = near_corr64(g, l, x, (double)(float)kr, (double)(float)ki, false, gl, OpCoef());
  const double h = g.diam[l];
  for (int q = 0; q < kNetIn; ++q) feat[t * kNetIn + q] = f[q];
  target[2 * t] = (float)(c.x / h);
  target[2 * t + 1] = (float)(c.y / h);
  if (pairs) {
    pairs[2 * t] = (int32_t)i;
    pairs[2 * t + 1] = (int32_t)l;
  }
  if (ks) {
    ks[2 * t] = (double)(float)kr;
    ks[2 * t + 1] = (double)(float)ki;
  }
}

const GL8& gl8() {
  static const GL8 g = make_gl8();
  return g;
}

bem_status ensure_near_work(bem_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->near_work_bytes) return BEM_OK;
  cudaFree(ctx->d_near_work);
  ctx->d_near_work = nullptr;
  ctx->near_work_bytes = 0;
  if (cudaMalloc(&ctx->d_near_work, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, BEM_ENOMEM, "near field: device allocation failed");
  }
  ctx->near_work_bytes = bytes;
  return BEM_OK;
}

}  // namespace

bem_status ensure_near(bem_ctx* ctx, cudaStream_t s) {
  if (ctx->near_mode == 0 || ctx->near_mesh_version == ctx->mesh_version) return BEM_OK;
  const int64_t n = ctx->geo.n;
  if (n == 0) return fail(ctx, BEM_ESTATE, "near field: no mesh set");
  if (n + 1 > ctx->near_cap_n) {
    cudaFree(ctx->d_near_ptr);
    ctx->d_near_ptr = nullptr;
    ctx->near_cap_n = 0;
    if (cudaMalloc(&ctx->d_near_ptr, (n + 1) * sizeof(int32_t)) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, BEM_ENOMEM, "near field: device allocation failed");
    }
    ctx->near_cap_n = n + 1;
  }
  const unsigned blocks = (unsigned)((n + kScanTile - 1) / kScanTile);
  near_scan_kernel<<<blocks, kScanTile, 0, s>>>(ctx->geo, ctx->d_near_ptr, nullptr, nullptr);
  ctx->launches++;
  std::vector<int32_t> h(n + 1);
  bem_status st = cuda_check(ctx, cudaMemcpyAsync(h.data(), ctx->d_near_ptr, n * sizeof(int32_t),
                                                  cudaMemcpyDeviceToHost, s),
                             "near field copy");
  if (st == BEM_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), "near field copy");
  if (st != BEM_OK) return st;
  int64_t total = 0;
  for (int64_t i = 0; i < n; ++i) {   // counts -> row pointers
    const int64_t c = h[i];
    h[i] = (int32_t)total;
    total += c;
  }
  if (total > 0x7fffffff) return fail(ctx, BEM_EINVAL, "near field: too many near pairs");
  h[n] = (int32_t)total;
  if (total > ctx->near_cap_nnz) {
    cudaFree(ctx->d_near_cols);
    ctx->d_near_cols = nullptr;
    ctx->near_cap_nnz = 0;
    if (cudaMalloc(&ctx->d_near_cols, std::max<int64_t>(1, total) * sizeof(int32_t)) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, BEM_ENOMEM, "near field: device allocation failed");
    }
    ctx->near_cap_nnz = std::max<int64_t>(1, total);
  }
  st = cuda_check(ctx, cudaMemcpyAsync(ctx->d_near_ptr, h.data(), (n + 1) * sizeof(int32_t),
                                       cudaMemcpyHostToDevice, s),
                  "near field copy");
  if (st != BEM_OK) return st;
  near_scan_kernel<<<blocks, kScanTile, 0, s>>>(ctx->geo, nullptr, ctx->d_near_ptr,
                                                ctx->d_near_cols);
  ctx->launches++;
  st = cuda_check(ctx, cudaGetLastError(), "near field kernels");
  if (st == BEM_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), "near field build");
  if (st != BEM_OK) return st;
  ctx->near_nnz = total;
  ctx->near_mesh_version = ctx->mesh_version;
  return BEM_OK;
}

bem_status near_apply64(bem_ctx* ctx, const double* V, int64_t ldv, int nu, double* Y,
                        cudaStream_t s) {
  const int64_t n = ctx->geo.n;
  bem_status st = ensure_near_work(ctx, (size_t)n * nu * sizeof(double2));
  if (st != BEM_OK) return st;
  double2* Vt = reinterpret_cast<double2*>(ctx->d_near_work);
  transpose64_kernel<<<(unsigned)((n * nu + 255) / 256), 256, 0, s>>>(
      reinterpret_cast<const double2*>(V), ldv, n, nu, Vt);
  const int N = ctx->con.N;
  near_apply64_kernel<<<(unsigned)((32 * n * (int64_t)N + 255) / 256), 256, 0, s>>>(
      ctx->geo, ctx->d_near_ptr, ctx->d_near_cols, ctx->con.z, N, Vt, nu,
      reinterpret_cast<double2*>(Y), gl8(), ctx->op);
  ctx->launches += 2;
  return cuda_check(ctx, cudaGetLastError(), "near field kernels");
}

bem_status near_apply32(bem_ctx* ctx, const float2* V32, int nu, int nup, int C, int n_pad,
                        float* Yp, int slice, cudaStream_t s) {
  const int64_t n = ctx->geo.n;
  const int N = ctx->con.N;
  const int64_t nnz = ctx->near_nnz;
  // the inference copy of the network (BF16-rounded weights) follows the master weights
  const float* net = (ctx->near_mode == 2 && ctx->net_ready) ? ctx->d_net + kNetFloats : nullptr;
  // the pair values of every node first, by the 64-point rule or the network (work buffer:
  // the row-major basis, N x nnz values, the pairs' rows, the network's pair features)
  const bool values = nnz > 0;
  const size_t vt_bytes = (size_t)n * nu * sizeof(float2);
  const size_t cv_bytes = values ? (size_t)N * nnz * sizeof(float2) : 0;
  const size_t rows_bytes = values ? ((size_t)nnz * sizeof(int32_t) + 15) / 16 * 16 : 0;
  const size_t pf_bytes = (values && net) ? (size_t)11 * nnz * sizeof(float) : 0;
  bem_status st = ensure_near_work(ctx, vt_bytes + cv_bytes + rows_bytes + pf_bytes);
  if (st != BEM_OK) return st;
  float2* Vt = reinterpret_cast<float2*>(ctx->d_near_work);
  transpose32_kernel<<<(unsigned)((n * nu + 255) / 256), 256, 0, s>>>(V32, n, nu, Vt);
  ctx->launches++;
  float2* Cv = nullptr;
  if (values) {
    char* wk = static_cast<char*>(ctx->d_near_work);
    Cv = reinterpret_cast<float2*>(wk + vt_bytes);
    int32_t* rows = reinterpret_cast<int32_t*>(wk + vt_bytes + cv_bytes);
    near_rows_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ctx->d_near_ptr, n, rows);
    ctx->launches++;
    if (net) {
      float* pf = reinterpret_cast<float*>(wk + vt_bytes + cv_bytes + rows_bytes);
      surrogate_pair_features_kernel<<<(unsigned)((nnz + 255) / 256), 256, 0, s>>>(
          ctx->geo, rows, ctx->d_near_cols, nnz, pf);
      st = cuda_check(ctx, cudaFuncSetAttribute(surrogate_values_tc_kernel,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)kSurSmem),
                      "surrogate kernel attribute");
      if (st != BEM_OK) return st;
      int sms = 0;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
      const int64_t tiles = (nnz * N + kSurTile - 1) / kSurTile;
      const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, 3 * (int64_t)std::max(1, sms)));
      if (!ctx->d_sur_usage) {
        st = cuda_check(ctx, cudaMalloc(&ctx->d_sur_usage, 2 * sizeof(unsigned long long)),
                        "surrogate usage counters");
        if (st != BEM_OK) return st;
        st = cuda_check(ctx, cudaMemsetAsync(ctx->d_sur_usage, 0, 2 * sizeof(unsigned long long), s),
                        "surrogate usage counters");
        if (st != BEM_OK) return st;
      }
      surrogate_values_tc_kernel<<<grid, kSurTile, kSurSmem, s>>>(
          ctx->geo, rows, ctx->d_near_cols, nnz, ctx->con.z, N, pf, net, gl8(), ctx->op, Cv,
          ctx->d_status, ctx->stage_wait_limit, ctx->d_sur_usage);
      ctx->launches += 2;
    } else {
      const int64_t threads = nnz * ((N + kNearNodes - 1) / kNearNodes);
      if (op_single(ctx->op))
        near_values32_kernel<false><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
            ctx->geo, rows, ctx->d_near_cols, nnz, ctx->con.z, N, gl8(), ctx->op, Cv);
      else
        near_values32_kernel<true><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
            ctx->geo, rows, ctx->d_near_cols, nnz, ctx->con.z, N, gl8(), ctx->op, Cv);
      ctx->launches++;
    }
  }
  const unsigned blocks = (unsigned)((32 * (int64_t)n_pad * N + 255) / 256);
  near_spmm32_kernel<<<blocks, 256, 0, s>>>(ctx->d_near_ptr, ctx->d_near_cols, n, nnz, N, Cv, Vt,
                                            nu, nup, C, n_pad, Yp, slice);
  ctx->launches++;
  return cuda_check(ctx, cudaGetLastError(), "near field kernels");
}

cudaError_t launch_near_percol64(bem_ctx* ctx, int m, const double* lam_dev, const double* X,
                                 int64_t ldx, double* R, bool deriv, cudaStream_t s) {
  const int64_t n = ctx->geo.n;
  const unsigned blocks = (unsigned)((32 * n * (int64_t)m + 255) / 256);
  if (deriv)
    near_percol64_kernel<true><<<blocks, 256, 0, s>>>(
        ctx->geo, ctx->d_near_ptr, ctx->d_near_cols, lam_dev, m,
        reinterpret_cast<const double2*>(X), ldx, reinterpret_cast<double2*>(R), gl8(), ctx->op);
  else
    near_percol64_kernel<false><<<blocks, 256, 0, s>>>(
        ctx->geo, ctx->d_near_ptr, ctx->d_near_cols, lam_dev, m,
        reinterpret_cast<const double2*>(X), ldx, reinterpret_cast<double2*>(R), gl8(), ctx->op);
  ctx->launches++;
  return cudaGetLastError();
}

}  // namespace bem

using namespace bem;

extern "C" bem_status bem_set_near_field(bem_ctx* ctx, int mode, void* stream) {
  if (!ctx) return BEM_EINVAL;
  if (mode < 0 || mode > 2) return fail(ctx, BEM_EINVAL, "bem_set_near_field: mode must be 0, 1 or 2");
  if (mode == 2 && !op_single(ctx->op) && (ctx->op.chr != 0.0 || ctx->op.chi != 0.0))
    return fail(ctx, BEM_EINVAL,
                "bem_set_near_field: the surrogate (mode 2) covers the single layer only");
  if (mode == 2 && !ctx->net_ready)
    return fail(ctx, BEM_ESTATE, "bem_set_near_field: no surrogate network loaded");
  cudaSetDevice(ctx->device);
  ctx->near_mode = mode;
  ctx->near_mesh_version = -1;
  if (mode == 0 || ctx->geo.n == 0) return BEM_OK;
  return ensure_near(ctx, (cudaStream_t)stream);
}

extern "C" bem_status bem_surrogate_usage(bem_ctx* ctx, int64_t* network, int64_t* rule,
                                          void* stream) {
  if (!ctx || !network || !rule) return BEM_EINVAL;
  *network = 0;
  *rule = 0;
  if (!ctx->d_sur_usage) return BEM_OK;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long h[2] = {0, 0};
  bem_status st = cuda_check(ctx, cudaMemcpyAsync(h, ctx->d_sur_usage, sizeof(h),
                                                  cudaMemcpyDeviceToHost, s),
                             "bem_surrogate_usage copy");
  if (st == BEM_OK)
    st = cuda_check(ctx, cudaMemsetAsync(ctx->d_sur_usage, 0, sizeof(h), s), "bem_surrogate_usage reset");
  if (st == BEM_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), "bem_surrogate_usage");
  *network = (int64_t)h[0];
  *rule = (int64_t)h[1];
  return st;
}

extern "C" bem_status bem_near_pairs(bem_ctx* ctx, int64_t* nnz, int32_t* row_ptr_host,
                                     int32_t* cols_host, void* stream) {
  if (!ctx || !nnz) return BEM_EINVAL;
  if (ctx->near_mode == 0) return fail(ctx, BEM_ESTATE, "bem_near_pairs: near field is off");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  bem_status st = ensure_near(ctx, s);
  if (st != BEM_OK) return st;
  *nnz = ctx->near_nnz;
  if (row_ptr_host)
    st = cuda_check(ctx, cudaMemcpyAsync(row_ptr_host, ctx->d_near_ptr,
                                         (ctx->geo.n + 1) * sizeof(int32_t),
                                         cudaMemcpyDeviceToHost, s), "bem_near_pairs copy");
  if (st == BEM_OK && cols_host && ctx->near_nnz > 0)
    st = cuda_check(ctx, cudaMemcpyAsync(cols_host, ctx->d_near_cols,
                                         ctx->near_nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s),
                    "bem_near_pairs copy");
  if (st == BEM_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), "bem_near_pairs copy");
  return st;
}

extern "C" bem_status bem_surrogate_samples(bem_ctx* ctx, double kr_lo, double kr_hi, double ki_lo,
                                            double ki_hi, int64_t count, uint64_t seed,
                                            float* feat_dev, float* target_dev, int32_t* pairs_dev,
                                            double* k_dev, void* stream) {
  if (!ctx) return BEM_EINVAL;
  if (count < 1 || !feat_dev || !target_dev || !(kr_hi >= kr_lo) || !(ki_hi >= ki_lo))
    return fail(ctx, BEM_EINVAL, "bem_surrogate_samples: bad arguments");
  if (ctx->near_mode == 0) return fail(ctx, BEM_ESTATE, "bem_surrogate_samples: near field is off");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  bem_status st = ensure_near(ctx, s);
  if (st != BEM_OK) return st;
  if (ctx->near_nnz == 0) return fail(ctx, BEM_ESTATE, "bem_surrogate_samples: mesh has no near pairs");
  surrogate_samples_kernel<<<(unsigned)((count + 127) / 128), 128, 0, s>>>(
      ctx->geo, ctx->d_near_ptr, ctx->d_near_cols, ctx->near_nnz, count, seed, kr_lo, kr_hi, ki_lo,
      ki_hi, feat_dev, target_dev, pairs_dev, k_dev, gl8());
  ctx->launches++;
  return cuda_check(ctx, cudaGetLastError(), "bem_surrogate_samples");
}
