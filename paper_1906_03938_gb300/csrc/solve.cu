// The steps around the projection: basis improvement by inverse power steps (Algorithm 1)
// and refinement of Ritz pairs against the true operator (residual inverse iteration).
//
// Inverse power (Algorithm 1; Eq. wjp1, Eq. vjp1, Eq. viupd, Eq. linsyssim), shift s:
//   S u' = sum_j B_j v_j / (z_j - s),  S = sum_j B_j / (z_j - s),  B_j = w_j A(z_j),
//   v_j' = (v_j - u') / (z_j - s),
// for every basis column at once, q times, from v_j = u / (z_j - s). S is assembled densely
// (FP32) and factorised once (blocked LU); the right-hand side is applied matrix-free by
// the node-summed fused kernel (FP32 evaluation, BF16x3 tcgen05 contraction). The iterates
// are rescaled column by column (direction only).
//
// Refinement: for an approximate eigenpair (lambda, x) of A(k) x = 0, residual inverse
// iteration with a frozen factorisation of A(sigma) (Neumaier 1985) and a Newton step for
// lambda on f(lambda) = e^H A(sigma)^{-1} A(lambda) x:
//   r = A(lambda) x, r' = A'(lambda) x           (double-FP32, matrix-free, one pass)
//   [s1 s2] = A(sigma)^{-1} [r r']                (FP32 LU)
//   dlambda = -(e^H s1) / (e^H s2), x <- x - (s1 + dlambda s2), x <- x / (e^H x)
// The fixed point is an eigenpair to the residuals' accuracy (entries to ~1e-13) whatever
// the LU's precision; sigma is moved to the current lambda when the iteration stalls. The
// residuals reported at the end are recomputed in FP64.
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"
#include "small_eig.h"

namespace bem {
namespace {

// refinement: factorisations of A(sigma) per eigenpair at most (the last one is kept), and
// the relative residual at which an eigenpair is converged (the double-FP32 entries'
// rounding, ~1e-13, times the growth of the row sums at n ~ 1e5; three orders below the
// 1e-8 the eigenpairs are certified to)
constexpr int kMaxFactorisations = 4;
constexpr double kResidualStop = 1e-11;
// relative lambda steps below this are the double-FP32 residuals' noise: converged
constexpr double kStepFloor = 1e-12;

// Vn_j = u / (z_j - s) (u FP64 n x nu, ld ldu)
__global__ void ip_start_kernel(const double2* __restrict__ U, int64_t ldu, int64_t n, int nu,
                                int N, const double2* __restrict__ z, double2 s, float2* Vn) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per = n * nu;
  if (t >= per * N) return;
  const int j = (int)(t / per);
  const int64_t e = t % per;
  const int c = (int)(e / n);
  const int64_t i = e % n;
  const double2 u = U[(int64_t)c * ldu + i];
  const double2 d = make_double2(z[j].x - s.x, z[j].y - s.y);
  const double dd = d.x * d.x + d.y * d.y;
  Vn[t] = make_float2((float)((u.x * d.x + u.y * d.y) / dd), (float)((u.y * d.x - u.x * d.y) / dd));
}

// Vn_j = (Vn_j - u') / (z_j - s); then column scaling by inv[c] (both FP32)
__global__ void ip_update_kernel(float2* Vn, const float2* __restrict__ Up, int64_t n, int nu,
                                 int N, const double2* __restrict__ z, double2 s) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per = n * nu;
  if (t >= per * N) return;
  const int j = (int)(t / per);
  const int64_t e = t % per;
  const float2 v = Vn[t], u = Up[e];
  const double2 d = make_double2(z[j].x - s.x, z[j].y - s.y);
  const double dd = d.x * d.x + d.y * d.y;
  const double ar = v.x - u.x, ai = v.y - u.y;
  Vn[t] = make_float2((float)((ar * d.x + ai * d.y) / dd), (float)((ai * d.x - ar * d.y) / dd));
}

// column sums of squares of the node-major block (fixed order): one block per column
__global__ void ip_colnorm_kernel(const float2* __restrict__ Vn, int64_t n, int nu, int N,
                                  double* __restrict__ out) {
  __shared__ double red[256];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int j = 0; j < N; ++j) {
    const float2* v = Vn + ((int64_t)j * nu + c) * n;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += (double)v[i].x * v[i].x + (double)v[i].y * v[i].y;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = red[0];
}

__global__ void ip_scale_kernel(float2* Vn, float2* Up, int64_t n, int nu, int N,
                                const double* __restrict__ nrm2) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per = n * nu;
  if (t >= per * N) return;
  const int c = (int)((t % per) / n);
  const float f = (float)(1.0 / sqrt(fmax(nrm2[c], 1e-300)));
  Vn[t].x *= f;
  Vn[t].y *= f;
  if (t < per) {
    Up[t].x *= f;
    Up[t].y *= f;
  }
}

__global__ void f32_to_f64_kernel(const float2* __restrict__ a, int64_t n, int m, double2* b,
                                  int64_t ldb) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * m) return;
  const int c = (int)(t / n);
  const int64_t i = t % n;
  b[(int64_t)c * ldb + i] = make_double2(a[t].x, a[t].y);
}

// ---- refinement helpers (one eigenpair: vectors of length n) ----

// [r r'] (FP64, n x 2 contiguous) -> FP32
// node blocks of X (FP64, leading dimension ldx, node_stride elements apart) -> FP32,
// node-major with leading dimension n
__global__ void x_to_f32_kernel(const double2* __restrict__ X, int64_t ldx, int64_t node_stride,
                                int64_t n, int nu, int nnodes, float2* __restrict__ X32) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per = n * nu;
  if (t >= per * nnodes) return;
  const int64_t node = t / per, i = (t % per) % n, c = (t % per) / n;
  const double2 v = X[node * node_stride + c * ldx + i];
  X32[t] = make_float2((float)v.x, (float)v.y);
}

__global__ void to_f32_kernel(const double2* __restrict__ a, int64_t count, float2* b) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < count) b[t] = make_float2((float)a[t].x, (float)a[t].y);
}

// dots[c] = e^H s_c for the two solutions (FP64 sums in a fixed order)
__global__ void dot2_kernel(const double2* __restrict__ e, const float2* __restrict__ S, int64_t n,
                            double2* __restrict__ dots) {
  __shared__ double2 red[256];
  const int c = blockIdx.x;
  const float2* sc = S + (int64_t)c * n;
  double2 acc = make_double2(0.0, 0.0);
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 a = e[i];
    const double2 b = make_double2(sc[i].x, sc[i].y);
    acc.x += a.x * b.x + a.y * b.y;
    acc.y += a.x * b.y - a.y * b.x;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      red[threadIdx.x].x += red[threadIdx.x + w].x;
      red[threadIdx.x].y += red[threadIdx.x + w].y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) dots[c] = red[0];
}

// x <- x - (s1 + dl s2)
__global__ void refine_update_kernel(double2* x, const float2* __restrict__ S, int64_t n,
                                     double2 dl) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float2 s1 = S[i], s2 = S[n + i];
  x[i].x -= s1.x + (dl.x * s2.x - dl.y * s2.y);
  x[i].y -= s1.y + (dl.x * s2.y + dl.y * s2.x);
}

// x <- x / alpha
__global__ void scale_vec_kernel(double2* x, int64_t n, double2 alpha) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double d = alpha.x * alpha.x + alpha.y * alpha.y;
  const double2 v = x[i];
  x[i] = make_double2((v.x * alpha.x + v.y * alpha.y) / d, (v.y * alpha.x - v.x * alpha.y) / d);
}

// e^H x for one vector (one block)
__global__ void dot1_kernel(const double2* __restrict__ e, const double2* __restrict__ x, int64_t n,
                            double2* out) {
  __shared__ double2 red[256];
  double2 acc = make_double2(0.0, 0.0);
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    acc.x += e[i].x * x[i].x + e[i].y * x[i].y;
    acc.y += e[i].x * x[i].y - e[i].y * x[i].x;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      red[threadIdx.x].x += red[threadIdx.x + w].x;
      red[threadIdx.x].y += red[threadIdx.x + w].y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// ---- Algorithm 2 (inverse power for the Chebyshev interpolant, shift at the centre) ----

// W_i = T_i(0) V for the m blocks (T_i(0) = 1, 0, -1, 0, ...)
__global__ void cip_start_kernel(const double2* __restrict__ V, int64_t ldv, int64_t n, int nu,
                                 int m, float2* W) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per = n * nu;
  if (t >= per * m) return;
  const int i = (int)(t / per);
  const int64_t e = t % per;
  const double2 v = V[(e / n) * ldv + e % n];
  const float s = (i % 2) ? 0.f : ((i / 2) % 2 ? -1.f : 1.f);
  W[t] = make_float2(s * (float)v.x, s * (float)v.y);
}

// E: the part of A^{-1} M w that the block rows 0..m-2 fix (E_0 = 0, E_1 = y_0,
// E_{r+1} = y_r - E_{r-1}; y_0 = w_0, y_r = 2 w_r), one thread per element of a block
__global__ void cip_recur_kernel(const float2* __restrict__ W, int64_t n, int nu, int m,
                                 float2* __restrict__ E) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per = n * nu;
  if (e >= per) return;
  float2 em1 = make_float2(0.f, 0.f), ei = W[e];
  E[e] = em1;
  if (m > 1) E[per + e] = ei;
  for (int r = 1; r + 1 < m; ++r) {
    const float2 y = W[(int64_t)r * per + e];
    const float2 en = make_float2(2.f * y.x - em1.x, 2.f * y.y - em1.y);
    E[(int64_t)(r + 1) * per + e] = en;
    em1 = ei;
    ei = en;
  }
}

// X_k = cm_k w_{m-1} - sum_i L_ki E_i (the per-node blocks whose node sum
// sum_k A(x_k) X_k is the right-hand side b of G u = b)
__global__ void cip_nodes_kernel(const float2* __restrict__ W, const float2* __restrict__ E,
                                 int64_t n, int nu, int m, int N, const float* __restrict__ Lk,
                                 const float* __restrict__ cm, float2* __restrict__ X) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per = n * nu;
  if (e >= per) return;
  const float2 wl = W[(int64_t)(m - 1) * per + e];
  for (int k = 0; k < N; ++k) {
    float2 x = make_float2(cm[k] * wl.x, cm[k] * wl.y);
    for (int i = 0; i < m; ++i) {
      const float l = Lk[k * m + i];
      if (l == 0.f) continue;
      const float2 ei = E[(int64_t)i * per + e];
      x.x -= l * ei.x;
      x.y -= l * ei.y;
    }
    X[(int64_t)k * per + e] = x;
  }
}

// W_i = E_i + T_i(0) U
__global__ void cip_combine_kernel(float2* W, const float2* __restrict__ E,
                                   const float2* __restrict__ U, int64_t n, int nu, int m) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per = n * nu;
  if (t >= per * m) return;
  const int i = (int)(t / per);
  const float s = (i % 2) ? 0.f : ((i / 2) % 2 ? -1.f : 1.f);
  const float2 u = U[t % per], ev = E[t];
  W[t] = make_float2(ev.x + s * u.x, ev.y + s * u.y);
}

// Xout[:, cols[c]] = Xc Y[:, c] (Xc n x k, Y k x k column-major, FP64 complex)
__global__ void combine_cols_kernel(const double2* __restrict__ Xc, int64_t n, int k,
                                    const double2* __restrict__ Y, const int* __restrict__ cols,
                                    double2* __restrict__ Xout, int64_t ldx) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int64_t i = t % n;
  const int c = (int)(t / n);
  double2 acc = make_double2(0.0, 0.0);
  for (int q = 0; q < k; ++q) {
    const double2 x = Xc[(int64_t)q * n + i], y = Y[(int64_t)c * k + q];
    acc.x += x.x * y.x - x.y * y.y;
    acc.y += x.x * y.y + x.y * y.x;
  }
  Xout[(int64_t)cols[c] * ldx + i] = acc;
}

unsigned nblk(int64_t count, int t = 256) { return (unsigned)((count + t - 1) / t); }

}  // namespace
}  // namespace bem

using namespace bem;

namespace bem {
namespace {

// q steps of Algorithm 1 on every column of V. mf = false: S assembled densely in FP32 and
// LU-factorised once; mf = true: S applied matrix-free, each solve by restarted GMRES to
// the relative residual tol (at most max_iter Arnoldi steps per solve).
bem_status inverse_power_impl(bem_ctx* ctx, double* V_dev, int64_t ldv, int nu, int q,
                              double shift_re, double shift_im, bool mf, double tol,
                              int max_iter, int* gmres_iters, const char* name, cudaStream_t s) {
  if (!ctx) return BEM_EINVAL;
  if (ctx->geo.n == 0 || ctx->con.N == 0)
    return fail(ctx, BEM_ESTATE, std::string(name) + ": mesh and contour must be set");
  const int64_t n = ctx->geo.n;
  const int N = ctx->con.N;
  if (!V_dev || nu < 1 || nu > kMaxNu || ldv < n || q < 0 || N > kMaxNodesSolve ||
      (mf && (!(tol > 0.0) || max_iter < 1)))
    return fail(ctx, BEM_EINVAL, std::string(name) +
                                     ": need V, 1 <= nu <= 256, ldv >= n, N <= 64 (and tol > 0, "
                                     "max_iter >= 1 without a factorisation)");
  if (gmres_iters) *gmres_iters = 0;
  if (q == 0) return BEM_OK;
  cudaSetDevice(ctx->device);
  // coefficients c_j = w_j / (z_j - s)
  std::vector<double> coef(2 * N);
  for (int j = 0; j < N; ++j) {
    const double zr = ctx->con.z_host[2 * j] - shift_re, zi = ctx->con.z_host[2 * j + 1] - shift_im;
    const double wr = ctx->con.w_host[2 * j], wi = ctx->con.w_host[2 * j + 1];
    const double d = zr * zr + zi * zi;
    coef[2 * j] = (wr * zr + wi * zi) / d;
    coef[2 * j + 1] = (wi * zr - wr * zi) / d;
  }
  const int restart = 40;
  // workspace: S (n^2) and pivots, or the GMRES basis; Vn (N n nu), u' (n nu), b (n nu),
  // norms, node-summed apply
  size_t off = 0;
  auto take = [&](size_t b) { const size_t o = off; off += (b + 255) / 256 * 256; return o; };
  const size_t oS = take(mf ? 0 : (size_t)n * n * sizeof(float2)),
               oP = take(mf ? 0 : (size_t)n * sizeof(int)),
               oG = take(mf ? gmres_sum_work_bytes(ctx, nu, restart) : 0),
               oV = take((size_t)N * n * nu * sizeof(float2)), oU = take((size_t)n * nu * sizeof(float2)),
               oB = take(mf ? (size_t)n * nu * sizeof(float2) : 0),
               oN = take((size_t)nu * sizeof(double)),
               oW = take(mixed_sum_work_bytes(ctx, nu, true));
  bem_status st = ensure_scratch(ctx, off);
  if (st != BEM_OK) return st;
  st = ensure_self32(ctx, s);
  if (st != BEM_OK) return st;
  unsigned char* base = reinterpret_cast<unsigned char*>(ctx->d_scratch);
  float2* S = reinterpret_cast<float2*>(base + oS);
  int* piv = reinterpret_cast<int*>(base + oP);
  float2* Vn = reinterpret_cast<float2*>(base + oV);
  float2* Up = reinterpret_cast<float2*>(base + oU);
  float2* Bt = reinterpret_cast<float2*>(base + oB);
  double* nrm = reinterpret_cast<double*>(base + oN);
  void* sum_work = base + oW;
  if (!mf) {
    st = assemble32(ctx, N, ctx->con.z_host, coef.data(), S, s);
    if (st == BEM_OK) st = lu32(ctx, S, n, piv, s);
    if (st != BEM_OK) return st;
  }
  const double2 sh = make_double2(shift_re, shift_im);
  const double2* z = reinterpret_cast<const double2*>(ctx->con.z);
  const int64_t total = (int64_t)N * n * nu;
  ip_start_kernel<<<nblk(total), 256, 0, s>>>(reinterpret_cast<const double2*>(V_dev), ldv, n, nu,
                                              N, z, sh, Vn);
  ctx->launches++;
  for (int step = 0; step < q; ++step) {
    // b = sum_j c_j A(z_j) v_j (Eq. linsyssim with the sign of Algorithm 1 absorbed in c_j)
    st = mixed_sum_apply(ctx, Vn, n, n * nu, true, nu, coef.data(), mf ? Bt : Up, sum_work, s);
    if (st != BEM_OK) return st;
    if (mf) {
      int it = 0;
      st = gmres_sum32(ctx, coef.data(), Bt, Up, nu, tol, max_iter, restart, base + oG, s, &it,
                       nullptr);
      if (gmres_iters) *gmres_iters += it;
    } else {
      st = lu32_solve(ctx, S, piv, n, Up, nu, s);
    }
    if (st != BEM_OK) return st;
    ip_update_kernel<<<nblk(total), 256, 0, s>>>(Vn, Up, n, nu, N, z, sh);
    ip_colnorm_kernel<<<nu, 256, 0, s>>>(Vn, n, nu, N, nrm);
    ip_scale_kernel<<<nblk(total), 256, 0, s>>>(Vn, Up, n, nu, N, nrm);
    ctx->launches += 3;
  }
  f32_to_f64_kernel<<<nblk(n * nu), 256, 0, s>>>(Up, n, nu, reinterpret_cast<double2*>(V_dev), ldv);
  ctx->launches++;
  st = cuda_check(ctx, cudaGetLastError(), name);
  if (st != BEM_OK) return st;
  return take_status(ctx, s, name);
}

}  // namespace
}  // namespace bem

extern "C" bem_status bem_inverse_power_chebyshev(bem_ctx* ctx, double* V_dev, int64_t ldv,
                                                  int nu, int q, void* stream) {
  const char* name = "bem_inverse_power_chebyshev";
  if (!ctx) return BEM_EINVAL;
  if (ctx->geo.n == 0 || ctx->con.N == 0 || ctx->con.kind != BEM_CONTOUR_CHEBYSHEV)
    return fail(ctx, BEM_ESTATE, std::string(name) + ": mesh and a Chebyshev contour must be set");
  const int64_t n = ctx->geo.n;
  const int N = ctx->con.N, m = N - 1;
  if (!V_dev || nu < 1 || nu > kMaxNu || ldv < n || q < 0 || N < 4 || N > kMaxNodesSolve)
    return fail(ctx, BEM_EINVAL, std::string(name) +
                                     ": need V, 1 <= nu <= 256, ldv >= n, 4 <= N <= 64 points");
  if (q == 0) return BEM_OK;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  // coefficients: B_i = sum_k c_ik A(x_k), c_ik = (2 - delta_i0) / N cos(i pi (k + 1/2) / N);
  // the last block row's L_i = -B_i (i <= m-3), B_m - B_{m-2}, -B_{m-1} as node weights
  // l_ik; G = sum_i T_i(0) L_i = sum_k g_k A(x_k); cm_k = 2 c_mk (y_{m-1} = 2 B_m w_{m-1})
  auto cik = [&](int i, int k) {
    return (i == 0 ? 1.0 : 2.0) / N * cos(i * M_PI * (k + 0.5) / N);
  };
  std::vector<float> Lk((size_t)N * m), cm(N);
  std::vector<double> g(2 * N, 0.0), ones(2 * N, 0.0);
  for (int k = 0; k < N; ++k) {
    for (int i = 0; i < m; ++i) {
      double l;
      if (i <= m - 3) l = -cik(i, k);
      else if (i == m - 2) l = cik(m, k) - cik(m - 2, k);
      else l = -cik(m - 1, k);
      Lk[(size_t)k * m + i] = (float)l;
      const double t0 = (i % 2) ? 0.0 : ((i / 2) % 2 ? -1.0 : 1.0);
      g[2 * k] += t0 * l;
    }
    cm[k] = (float)(2.0 * cik(m, k));
    ones[2 * k] = 1.0;
  }
  size_t off = 0;
  auto take = [&](size_t b) { const size_t o = off; off += (b + 255) / 256 * 256; return o; };
  const size_t blk = (size_t)n * nu * sizeof(float2);
  const size_t oG = take((size_t)n * n * sizeof(float2)), oP = take((size_t)n * sizeof(int)),
               oW = take((size_t)m * blk), oE = take((size_t)m * blk), oX = take((size_t)N * blk),
               oU = take(blk), oN = take((size_t)nu * sizeof(double)),
               oL = take(((size_t)N * m + N) * sizeof(float)),
               oS = take(mixed_sum_work_bytes(ctx, nu, true));
  bem_status st = ensure_scratch(ctx, off);
  if (st != BEM_OK) return st;
  st = ensure_self32(ctx, s);
  if (st != BEM_OK) return st;
  unsigned char* base = reinterpret_cast<unsigned char*>(ctx->d_scratch);
  float2* G = reinterpret_cast<float2*>(base + oG);
  int* piv = reinterpret_cast<int*>(base + oP);
  float2* W = reinterpret_cast<float2*>(base + oW);
  float2* E = reinterpret_cast<float2*>(base + oE);
  float2* X = reinterpret_cast<float2*>(base + oX);
  float2* U = reinterpret_cast<float2*>(base + oU);
  double* nrm = reinterpret_cast<double*>(base + oN);
  float* dL = reinterpret_cast<float*>(base + oL);
  float* dcm = dL + (size_t)N * m;
  st = cuda_check(ctx, cudaMemcpyAsync(dL, Lk.data(), Lk.size() * sizeof(float),
                                       cudaMemcpyHostToDevice, s), name);
  if (st == BEM_OK)
    st = cuda_check(ctx, cudaMemcpyAsync(dcm, cm.data(), cm.size() * sizeof(float),
                                         cudaMemcpyHostToDevice, s), name);
  if (st == BEM_OK) st = assemble32(ctx, N, ctx->con.z_host, g.data(), G, s);
  if (st == BEM_OK) st = lu32(ctx, G, n, piv, s);
  if (st != BEM_OK) return st;
  const int64_t per = n * nu;
  cip_start_kernel<<<nblk(per * m), 256, 0, s>>>(reinterpret_cast<const double2*>(V_dev), ldv, n,
                                                nu, m, W);
  ctx->launches++;
  for (int step = 0; step < q; ++step) {
    cip_recur_kernel<<<nblk(per), 256, 0, s>>>(W, n, nu, m, E);
    cip_nodes_kernel<<<nblk(per), 256, 0, s>>>(W, E, n, nu, m, N, dL, dcm, X);
    ctx->launches += 2;
    // b = sum_k A(x_k) X_k (the node-summed fused kernel), then u = G^{-1} b
    st = mixed_sum_apply(ctx, X, n, n * nu, true, nu, ones.data(), U, base + oS, s);
    if (st == BEM_OK) st = lu32_solve(ctx, G, piv, n, U, nu, s);
    if (st != BEM_OK) return st;
    cip_combine_kernel<<<nblk(per * m), 256, 0, s>>>(W, E, U, n, nu, m);
    ip_colnorm_kernel<<<nu, 256, 0, s>>>(W, n, nu, m, nrm);
    ip_scale_kernel<<<nblk(per * m), 256, 0, s>>>(W, U, n, nu, m, nrm);
    ctx->launches += 3;
  }
  // the basis: u = v_0, the y-part of the linearisation
  f32_to_f64_kernel<<<nblk(per), 256, 0, s>>>(W, n, nu, reinterpret_cast<double2*>(V_dev), ldv);
  ctx->launches++;
  st = cuda_check(ctx, cudaGetLastError(), name);
  if (st != BEM_OK) return st;
  return take_status(ctx, s, name);
}

extern "C" bem_status bem_inverse_power(bem_ctx* ctx, double* V_dev, int64_t ldv, int nu, int q,
                                        double shift_re, double shift_im, void* stream) {
  return inverse_power_impl(ctx, V_dev, ldv, nu, q, shift_re, shift_im, false, 0.0, 0, nullptr,
                            "bem_inverse_power", (cudaStream_t)stream);
}

extern "C" bem_status bem_inverse_power_mf(bem_ctx* ctx, double* V_dev, int64_t ldv, int nu,
                                           int q, double shift_re, double shift_im, double tol,
                                           int max_iter, int* gmres_iters, void* stream) {
  return inverse_power_impl(ctx, V_dev, ldv, nu, q, shift_re, shift_im, true, tol, max_iter,
                            gmres_iters, "bem_inverse_power_mf", (cudaStream_t)stream);
}

extern "C" bem_status bem_solve_sum(bem_ctx* ctx, const double* coef_host, const double* B_dev,
                                    int64_t ldb, int nu, double tol, int max_iter,
                                    double* X_dev, int64_t ldx, int* iters, double* relres_host,
                                    void* stream) {
  if (!ctx) return BEM_EINVAL;
  if (ctx->geo.n == 0 || ctx->con.N == 0)
    return fail(ctx, BEM_ESTATE, "bem_solve_sum: mesh and contour must be set");
  const int64_t n = ctx->geo.n;
  if (!coef_host || !B_dev || !X_dev || nu < 1 || nu > kMaxNu || ldb < n || ldx < n ||
      !(tol > 0.0) || max_iter < 1)
    return fail(ctx, BEM_EINVAL,
                "bem_solve_sum: need coefficients, B, X, 1 <= nu <= 256, ldb, ldx >= n, tol > 0, "
                "max_iter >= 1");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int restart = 40;
  size_t off = 0;
  auto take = [&](size_t b) { const size_t o = off; off += (b + 255) / 256 * 256; return o; };
  const size_t oB = take((size_t)n * nu * sizeof(float2)), oX = take((size_t)n * nu * sizeof(float2)),
               oG = take(gmres_sum_work_bytes(ctx, nu, restart));
  bem_status st = ensure_scratch(ctx, off);
  if (st != BEM_OK) return st;
  st = ensure_self32(ctx, s);
  if (st != BEM_OK) return st;
  unsigned char* base = reinterpret_cast<unsigned char*>(ctx->d_scratch);
  float2* B32 = reinterpret_cast<float2*>(base + oB);
  float2* X32 = reinterpret_cast<float2*>(base + oX);
  x_to_f32_kernel<<<nblk(n * nu), 256, 0, s>>>(reinterpret_cast<const double2*>(B_dev), ldb, 0,
                                               n, nu, 1, B32);
  ctx->launches++;
  st = gmres_sum32(ctx, coef_host, B32, X32, nu, tol, max_iter, restart, base + oG, s, iters,
                   relres_host);
  if (st != BEM_OK) return st;
  f32_to_f64_kernel<<<nblk(n * nu), 256, 0, s>>>(X32, n, nu, reinterpret_cast<double2*>(X_dev), ldx);
  ctx->launches++;
  st = cuda_check(ctx, cudaGetLastError(), "bem_solve_sum");
  if (st != BEM_OK) return st;
  return take_status(ctx, s, "bem_solve_sum");
}

extern "C" bem_status bem_apply_sum(bem_ctx* ctx, const double* coef_host, const double* X_dev,
                                    int64_t ldx, int nu, int per_node, double* Y_dev,
                                    void* stream) {
  if (!ctx) return BEM_EINVAL;
  if (ctx->geo.n == 0 || ctx->con.N == 0)
    return fail(ctx, BEM_ESTATE, "bem_apply_sum: mesh and contour must be set");
  const int64_t n = ctx->geo.n;
  const int N = ctx->con.N;
  if (!coef_host || !X_dev || !Y_dev || nu < 1 || nu > kMaxNu || ldx < n)
    return fail(ctx, BEM_EINVAL, "bem_apply_sum: need coefficients, X, Y, 1 <= nu <= 256, ldx >= n");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int nn = per_node ? N : 1;
  size_t off = 0;
  auto take = [&](size_t b) { const size_t o = off; off += (b + 255) / 256 * 256; return o; };
  const size_t oX = take((size_t)nn * n * nu * sizeof(float2)),
               oY = take((size_t)n * nu * sizeof(float2)),
               oW = take(mixed_sum_work_bytes(ctx, nu, per_node != 0));
  bem_status st = ensure_scratch(ctx, off);
  if (st != BEM_OK) return st;
  unsigned char* base = reinterpret_cast<unsigned char*>(ctx->d_scratch);
  float2* X32 = reinterpret_cast<float2*>(base + oX);
  float2* Y32 = reinterpret_cast<float2*>(base + oY);
  x_to_f32_kernel<<<nblk((int64_t)nn * n * nu), 256, 0, s>>>(
      reinterpret_cast<const double2*>(X_dev), ldx, ldx * nu, n, nu, nn, X32);
  ctx->launches++;
  st = mixed_sum_apply(ctx, X32, n, n * nu, per_node != 0, nu, coef_host, Y32, base + oW, s);
  if (st != BEM_OK) return st;
  f32_to_f64_kernel<<<nblk(n * nu), 256, 0, s>>>(Y32, n, nu, reinterpret_cast<double2*>(Y_dev), n);
  ctx->launches++;
  st = cuda_check(ctx, cudaGetLastError(), "bem_apply_sum");
  if (st != BEM_OK) return st;
  return take_status(ctx, s, "bem_apply_sum");
}

extern "C" bem_status bem_refine(bem_ctx* ctx, int m, double* lam_host, double* X_dev,
                                 int64_t ldx, double tol, int maxit, double* relres_host,
                                 int* iters_host, void* stream) {
  if (!ctx) return BEM_EINVAL;
  if (ctx->geo.n == 0) return fail(ctx, BEM_ESTATE, "bem_refine: no mesh set");
  const int64_t n = ctx->geo.n;
  if (m < 1 || !lam_host || !X_dev || ldx < n || !relres_host || !(tol > 0.0) || maxit < 1)
    return fail(ctx, BEM_EINVAL, "bem_refine: bad arguments");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  {
    const bem_status sn = ensure_near(ctx, s);
    if (sn != BEM_OK) return sn;
  }
  size_t off = 0;
  auto take = [&](size_t b) { const size_t o = off; off += (b + 255) / 256 * 256; return o; };
  const size_t oA = take((size_t)n * n * sizeof(float2)), oP = take((size_t)n * sizeof(int)),
               oR = take((size_t)2 * n * sizeof(double2)), oF = take((size_t)2 * n * sizeof(float2)),
               oE = take((size_t)n * sizeof(double2)), oL = take(8 * sizeof(double2)),
               oD = take(8 * sizeof(double2));
  bem_status st = ensure_scratch(ctx, off);
  if (st != BEM_OK) return st;
  unsigned char* base = reinterpret_cast<unsigned char*>(ctx->d_scratch);
  float2* A = reinterpret_cast<float2*>(base + oA);
  int* piv = reinterpret_cast<int*>(base + oP);
  double2* R = reinterpret_cast<double2*>(base + oR);
  float2* F = reinterpret_cast<float2*>(base + oF);
  double2* e = reinterpret_cast<double2*>(base + oE);
  double2* dlam = reinterpret_cast<double2*>(base + oL);
  double2* dots = reinterpret_cast<double2*>(base + oD);
  double2 hd[3];
  const double one[2] = {1.0, 0.0};
  // eigenpairs in order of Re lambda, so that the Ritz values of one multiple eigenvalue
  // (equal to ~1e-7 relative) follow each other and share the factorisation of A(sigma),
  // the refinement's dominant cost at large n. Distinct eigenvalues, even those a mesh
  // splits by 1e-5 (sphere20480: 6.989352 x 3 and 6.989424 x 4), each get their own: a
  // shift nearer to the neighbour pulls the iteration onto the neighbour's eigenspace.
  std::vector<int> order(m);
  for (int c = 0; c < m; ++c) order[c] = c;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return lam_host[2 * a] < lam_host[2 * b]; });
  double sig_r = 0.0, sig_i = 0.0;
  bool have_lu = false;
  for (int oc = 0; oc < m; ++oc) {
    const int c = order[oc];
    double2* x = reinterpret_cast<double2*>(X_dev) + (int64_t)c * ldx;
    double lr = lam_host[2 * c], li = lam_host[2 * c + 1];
    if (have_lu && hypot(lr - sig_r, li - sig_i) > 1e-7 * hypot(sig_r, sig_i)) have_lu = false;
    // e = x0, x normalised so that e^H x = 1
    st = cuda_check(ctx, cudaMemcpyAsync(e, x, n * sizeof(double2), cudaMemcpyDeviceToDevice, s), "refine");
    if (st != BEM_OK) return st;
    dot1_kernel<<<1, 256, 0, s>>>(e, x, n, dots);
    ctx->launches++;
    st = cuda_check(ctx, cudaMemcpyAsync(hd, dots, sizeof(double2), cudaMemcpyDeviceToHost, s), "refine");
    if (st == BEM_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), "refine");
    if (st != BEM_OK) return st;
    scale_vec_kernel<<<nblk(n), 256, 0, s>>>(x, n, hd[0]);
    ctx->launches++;
    double dl_prev = INFINITY;
    int it = 0, factorisations = 0;
    // a Ritz value that is not an eigenvalue (reading of the paper's spurious values)
    // makes lambda wander off: stop once it leaves twice the contour's extent
    const double c_re = ctx->con.c_re, c_im = ctx->con.c_im;
    const double reach = 2.0 * std::max(ctx->con.a, ctx->con.b);
    for (; it < maxit; ++it) {
      if (!have_lu && factorisations >= kMaxFactorisations) have_lu = true;   // keep the last
      if (!have_lu) {
        ++factorisations;
        sig_r = lr;
        sig_i = li;
        const double k[2] = {sig_r, sig_i};
        st = assemble32(ctx, 1, k, one, A, s);
        if (st == BEM_OK) st = lu32(ctx, A, n, piv, s);
        if (st != BEM_OK) return st;
        have_lu = true;
      }
      const double lamv[2] = {lr, li};
      st = cuda_check(ctx, cudaMemcpyAsync(dlam, lamv, sizeof(double2), cudaMemcpyHostToDevice, s), "refine");
      if (st != BEM_OK) return st;
      // r = A(lambda) x and r' = A'(lambda) x in one double-FP32 pass (entries to ~1e-13,
      // far below the residuals the iteration reaches; the final residuals are FP64)
      if (launch_apply_ff(ctx, 1, reinterpret_cast<double*>(dlam), reinterpret_cast<double*>(x),
                          n, reinterpret_cast<double*>(R), reinterpret_cast<double*>(R + n),
                          s) != cudaSuccess)
        return fail(ctx, BEM_ECUDA, "refine residual");
      // ||r||^2 and ||x||^2 of the current pair (stop once the residual is at the level the
      // double-FP32 entries resolve)
      if (launch_colnorms(ctx, reinterpret_cast<double*>(R), n, reinterpret_cast<double*>(x), n,
                          n, 1, reinterpret_cast<double*>(dots + 2), s) != cudaSuccess)
        return fail(ctx, BEM_ECUDA, "refine norms");
      to_f32_kernel<<<nblk(2 * n), 256, 0, s>>>(R, 2 * n, F);
      ctx->launches++;
      st = lu32_solve(ctx, A, piv, n, F, 2, s);
      if (st != BEM_OK) return st;
      dot2_kernel<<<2, 256, 0, s>>>(e, F, n, dots);
      ctx->launches++;
      st = cuda_check(ctx, cudaMemcpyAsync(hd, dots, 3 * sizeof(double2), cudaMemcpyDeviceToHost, s), "refine");
      if (st == BEM_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), "refine");
      if (st != BEM_OK) return st;
      if (hd[2].y > 0.0 && sqrt(hd[2].x / hd[2].y) <= kResidualStop) break;
      // dlambda = -(e^H s1) / (e^H s2)
      const double dd = hd[1].x * hd[1].x + hd[1].y * hd[1].y;
      if (!(dd > 0.0)) break;
      const double dr = -(hd[0].x * hd[1].x + hd[0].y * hd[1].y) / dd;
      const double di = -(hd[0].y * hd[1].x - hd[0].x * hd[1].y) / dd;
      refine_update_kernel<<<nblk(n), 256, 0, s>>>(x, F, n, make_double2(dr, di));
      dot1_kernel<<<1, 256, 0, s>>>(e, x, n, dots);
      ctx->launches += 2;
      st = cuda_check(ctx, cudaMemcpyAsync(hd, dots, sizeof(double2), cudaMemcpyDeviceToHost, s), "refine");
      if (st == BEM_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), "refine");
      if (st != BEM_OK) return st;
      scale_vec_kernel<<<nblk(n), 256, 0, s>>>(x, n, hd[0]);
      ctx->launches++;
      lr += dr;
      li += di;
      if (hypot(lr - c_re, li - c_im) > reach) {   // not an eigenvalue near the contour
        ++it;
        break;
      }
      const double step = hypot(dr, di), lam_abs = hypot(lr, li);
      // steps below the double-FP32 residuals' resolution (~1e-13 of lambda) are noise
      if (step <= std::max(tol, kStepFloor) * lam_abs) {
        ++it;
        break;
      }
      // stalled well above that floor: refactor at the current lambda
      if (step > 0.1 * dl_prev && step > 1e-9 * lam_abs) have_lu = false;
      dl_prev = step;
    }
    lam_host[2 * c] = lr;
    lam_host[2 * c + 1] = li;
    if (iters_host) iters_host[c] = it;
  }
  // final FP64 residuals
  return bem_residual_arith(ctx, m, lam_host, X_dev, ldx, nullptr, nullptr, relres_host,
                            ctx->final_residual_arith, stream);
}

namespace bem {
namespace {

// theta and y of M0 y = -theta M1 y (k x k, column-major, host): the eigenpairs of
// -M1^{-1} M0 (Gaussian elimination with partial pivoting, then the small dense solver).
bool small_pencil(int k, std::vector<small::zc> M0, std::vector<small::zc> M1,
                  std::vector<small::zc>& theta, std::vector<small::zc>& Y) {
  using namespace small;
  auto E = [k](std::vector<zc>& Mx, int i, int j) -> zc& { return Mx[(size_t)j * k + i]; };
  // solve M1 Z = -M0
  std::vector<zc> Z(k * k);
  for (int i = 0; i < k * k; ++i) Z[i] = scl(M0[i], -1.0);
  for (int c = 0; c < k; ++c) {
    int p = c;
    for (int r = c + 1; r < k; ++r)
      if (absz(E(M1, r, c)) > absz(E(M1, p, c))) p = r;
    if (!(absz(E(M1, p, c)) > 0.0)) return false;
    if (p != c) {
      for (int j = 0; j < k; ++j) std::swap(E(M1, c, j), E(M1, p, j));
      for (int j = 0; j < k; ++j) std::swap(E(Z, c, j), E(Z, p, j));
    }
    for (int r = c + 1; r < k; ++r) {
      const zc f = dvd(E(M1, r, c), E(M1, c, c));
      for (int j = c; j < k; ++j)
        E(M1, r, j) = sub(E(M1, r, j), mul(f, E(M1, c, j)));
      for (int j = 0; j < k; ++j)
        E(Z, r, j) = sub(E(Z, r, j), mul(f, E(Z, c, j)));
    }
  }
  for (int j = 0; j < k; ++j)
    for (int r = k - 1; r >= 0; --r) {
      zc v = E(Z, r, j);
      for (int q = r + 1; q < k; ++q) v = sub(v, mul(E(M1, r, q), E(Z, q, j)));
      E(Z, r, j) = dvd(v, E(M1, r, r));
    }
  theta.assign(k, mk(0.0, 0.0));
  Y.assign(k * k, mk(0.0, 0.0));
  std::vector<zc> W(k * k);
  return eig(k, Z.data(), theta.data(), Y.data(), W.data()) == 0;
}

// Near-degenerate clusters of Ritz values (consecutive values within 1e-3 relative, whose
// spread exceeds 1e-7 relative: distinct eigenvalues that the mesh splits, such as
// sphere20480's 6.989352 x 3 and 6.989424 x 4, 7e-5 apart). The mixed projection's error
// (~1e-5) mixes the Ritz vectors of such eigenvalues, and a refinement vector by vector then
// lands on the wrong one. On the subspace X of a cluster's Ritz vectors:
//  (1) two steps of block inverse iteration X <- orth(A(s)^{-1} A'(s) X), s the cluster's
//      mean: its invariant subspace gains |rest - s| / |cluster - s| (~1e4) per step;
//  (2) the projected problem X^H A(lambda) X y = 0 by successive linear problems (Ruhe):
//      at mu, M0 = X^H A(mu) X, M1 = X^H A'(mu) X and M0 y = -theta M1 y; all k values
//      from mu = s, then one more step for each at its own mu = s + theta;
//  (3) the cluster's Ritz pairs replaced by (mu + theta, X y), y from the step at s (so
//      that the members of a multiple eigenvalue keep independent vectors).
// A(s) is factorised in FP32; the applications of A and A' are double-FP32.
bem_status separate_clusters(bem_ctx* ctx, int k, double* lam, double* X_dev, int64_t ldx,
                             cudaStream_t s) {
  using namespace small;
  const int64_t n = ctx->geo.n;
  std::vector<int> order(k);
  for (int i = 0; i < k; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return lam[2 * a] < lam[2 * b]; });
  const double one[2] = {1.0, 0.0};
  for (int b0 = 0; b0 < k;) {
    int b1 = b0 + 1;
    while (b1 < k && hypot(lam[2 * order[b1]] - lam[2 * order[b1 - 1]],
                           lam[2 * order[b1] + 1] - lam[2 * order[b1 - 1] + 1]) <=
                         1e-3 * hypot(lam[2 * order[b1]], lam[2 * order[b1] + 1]))
      ++b1;
    const int kc = b1 - b0;
    double sr = 0.0, si = 0.0, spread = 0.0;
    for (int q = b0; q < b1; ++q) {
      sr += lam[2 * order[q]] / kc;
      si += lam[2 * order[q] + 1] / kc;
    }
    for (int q = b0; q < b1; ++q)
      spread = std::max(spread, hypot(lam[2 * order[q]] - sr, lam[2 * order[q] + 1] - si));
    const int c0 = b0;
    b0 = b1;
    if (kc < 2 || kc > 32 || spread <= 1e-7 * hypot(sr, si)) continue;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
    const size_t oA = take((size_t)n * n * sizeof(float2)), oP = take((size_t)n * sizeof(int)),
                 oX = take((size_t)n * kc * sizeof(double2)), oR = take((size_t)n * kc * sizeof(double2)),
                 oD = take((size_t)n * kc * sizeof(double2)), oF = take((size_t)n * kc * sizeof(float2)),
                 oM = take((size_t)2 * kc * kc * sizeof(double2)), oL = take((size_t)2 * kc * sizeof(double)),
                 oY = take((size_t)kc * kc * sizeof(double2)), oC = take((size_t)kc * sizeof(int));
    bem_status st = ensure_scratch(ctx, off);
    if (st != BEM_OK) return st;
    unsigned char* base = reinterpret_cast<unsigned char*>(ctx->d_scratch);
    float2* A = reinterpret_cast<float2*>(base + oA);
    int* piv = reinterpret_cast<int*>(base + oP);
    double2* Xc = reinterpret_cast<double2*>(base + oX);
    double2* R = reinterpret_cast<double2*>(base + oR);
    double2* D = reinterpret_cast<double2*>(base + oD);
    float2* F = reinterpret_cast<float2*>(base + oF);
    double2* M = reinterpret_cast<double2*>(base + oM);
    double* dlam = reinterpret_cast<double*>(base + oL);
    double2* dY = reinterpret_cast<double2*>(base + oY);
    int* dcols = reinterpret_cast<int*>(base + oC);
    std::vector<int> cols(kc);
    for (int q = 0; q < kc; ++q) {
      cols[q] = order[c0 + q];
      st = cuda_check(ctx, cudaMemcpyAsync(Xc + (int64_t)q * n, reinterpret_cast<double2*>(X_dev) +
                                               (int64_t)cols[q] * ldx, n * sizeof(double2),
                                           cudaMemcpyDeviceToDevice, s), "cluster copy");
      if (st != BEM_OK) return st;
    }
    const double sh[2] = {sr, si};
    st = assemble32(ctx, 1, sh, one, A, s);
    if (st == BEM_OK) st = lu32(ctx, A, n, piv, s);
    if (st != BEM_OK) return st;
    std::vector<double> lv(2 * kc);
    // M0 = Xc^H A(mu) Xc, M1 = Xc^H A'(mu) Xc on the host
    auto project_at = [&](double mr, double mi, std::vector<zc>& M0, std::vector<zc>& M1) {
      for (int q = 0; q < kc; ++q) { lv[2 * q] = mr; lv[2 * q + 1] = mi; }
      bem_status r = cuda_check(ctx, cudaMemcpyAsync(dlam, lv.data(), lv.size() * sizeof(double),
                                                     cudaMemcpyHostToDevice, s), "cluster");
      if (r != BEM_OK) return r;
      if (launch_apply_ff(ctx, kc, dlam, reinterpret_cast<double*>(Xc), n,
                          reinterpret_cast<double*>(R), reinterpret_cast<double*>(D), s) != cudaSuccess ||
          launch_xhy_fp64(ctx, reinterpret_cast<double*>(Xc), n, kc, reinterpret_cast<double*>(R),
                          n, 0, kc, n, 1, nullptr, reinterpret_cast<double*>(M), s) != cudaSuccess ||
          launch_xhy_fp64(ctx, reinterpret_cast<double*>(Xc), n, kc, reinterpret_cast<double*>(D),
                          n, 0, kc, n, 1, nullptr, reinterpret_cast<double*>(M + kc * kc), s) != cudaSuccess)
        return fail(ctx, BEM_ECUDA, "cluster projection");
      std::vector<double2> h(2 * kc * kc);
      r = cuda_check(ctx, cudaMemcpyAsync(h.data(), M, h.size() * sizeof(double2),
                                          cudaMemcpyDeviceToHost, s), "cluster");
      if (r == BEM_OK) r = cuda_check(ctx, cudaStreamSynchronize(s), "cluster");
      M0.resize(kc * kc);
      M1.resize(kc * kc);
      for (int q = 0; q < kc * kc; ++q) {
        M0[q] = mk(h[q].x, h[q].y);
        M1[q] = mk(h[kc * kc + q].x, h[kc * kc + q].y);
      }
      return r;
    };
    // (1) block inverse iteration with A(s)^{-1} A'(s)
    for (int step = 0; step < 2; ++step) {
      for (int q = 0; q < kc; ++q) { lv[2 * q] = sr; lv[2 * q + 1] = si; }
      st = cuda_check(ctx, cudaMemcpyAsync(dlam, lv.data(), lv.size() * sizeof(double),
                                           cudaMemcpyHostToDevice, s), "cluster");
      if (st != BEM_OK) return st;
      if (launch_apply_ff(ctx, kc, dlam, reinterpret_cast<double*>(Xc), n,
                          reinterpret_cast<double*>(R), reinterpret_cast<double*>(D), s) != cudaSuccess)
        return fail(ctx, BEM_ECUDA, "cluster iteration");
      to_f32_kernel<<<nblk(n * kc), 256, 0, s>>>(D, n * kc, F);
      ctx->launches++;
      st = lu32_solve(ctx, A, piv, n, F, kc, s);
      if (st != BEM_OK) return st;
      f32_to_f64_kernel<<<nblk(n * kc), 256, 0, s>>>(F, n, kc, Xc, n);
      ctx->launches++;
      st = bem_cholqr2(ctx, reinterpret_cast<double*>(Xc), n, n, kc, nullptr, s);
      if (st != BEM_OK) return st;
    }
    // (2) successive linear problems on the projected problem
    std::vector<zc> M0, M1, th, Yv, th2, Y2, Ysel(kc * kc);
    st = project_at(sr, si, M0, M1);
    if (st != BEM_OK) return st;
    if (!small_pencil(kc, M0, M1, th, Yv)) continue;   // leave the cluster to the refinement
    std::vector<double> newlam(2 * kc);
    bool ok = true;
    for (int q = 0; q < kc && ok; ++q) {
      const double mr = sr + th[q].re, mi = si + th[q].im;
      st = project_at(mr, mi, M0, M1);
      if (st != BEM_OK) return st;
      ok = small_pencil(kc, M0, M1, th2, Y2);
      if (!ok) break;
      int best = 0;
      for (int r = 1; r < kc; ++r)
        if (absz(th2[r]) < absz(th2[best])) best = r;
      newlam[2 * q] = mr + th2[best].re;
      newlam[2 * q + 1] = mi + th2[best].im;
      // the vectors from the step at s: distinct for every member of a multiple
      // eigenvalue (the refinement polishes them)
      for (int r = 0; r < kc; ++r) Ysel[(int64_t)q * kc + r] = Yv[(size_t)q * kc + r];
    }
    if (!ok) continue;
    // (3) the cluster's pairs: (mu + theta, Xc y)
    std::vector<double2> hy(kc * kc);
    for (int q = 0; q < kc * kc; ++q) hy[q] = make_double2(Ysel[q].re, Ysel[q].im);
    st = cuda_check(ctx, cudaMemcpyAsync(dY, hy.data(), hy.size() * sizeof(double2),
                                         cudaMemcpyHostToDevice, s), "cluster");
    if (st == BEM_OK)
      st = cuda_check(ctx, cudaMemcpyAsync(dcols, cols.data(), kc * sizeof(int),
                                           cudaMemcpyHostToDevice, s), "cluster");
    if (st != BEM_OK) return st;
    combine_cols_kernel<<<nblk(n * kc), 256, 0, s>>>(Xc, n, kc, dY, dcols,
                                                     reinterpret_cast<double2*>(X_dev), ldx);
    ctx->launches++;
    st = cuda_check(ctx, cudaStreamSynchronize(s), "cluster");
    if (st != BEM_OK) return st;
    for (int q = 0; q < kc; ++q) {
      lam[2 * cols[q]] = newlam[2 * q];
      lam[2 * cols[q] + 1] = newlam[2 * q + 1];
    }
  }
  return BEM_OK;
}

}  // namespace
}  // namespace bem

extern "C" bem_status bem_solve(bem_ctx* ctx, const double* V0_dev, int64_t ldv, int nu, int q,
                                int precision, double tol, int kmax, double* lam_host,
                                double* X_dev, int64_t ldx, int* k_found, double* relres_host,
                                void* stream) {
  if (!ctx) return BEM_EINVAL;
  if (ctx->geo.n == 0 || ctx->con.N == 0)
    return fail(ctx, BEM_ESTATE, "bem_solve: mesh and contour must be set");
  if (ctx->con.kind == BEM_CONTOUR_CHEBYSHEV)
    return fail(ctx, BEM_ESTATE, "bem_solve: needs a closed contour (circle or ellipse)");
  const int64_t n = ctx->geo.n;
  const int N = ctx->con.N;
  if (!V0_dev || nu < 1 || nu > kMaxNu || nu > n || ldv < n || q < 0 || kmax < 1 ||
      !lam_host || !X_dev || ldx < n || !k_found || !relres_host || !(tol > 0.0))
    return fail(ctx, BEM_EINVAL, "bem_solve: bad arguments");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  {
    const bem_status sn = ensure_near(ctx, s);
    if (sn != BEM_OK) return sn;
  }
  const Contour& con = ctx->con;
  const int p = (int)std::min<int64_t>(std::min<int64_t>((int64_t)N * nu, 256), std::max(2 * nu, 32));
  // solve-owned buffers: basis V (n nu), Bhat (N nu^2), Y (nu p), Ritz vectors (n p)
  const size_t bV = (size_t)n * nu * 16, bB = (size_t)N * nu * nu * 16, bY = (size_t)nu * p * 16,
               bX = (size_t)n * p * 16;
  const size_t need = bV + bB + bY + bX + 4 * 256;
  if (need > ctx->solve_bytes) {
    cudaFree(ctx->d_solve);
    ctx->d_solve = nullptr;
    ctx->solve_bytes = 0;
    if (cudaMalloc(&ctx->d_solve, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, BEM_ENOMEM, "bem_solve: buffer allocation failed");
    }
    ctx->solve_bytes = need;
  }
  unsigned char* base = reinterpret_cast<unsigned char*>(ctx->d_solve);
  double* V = reinterpret_cast<double*>(base);
  double* Bh = reinterpret_cast<double*>(base + (bV + 255) / 256 * 256);
  double* Y = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(Bh) + (bB + 255) / 256 * 256);
  double* Xc = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(Y) + (bY + 255) / 256 * 256);
  bem_status st = cuda_check(ctx, cudaMemcpy2DAsync(V, n * 16, V0_dev, ldv * 16, n * 16, nu,
                                                    cudaMemcpyDeviceToDevice, s), "bem_solve copy");
  if (st != BEM_OK) return st;
  // 1. basis: q inverse power steps about the contour's centre (Algorithm 1), then
  //    CholeskyQR2 (orthonormal basis for the Rayleigh-Ritz projection). The Cauchy
  //    linearisation has n eigenvalues clustered at every node; on a flat ellipse the
  //    nodes nearest the centre are closer to the shift than the wanted eigenvalues and
  //    would capture the iteration, so the basis is built on the circle of radius
  //    2 max(a, b) about the same centre (nodes at least twice as far as anything inside
  //    the contour), and the contour is restored for the projection.
  const int kind0 = con.kind, N0 = con.N;
  const double c_re = con.c_re, c_im = con.c_im, a0 = con.a, b0 = con.b;
  const double rb = 2.0 * std::max(a0, b0);
  st = bem_set_contour(ctx, BEM_CONTOUR_CIRCLE, c_re, c_im, rb, rb, N0, nullptr, nullptr, stream);
  // The shift sits 0.3 rb above the centre: Algorithm 1 only rescales its columns between
  //    steps, so an eigenvalue within ~1 % of the radius from the shift (sphere20480:
  //    6.9894 against the centre 7.0; ellipsoid98304: 9.0087 against 9.0) outgrows every
  //    other direction by ~100^q and collapses the whole block onto its eigenvector,
  //    losing the other eigenvalues inside the contour. Off the real axis (where the
  //    interior eigenvalues lie) no eigenvalue is that close, and the node clusters of
  //    the basis circle stay at 0.7 rb.
  if (st == BEM_OK) st = bem_inverse_power(ctx, V, n, nu, q, c_re, c_im + 0.3 * rb, stream);
  const bem_status st_restore =
      bem_set_contour(ctx, kind0, c_re, c_im, a0, b0, N0, nullptr, nullptr, stream);
  if (st == BEM_OK) st = st_restore;
  if (st == BEM_OK) st = bem_cholqr2(ctx, V, n, n, nu, nullptr, stream);
  // 2. projection and the reduced problem
  if (st == BEM_OK) st = bem_project(ctx, V, n, nu, Bh, nullptr, precision, stream);
  if (st != BEM_OK) return st;
  // 3. reduced problem: shift-and-invert at K shifts spread along the major axis
  //    (K = round(a/b) for a flat ellipse). The reduced linearisation
  //    has nu eigenvalues clustered at each node; a shift only sees the eigenvalues that
  //    are nearer to it than the nearest node cluster, so on a flat ellipse one shift at
  //    the centre would return node clusters instead of the eigenvalues inside. Each
  //    shift keeps the converged Ritz pairs inside the contour that are nearer to it
  //    than to any other shift (every eigenvalue is reported once).
  //    On a circle (and a near-circular ellipse) one shift at the centre converges the
  //    eigenvalues nearest it first and stops once those have: eigenvalues out towards the
  //    contour, as near to the node clusters as to the centre, are then missed. There the
  //    centre is joined by eight shifts on the ellipse of 0.45 times the semi-axes: an
  //    eigenvalue at 0.75 of the radius is then ~0.36 radii from its nearest shift, the
  //    node clusters at least 0.55 radii from every shift.
  const double amaj = std::max(con.a, con.b), amin = std::min(con.a, con.b);
  const bool along_re = con.a >= con.b;
  int K = std::max(1, std::min(16, (int)lround(amaj / amin)));
  std::vector<double> sr, si;
  if (K == 1) {
    sr.push_back(con.c_re);
    si.push_back(con.c_im + 1e-3 * amin);   // off the real axis
    for (int kk = 0; kk < 8; ++kk) {
      const double t = M_PI * (2.0 * kk + 1.0) / 8.0;
      sr.push_back(con.c_re + 0.45 * con.a * cos(t));
      si.push_back(con.c_im + 0.45 * con.b * sin(t));
    }
    K = 9;
  } else {
    for (int kk = 0; kk < K; ++kk) {
      const double x = -1.0 + (2.0 * kk + 1.0) / K;
      sr.push_back(con.c_re + (along_re ? amaj * x : 0.0));
      si.push_back(con.c_im + (along_re ? 0.0 : amaj * x) + 1e-3 * amin);   // off the real axis
    }
  }
  const int pk = std::min(p, 32);
  std::vector<double> lam(2 * pk), res(pk), lk, ysel;
  std::vector<int> cand_shift;
  int iters = 0;
  int nsel = 0;
  for (int kk = 0; kk < K; ++kk) {
    st = bem_solve_reduced(ctx, Bh, nu, sr[kk], si[kk], pk, 300, 1e-11, lam.data(), Y, res.data(),
                           &iters, stream);
    if (st != BEM_OK) return st;
    for (int i = 0; i < pk; ++i) {
      const double lr = lam[2 * i], li = lam[2 * i + 1];
      const double xr = (lr - con.c_re) / con.a, xi = (li - con.c_im) / con.b;
      if (!(xr * xr + xi * xi < 1.0) || !(res[i] <= 1e-6)) continue;
      int owner = 0;
      double best = INFINITY;
      for (int k2 = 0; k2 < K; ++k2) {
        const double d = hypot(lr - sr[k2], li - si[k2]);
        if (d < best) { best = d; owner = k2; }
      }
      if (owner != kk || nsel >= std::min(kmax, p)) continue;
      st = cuda_check(ctx, cudaMemcpyAsync(Xc + (size_t)2 * nu * nsel, Y + (size_t)2 * nu * i,
                                           nu * 16, cudaMemcpyDeviceToDevice, s), "bem_solve gather");
      if (st != BEM_OK) return st;
      lk.push_back(lr);
      lk.push_back(li);
      ++nsel;
    }
  }
  const int k = nsel;
  *k_found = 0;
  if (k == 0) return take_status(ctx, s, "bem_solve");
  st = bem_ritz_vectors(ctx, V, n, nu, Xc, k, X_dev, ldx, stream);
  if (st != BEM_OK) return st;
  // near-degenerate clusters separated on their own subspace before the refinement
  st = separate_clusters(ctx, k, lk.data(), X_dev, ldx, s);
  if (st != BEM_OK) return st;
  std::vector<double> rr(k);
  // 4. FP64 refinement of every candidate against A(k) itself
  st = bem_refine(ctx, k, lk.data(), X_dev, ldx, tol, 40, rr.data(), nullptr, stream);
  if (st != BEM_OK) return st;
  for (int t = 0; t < k; ++t) {
    lam_host[2 * t] = lk[2 * t];
    lam_host[2 * t + 1] = lk[2 * t + 1];
    relres_host[t] = rr[t];
  }
  *k_found = k;
  return BEM_OK;
}
