// Residuals of approximate eigenpairs, matrix-free in FP64 (Section 4: the accuracy of an
// eigenpair (lambda, u) is ||T(lambda) u||_2 / ||u||_2).
//
// residual_kernel: r = A(lambda_c) x_c, one thread per row, columns of A streamed through
// shared memory in chunks; norms_kernel: ||r_c||^2 and ||x_c||^2 by a fixed-order block
// reduction (deterministic).
#include <math.h>

#include <string>
#include <vector>

#include "internal.h"
#include "selfterm.cuh"

namespace bem {
namespace {

constexpr int kRowsPerBlock = 128;
constexpr int kChunk = 128;

// kDeriv: the k-derivative of the off-diagonal entries, sum_q W_lq i exp(i k r) / (4 pi).
template <bool kDeriv>
__global__ void __launch_bounds__(kRowsPerBlock)
residual_kernel(Geometry g, const double* __restrict__ lam, const double* __restrict__ X,
                int64_t ldx, double* __restrict__ R, OpCoef op) {
  __shared__ double sQ[4][7][kChunk];
  __shared__ double sN[3][kChunk];
  const bool general = !op_single(op);
  __shared__ double2 sX[kChunk];
  const int64_t n = g.n;
  const int c = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * kRowsPerBlock + threadIdx.x;
  const double kr = lam[2 * c], ki = lam[2 * c + 1];
  const double2* x = reinterpret_cast<const double2*>(X) + (int64_t)c * ldx;
  double xi = 0, yi = 0, zi = 0;
  if (i < n) {
    xi = g.cx[i]; yi = g.cx[n + i]; zi = g.cx[2 * n + i];
  }
  double2 acc = make_double2(0.0, 0.0);
  double2 self_x = make_double2(0.0, 0.0);   // x_i, multiplied by the self term below
  for (int64_t l0 = 0; l0 < n; l0 += kChunk) {
    __syncthreads();
    for (int t = threadIdx.x; t < 7 * kChunk; t += blockDim.x) {
      const int q = t / kChunk, lc = t % kChunk;
      const int64_t l = l0 + lc;
      const bool ok = l < n;
      sQ[0][q][lc] = ok ? g.qp[q * n + l] : 0.0;
      sQ[1][q][lc] = ok ? g.qp[(7 + q) * n + l] : 0.0;
      sQ[2][q][lc] = ok ? g.qp[(14 + q) * n + l] : 0.0;
      sQ[3][q][lc] = ok ? g.qw[q * n + l] : 0.0;
    }
    for (int t = threadIdx.x; t < kChunk; t += blockDim.x) {
      const int64_t l = l0 + t;
      sX[t] = (l < n) ? x[l] : make_double2(0.0, 0.0);
      if (general)
        for (int c2 = 0; c2 < 3; ++c2) sN[c2][t] = (l < n) ? g.nrm[c2 * n + l] : 0.0;
    }
    __syncthreads();
    if (i < n) {
      const int lim = (int)((n - l0) < kChunk ? (n - l0) : kChunk);
      for (int lc = 0; lc < lim; ++lc) {
        const int64_t l = l0 + lc;
        if (l == i) {
          self_x = sX[lc];
          continue;
        }
        double2 a = make_double2(0.0, 0.0);
        if (general) {   // T = c_G G + c_H (1/2 I + K), or its k-derivative
          for (int q = 0; q < 7; ++q)
            op_point64(a, op, sQ[3][q][lc], sQ[0][q][lc] - xi, sQ[1][q][lc] - yi,
                       sQ[2][q][lc] - zi, sN[0][lc], sN[1][lc], sN[2][lc], kr, ki, kDeriv);
        } else
        for (int q = 0; q < 7; ++q) {
          const double dx = xi - sQ[0][q][lc], dy = yi - sQ[1][q][lc], dz = zi - sQ[2][q][lc];
          const double r = sqrt(dx * dx + dy * dy + dz * dz);
          double s, co;
          sincos(kr * r, &s, &co);
          const double amp = kDeriv ? sQ[3][q][lc] * exp(-ki * r) : sQ[3][q][lc] * exp(-ki * r) / r;
          if (kDeriv) {   // i * amp * (co + i s)
            a.x -= amp * s;
            a.y += amp * co;
          } else {
            a.x += amp * co;
            a.y += amp * s;
          }
        }
        const double2 v = sX[lc];
        acc.x += a.x * v.x - a.y * v.y;
        acc.y += a.x * v.y + a.y * v.x;
      }
    }
  }
  if (i < n) {
    // R holds A_ii(lambda_c), written by self_at_kernel before this kernel runs
    double2* Rc = reinterpret_cast<double2*>(R) + (int64_t)c * n;
    const double2 sd = Rc[i];
    acc.x += sd.x * self_x.x - sd.y * self_x.y;
    acc.y += sd.x * self_x.y + sd.y * self_x.x;
    Rc[i] = acc;
  }
}

// Self term A_ii(lambda_c) (or its k-derivative) of every row, written into R as the
// multiplier of x_i.
__global__ void self_at_kernel(Geometry g, const double* __restrict__ lam, GL16 gl,
                               double* __restrict__ R, bool deriv, OpCoef op) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= g.n) return;
  double v[3][3], x[3];
  for (int e = 0; e < 3; ++e) {
    const int32_t vi = g.tri[3 * i + e];
    for (int d = 0; d < 3; ++d) v[e][d] = g.xyz[3 * (int64_t)vi + d];
  }
  for (int d = 0; d < 3; ++d) x[d] = g.cx[d * g.n + i];
  // T's self entry: c_G A_ii (+ c_H / 2, whose k-derivative is 0)
  const double2 a = self_term(v, x, make_double2(lam[2 * c], lam[2 * c + 1]), gl, deriv);
  reinterpret_cast<double2*>(R)[(int64_t)c * g.n + i] =
      make_double2(op.cgr * a.x - op.cgi * a.y + (deriv ? 0.0 : 0.5 * op.chr),
                   op.cgr * a.y + op.cgi * a.x + (deriv ? 0.0 : 0.5 * op.chi));
}

__global__ void norms_kernel(const double* __restrict__ R, const double* __restrict__ X,
                             int64_t ldx, int64_t n, double* __restrict__ out) {
  __shared__ double sr[256], sx[256];
  const int c = blockIdx.x;
  const double2* r = reinterpret_cast<const double2*>(R) + (int64_t)c * n;
  const double2* x = reinterpret_cast<const double2*>(X) + (int64_t)c * ldx;
  double ar = 0.0, ax = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    ar += r[i].x * r[i].x + r[i].y * r[i].y;
    ax += x[i].x * x[i].x + x[i].y * x[i].y;
  }
  sr[threadIdx.x] = ar;
  sx[threadIdx.x] = ax;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sr[threadIdx.x] += sr[threadIdx.x + w];
      sx[threadIdx.x] += sx[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * c] = sr[0];
    out[2 * c + 1] = sx[0];
  }
}

}  // namespace

cudaError_t launch_apply_percol64(bem_ctx* ctx, int m, const double* lam_dev, const double* X,
                                  int64_t ldx, double* R, bool deriv, cudaStream_t s) {
  static const GL16 gl = make_gl16();
  const int64_t n = ctx->geo.n;
  dim3 g1((unsigned)((n + 127) / 128), (unsigned)m);
  self_at_kernel<<<g1, 128, 0, s>>>(ctx->geo, lam_dev, gl, R, deriv, ctx->op);
  dim3 g2((unsigned)((n + kRowsPerBlock - 1) / kRowsPerBlock), (unsigned)m);
  if (deriv)
    residual_kernel<true><<<g2, kRowsPerBlock, 0, s>>>(ctx->geo, lam_dev, X, ldx, R, ctx->op);
  else
    residual_kernel<false><<<g2, kRowsPerBlock, 0, s>>>(ctx->geo, lam_dev, X, ldx, R, ctx->op);
  ctx->launches += 2;
  if (near_active(ctx)) return launch_near_percol64(ctx, m, lam_dev, X, ldx, R, deriv, s);
  return cudaGetLastError();
}

cudaError_t launch_self_at(bem_ctx* ctx, int m, const double* lam_dev, double* R, bool deriv,
                           cudaStream_t s) {
  static const GL16 gl = make_gl16();
  dim3 g1((unsigned)((ctx->geo.n + 127) / 128), (unsigned)m);
  self_at_kernel<<<g1, 128, 0, s>>>(ctx->geo, lam_dev, gl, R, deriv, ctx->op);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t launch_colnorms(bem_ctx* ctx, const double* R, int64_t ldr, const double* X,
                            int64_t ldx, int64_t n, int m, double* out, cudaStream_t s) {
  (void)ldr;
  norms_kernel<<<m, 256, 0, s>>>(R, X, ldx, n, out);
  ctx->launches++;
  return cudaGetLastError();
}

}  // namespace bem

using namespace bem;

namespace {

bem_status residual_impl(bem_ctx* ctx, int m, const double* lam_host, const double* X_dev,
                         int64_t ldx, double* R_dev, double* Rd_dev, double* relres_host,
                         int arith, void* stream, const char* name) {
  if (!ctx) return BEM_EINVAL;
  if (ctx->geo.n == 0) return fail(ctx, BEM_ESTATE, std::string(name) + ": no mesh set");
  const int64_t n = ctx->geo.n;
  if (m < 1 || m > 65535 || !lam_host || !X_dev || !relres_host || ldx < n ||
      (arith != 0 && arith != 1))
    return fail(ctx, BEM_EINVAL, std::string(name) +
                                     ": need 1 <= m <= 65535, lam, X, relres, ldx >= n, arith 0/1");
  for (int c = 0; c < 2 * m; ++c)
    if (!isfinite(lam_host[c])) return fail(ctx, BEM_EINVAL, std::string(name) + ": non-finite lambda");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  bem_status st = ensure_near(ctx, s);
  if (st != BEM_OK) return st;
  // workspace: lambda (2m) + norms (2m) [+ R if the caller passes none]
  const size_t small = (size_t)4 * m * sizeof(double);
  st = ensure_small(ctx, small);
  if (st != BEM_OK) return st;
  double* R = R_dev;
  if (!R) {
    st = ensure_scratch(ctx, (size_t)2 * n * m * sizeof(double));
    if (st != BEM_OK) return st;
    R = ctx->d_scratch;
  }
  double* dlam = ctx->d_small;
  double* dnorm = ctx->d_small + 2 * m;
  st = cuda_check(ctx, cudaMemcpyAsync(dlam, lam_host, 2 * m * sizeof(double),
                                       cudaMemcpyHostToDevice, s), name);
  if (st != BEM_OK) return st;
  cudaError_t e;
  if (arith == 1) {
    e = launch_apply_ff(ctx, m, dlam, X_dev, ldx, R, Rd_dev, s);
  } else {
    e = launch_apply_percol64(ctx, m, dlam, X_dev, ldx, R, false, s);
    if (e == cudaSuccess && Rd_dev) e = launch_apply_percol64(ctx, m, dlam, X_dev, ldx, Rd_dev, true, s);
  }
  st = cuda_check(ctx, e, name);
  if (st != BEM_OK) return st;
  st = cuda_check(ctx, launch_colnorms(ctx, R, n, X_dev, ldx, n, m, dnorm, s), name);
  if (st != BEM_OK) return st;
  std::vector<double> h(2 * m);
  st = cuda_check(ctx, cudaMemcpyAsync(h.data(), dnorm, 2 * m * sizeof(double),
                                       cudaMemcpyDeviceToHost, s), name);
  if (st == BEM_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), name);
  if (st != BEM_OK) return st;
  for (int c = 0; c < m; ++c)
    relres_host[c] = h[2 * c + 1] > 0.0 ? sqrt(h[2 * c]) / sqrt(h[2 * c + 1]) : INFINITY;
  return BEM_OK;
}

}  // namespace

extern "C" bem_status bem_residual(bem_ctx* ctx, int m, const double* lam_host, const double* X_dev,
                                   int64_t ldx, double* R_dev, double* relres_host, void* stream) {
  return residual_impl(ctx, m, lam_host, X_dev, ldx, R_dev, nullptr, relres_host, 0, stream,
                       "bem_residual");
}

extern "C" bem_status bem_residual_arith(bem_ctx* ctx, int m, const double* lam_host,
                                         const double* X_dev, int64_t ldx, double* R_dev,
                                         double* Rd_dev, double* relres_host, int arith,
                                         void* stream) {
  return residual_impl(ctx, m, lam_host, X_dev, ldx, R_dev, Rd_dev, relres_host, arith, stream,
                       "bem_residual_arith");
}
