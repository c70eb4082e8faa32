// Choice of the approximation order (Section 4, Example 3): the N-node Cauchy approximation
// T~(z) = sum_j w_j T(z_j) / (z_j - z) of the operator is compared with T itself on an inner
// contour (same centre, semi-axes halved: the circle of radius r/2), applied to a block of
// test vectors, for growing N; the order is the first N whose largest relative error on the
// inner contour meets the tolerance. Every application of T is matrix-free in double-FP32
// arithmetic (entries to ~1e-13, launch_apply_ff), so errors down to ~1e-12 are resolved.
#include <math.h>

#include <string>
#include <vector>

#include "internal.h"

namespace bem {
namespace {

// acc_s += c_s R for the nsamples accumulators (coefficients c_s complex, FP64)
__global__ void order_axpy_kernel(const double2* __restrict__ R, int64_t count, int nsamples,
                                  const double2* __restrict__ c, double2* __restrict__ acc) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const double2 r = R[t];
  for (int s = 0; s < nsamples; ++s) {
    const double2 cs = c[s];
    double2& a = acc[(int64_t)s * count + t];
    a.x += cs.x * r.x - cs.y * r.y;
    a.y += cs.x * r.y + cs.y * r.x;
  }
}

// per sample: ||acc_s - exact_s||^2 and ||exact_s||^2 (fixed-order block reduction)
__global__ void order_err_kernel(const double2* __restrict__ acc, const double2* __restrict__ ex,
                                 int64_t count, double* __restrict__ out) {
  __shared__ double sd[256], se[256];
  const int s = blockIdx.x;
  double d = 0.0, e = 0.0;
  for (int64_t t = threadIdx.x; t < count; t += blockDim.x) {
    const double2 a = acc[(int64_t)s * count + t], x = ex[(int64_t)s * count + t];
    d += (a.x - x.x) * (a.x - x.x) + (a.y - x.y) * (a.y - x.y);
    e += x.x * x.x + x.y * x.y;
  }
  sd[threadIdx.x] = d;
  se[threadIdx.x] = e;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sd[threadIdx.x] += sd[threadIdx.x + w];
      se[threadIdx.x] += se[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * s] = sd[0];
    out[2 * s + 1] = se[0];
  }
}

unsigned nblk(int64_t count) { return (unsigned)((count + 255) / 256); }

}  // namespace
}  // namespace bem

using namespace bem;

extern "C" bem_status bem_select_order(bem_ctx* ctx, int kind, double c_re, double c_im,
                                       double a, double b, const int* N_list, int count,
                                       int nsamples, const double* X_dev, int64_t ldx, int ncols,
                                       double tol, int* N_chosen, double* err_out,
                                       void* stream) {
  const char* name = "bem_select_order";
  if (!ctx) return BEM_EINVAL;
  if (ctx->geo.n == 0) return fail(ctx, BEM_ESTATE, std::string(name) + ": no mesh set");
  const int64_t n = ctx->geo.n;
  if ((kind != BEM_CONTOUR_CIRCLE && kind != BEM_CONTOUR_ELLIPSE) || !N_list || count < 1 ||
      nsamples < 1 || nsamples > 64 || !X_dev || ldx < n || ncols < 1 || ncols > 64 ||
      !N_chosen || !err_out || !(tol > 0.0) || !(a > 0.0) || !(b > 0.0 || kind == BEM_CONTOUR_CIRCLE))
    return fail(ctx, BEM_EINVAL, std::string(name) + ": bad arguments");
  for (int k = 0; k < count; ++k)
    if (N_list[k] < 2 || N_list[k] > 1024)
      return fail(ctx, BEM_EINVAL, std::string(name) + ": orders must lie in 2..1024");
  if (kind == BEM_CONTOUR_CIRCLE) b = a;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  bem_status st = ensure_near(ctx, s);
  if (st != BEM_OK) return st;
  // sample points on the inner contour, angles 2 pi (s + 1/4) / nsamples
  std::vector<double> zeta(2 * nsamples);
  for (int q = 0; q < nsamples; ++q) {
    const double t = 2.0 * M_PI * (q + 0.25) / nsamples;
    zeta[2 * q] = c_re + 0.5 * a * cos(t);
    zeta[2 * q + 1] = c_im + 0.5 * b * sin(t);
  }
  const int64_t cnt = n * ncols;
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
  const size_t oR = take((size_t)cnt * sizeof(double2)),
               oA = take((size_t)nsamples * cnt * sizeof(double2)),
               oE = take((size_t)nsamples * cnt * sizeof(double2)),
               oL = take((size_t)2 * ncols * sizeof(double)),
               oC = take((size_t)nsamples * sizeof(double2)),
               oN = take((size_t)2 * nsamples * sizeof(double));
  st = ensure_scratch(ctx, off);
  if (st != BEM_OK) return st;
  unsigned char* base = reinterpret_cast<unsigned char*>(ctx->d_scratch);
  double2* R = reinterpret_cast<double2*>(base + oR);
  double2* acc = reinterpret_cast<double2*>(base + oA);
  double2* exact = reinterpret_cast<double2*>(base + oE);
  double* dlam = reinterpret_cast<double*>(base + oL);
  double2* dc = reinterpret_cast<double2*>(base + oC);
  double* dn = reinterpret_cast<double*>(base + oN);
  std::vector<double> lam(2 * ncols);
  auto apply = [&](double zr, double zi, double2* out) -> bem_status {
    for (int c = 0; c < ncols; ++c) {
      lam[2 * c] = zr;
      lam[2 * c + 1] = zi;
    }
    bem_status r = cuda_check(ctx, cudaMemcpyAsync(dlam, lam.data(), lam.size() * sizeof(double),
                                                   cudaMemcpyHostToDevice, s), name);
    if (r != BEM_OK) return r;
    // the copy must land before the host reuses lam: the apply below reads it on the stream
    r = cuda_check(ctx, launch_apply_ff(ctx, ncols, dlam, X_dev, ldx, reinterpret_cast<double*>(out),
                                        nullptr, s), name);
    if (r == BEM_OK) r = cuda_check(ctx, cudaStreamSynchronize(s), name);
    return r;
  };
  // T(zeta_s) X on every sample point
  for (int q = 0; q < nsamples && st == BEM_OK; ++q)
    st = apply(zeta[2 * q], zeta[2 * q + 1], exact + (int64_t)q * cnt);
  if (st != BEM_OK) return st;
  *N_chosen = -1;
  std::vector<double> z, w, c(2 * nsamples), h(2 * nsamples);
  for (int k = 0; k < count; ++k) {
    const int N = N_list[k];
    z.assign(2 * N, 0.0);
    w.assign(2 * N, 0.0);
    contour_nodes(kind, c_re, c_im, a, b, N, z.data(), w.data());
    st = cuda_check(ctx, cudaMemsetAsync(acc, 0, (size_t)nsamples * cnt * sizeof(double2), s), name);
    if (st != BEM_OK) return st;
    for (int j = 0; j < N; ++j) {
      st = apply(z[2 * j], z[2 * j + 1], R);   // R = T(z_j) X
      if (st != BEM_OK) return st;
      for (int q = 0; q < nsamples; ++q) {   // w_j / (z_j - zeta_q)
        const double dr = z[2 * j] - zeta[2 * q], di = z[2 * j + 1] - zeta[2 * q + 1];
        const double d2 = dr * dr + di * di;
        c[2 * q] = (w[2 * j] * dr + w[2 * j + 1] * di) / d2;
        c[2 * q + 1] = (w[2 * j + 1] * dr - w[2 * j] * di) / d2;
      }
      st = cuda_check(ctx, cudaMemcpyAsync(dc, c.data(), c.size() * sizeof(double),
                                           cudaMemcpyHostToDevice, s), name);
      if (st != BEM_OK) return st;
      order_axpy_kernel<<<nblk(cnt), 256, 0, s>>>(R, cnt, nsamples, dc, acc);
      ctx->launches++;
      st = cuda_check(ctx, cudaStreamSynchronize(s), name);   // c is rewritten next
      if (st != BEM_OK) return st;
    }
    order_err_kernel<<<nsamples, 256, 0, s>>>(acc, exact, cnt, dn);
    ctx->launches++;
    st = cuda_check(ctx, cudaMemcpyAsync(h.data(), dn, h.size() * sizeof(double),
                                         cudaMemcpyDeviceToHost, s), name);
    if (st == BEM_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), name);
    if (st != BEM_OK) return st;
    double e = 0.0;
    for (int q = 0; q < nsamples; ++q)
      e = fmax(e, h[2 * q + 1] > 0.0 ? sqrt(h[2 * q] / h[2 * q + 1]) : INFINITY);
    err_out[k] = e;
    if (*N_chosen < 0 && e <= tol) *N_chosen = N;
  }
  return take_status(ctx, s, name);
}
