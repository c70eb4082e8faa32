// CholeskyQR2 orthonormalisation of the Ritz basis (FP64).
//
// The paper orthonormalises the basis U before the Rayleigh-Ritz projection (Section 4,
// Example 1). CholeskyQR2: G = V^H V, G = R^H R (R upper, positive diagonal),
// V <- V R^{-1}, and the same once more, which restores orthogonality to working
// precision for well-conditioned V. All steps are deterministic (fixed-order sums).
#include <math.h>

#include "internal.h"

namespace bem {
namespace {

// In-place Cholesky of the Hermitian nu x nu matrix G (column-major, upper triangle used):
// on exit the upper triangle holds R with G = R^H R, the strict lower triangle is zero.
// A pivot below 1e-13 of the largest diagonal entry of G counts as loss of rank.
__global__ void __launch_bounds__(1024) cholesky_kernel(double2* G, int nu, int* status) {
  __shared__ double rkk, dmax;
  const int tid = threadIdx.x;
  if (tid == 0) {
    dmax = 0.0;
    for (int k = 0; k < nu; ++k) dmax = fmax(dmax, G[(int64_t)k * nu + k].x);
  }
  __syncthreads();
  for (int k = 0; k < nu; ++k) {
    if (tid == 0) {
      const double d = G[(int64_t)k * nu + k].x;
      if (!(d > 1e-13 * dmax) || !isfinite(d)) {
        atomicOr(status, kStatusNotSPD);
        rkk = 0.0;
      } else {
        rkk = sqrt(d);
      }
      G[(int64_t)k * nu + k] = make_double2(rkk, 0.0);
    }
    __syncthreads();
    if (rkk == 0.0) return;
    for (int jj = k + 1 + tid; jj < nu; jj += blockDim.x) {
      double2 g = G[(int64_t)jj * nu + k];
      G[(int64_t)jj * nu + k] = make_double2(g.x / rkk, g.y / rkk);
    }
    __syncthreads();
    // trailing update of the upper triangle: G_ij -= conj(R_ki) R_kj, k < i <= j
    const int m = nu - k - 1;
    const int64_t total = (int64_t)m * m;
    for (int64_t t = tid; t < total; t += blockDim.x) {
      const int i = k + 1 + (int)(t % m);
      const int jj = k + 1 + (int)(t / m);
      if (i > jj) continue;
      const double2 a = G[(int64_t)i * nu + k];
      const double2 b = G[(int64_t)jj * nu + k];
      double2 g = G[(int64_t)jj * nu + i];
      g.x -= a.x * b.x + a.y * b.y;
      g.y -= a.x * b.y - a.y * b.x;
      G[(int64_t)jj * nu + i] = g;
    }
    __syncthreads();
  }
  for (int64_t t = tid; t < (int64_t)nu * nu; t += blockDim.x) {
    const int i = (int)(t % nu), jj = (int)(t / nu);
    if (i > jj) G[t] = make_double2(0.0, 0.0);
  }
}

// Rinv = R^{-1} for upper-triangular R; one thread per column (back substitution).
__global__ void triangular_inverse_kernel(const double2* R, int nu, double2* Rinv) {
  const int jcol = blockIdx.x * blockDim.x + threadIdx.x;
  if (jcol >= nu) return;
  for (int i = nu - 1; i >= 0; --i) {
    double2 s = make_double2(i == jcol ? 1.0 : 0.0, 0.0);
    if (i <= jcol) {
      for (int m = i + 1; m <= jcol; ++m) {
        const double2 r = R[(int64_t)m * nu + i];
        const double2 x = Rinv[(int64_t)jcol * nu + m];
        s.x -= r.x * x.x - r.y * x.y;
        s.y -= r.x * x.y + r.y * x.x;
      }
      const double2 d = R[(int64_t)i * nu + i];   // real positive
      Rinv[(int64_t)jcol * nu + i] = make_double2(s.x / d.x, s.y / d.x);
    } else {
      Rinv[(int64_t)jcol * nu + i] = make_double2(0.0, 0.0);
    }
  }
}

constexpr int kRows = 8;

// V <- V * M in place, M nu x nu (column-major); each block owns kRows rows of V.
__global__ void __launch_bounds__(256)
right_multiply_kernel(double2* V, int64_t ldv, int64_t n, int nu, const double2* __restrict__ M) {
  __shared__ double2 sV[kRows][kMaxNu];
  const int64_t r0 = (int64_t)blockIdx.x * kRows;
  for (int t = threadIdx.x; t < kRows * nu; t += blockDim.x) {
    const int rr = t % kRows, c = t / kRows;
    const int64_t r = r0 + rr;
    sV[rr][c] = (r < n) ? V[(int64_t)c * ldv + r] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kRows * nu; t += blockDim.x) {
    const int rr = t % kRows, c = t / kRows;
    const int64_t r = r0 + rr;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k <= c; ++k) {   // M is upper triangular
      const double2 a = sV[rr][k];
      const double2 b = M[(int64_t)c * nu + k];
      acc.x += a.x * b.x - a.y * b.y;
      acc.y += a.x * b.y + a.y * b.x;
    }
    if (r < n) V[(int64_t)c * ldv + r] = acc;
  }
}

// C = A * B for upper-triangular nu x nu A, B (one block).
__global__ void upper_product_kernel(const double2* A, const double2* B, int nu, double2* C) {
  for (int64_t t = threadIdx.x; t < (int64_t)nu * nu; t += blockDim.x) {
    const int i = (int)(t % nu), jj = (int)(t / nu);
    double2 acc = make_double2(0.0, 0.0);
    for (int k = i; k <= jj; ++k) {
      const double2 a = A[(int64_t)k * nu + i];
      const double2 b = B[(int64_t)jj * nu + k];
      acc.x += a.x * b.x - a.y * b.y;
      acc.y += a.x * b.y + a.y * b.x;
    }
    C[t] = acc;
  }
}

}  // namespace
}  // namespace bem

using namespace bem;

extern "C" bem_status bem_cholqr2(bem_ctx* ctx, double* V_dev, int64_t n, int64_t ldv, int nu,
                                  double* R_dev, void* stream) {
  if (!ctx) return BEM_EINVAL;
  if (!V_dev || n < 1 || nu < 1 || nu > kMaxNu || ldv < n || nu > n)
    return fail(ctx, BEM_EINVAL, "bem_cholqr2: need V, 1 <= nu <= min(n, 256), ldv >= n");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t mat = (size_t)nu * nu * 2;
  bem_status st = ensure_small(ctx, 4 * mat * sizeof(double));
  if (st != BEM_OK) return st;
  double2* G = reinterpret_cast<double2*>(ctx->d_small);
  double2* Rinv = G + (size_t)nu * nu;
  double2* R1 = Rinv + (size_t)nu * nu;
  double2* R2 = R1 + (size_t)nu * nu;
  for (int pass = 0; pass < 2; ++pass) {
    double2* R = pass == 0 ? R1 : R2;
    st = cuda_check(ctx, launch_xhy_fp64(ctx, V_dev, ldv, nu, V_dev, ldv, 0, nu, n, 1, nullptr,
                                         reinterpret_cast<double*>(R), s), "gram kernel");
    if (st != BEM_OK) return st;
    cholesky_kernel<<<1, 1024, 0, s>>>(R, nu, ctx->d_status);
    triangular_inverse_kernel<<<(nu + 63) / 64, 64, 0, s>>>(R, nu, Rinv);
    right_multiply_kernel<<<(unsigned)((n + kRows - 1) / kRows), 256, 0, s>>>(
        reinterpret_cast<double2*>(V_dev), ldv, n, nu, Rinv);
    ctx->launches += 3;
    st = cuda_check(ctx, cudaGetLastError(), "cholqr kernels");
    if (st != BEM_OK) return st;
  }
  if (R_dev) {
    upper_product_kernel<<<1, 256, 0, s>>>(R2, R1, nu, reinterpret_cast<double2*>(R_dev));
    ctx->launches++;
    st = cuda_check(ctx, cudaGetLastError(), "cholqr kernels");
    if (st != BEM_OK) return st;
  }
  (void)G;
  return take_status(ctx, s, "bem_cholqr2");
}
