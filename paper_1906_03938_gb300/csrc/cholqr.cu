// CholeskyQR2 orthonormalisation of the Ritz basis (FP64).
//
// The paper orthonormalises the basis U before the Rayleigh-Ritz projection (Section 4,
// Example 1). CholeskyQR2: G = V^H V, G = R^H R (R upper, positive diagonal),
// V <- V R^{-1}, and the same once more, which restores orthogonality to working
// precision for well-conditioned V. All steps are deterministic (fixed-order sums).
#include <math.h>

#include <algorithm>

#include "internal.h"

namespace bem {
namespace {

// In-place Cholesky of the Hermitian nu x nu matrix G (column-major, upper triangle used):
// on exit the upper triangle holds R with G = R^H R, the strict lower triangle is zero.
// A pivot below 1e-13 of the largest diagonal entry of G counts as loss of rank. One block;
// G is staged in shared memory when the dynamic allocation holds it (nu <= 64).
// With `deficient` non-null, a collapsed pivot does not fail: its column of R becomes the
// unit vector (the column of V is then replaced by the caller) and deficient[k] = 1.
__global__ void __launch_bounds__(1024) cholesky_kernel(double2* Gg, int nu, int* status,
                                                        int* deficient, const int* gate) {
  if (gate && *gate == 0) return;   // gated pass not needed
  extern __shared__ double2 sG[];
  __shared__ double rkk, dmax;
  const bool staged = nu <= 64;
  double2* G = staged ? sG : Gg;
  const int tid = threadIdx.x;
  if (staged)
    for (int t = tid; t < nu * nu; t += blockDim.x) sG[t] = Gg[t];
  __syncthreads();
  if (tid == 0) {
    dmax = 0.0;
    for (int k = 0; k < nu; ++k) dmax = fmax(dmax, G[(int64_t)k * nu + k].x);
  }
  __syncthreads();
  bool failed = false;
  for (int k = 0; k < nu; ++k) {
    if (tid == 0) {
      const double d = G[(int64_t)k * nu + k].x;
      if (!(d > 1e-13 * dmax) || !isfinite(d)) {
        if (deficient) {
          deficient[k] = 1;
          rkk = -1.0;   // marker: unit column, no trailing update
        } else {
          atomicOr(status, kStatusNotSPD);
          rkk = 0.0;
        }
      } else {
        if (deficient) deficient[k] = 0;
        rkk = sqrt(d);
      }
      G[(int64_t)k * nu + k] = make_double2(rkk < 0.0 ? 1.0 : rkk, 0.0);
    }
    __syncthreads();
    if (rkk == 0.0) {
      failed = true;
      break;
    }
    if (rkk < 0.0) {
      for (int jj = k + 1 + tid; jj < nu; jj += blockDim.x)
        G[(int64_t)jj * nu + k] = make_double2(0.0, 0.0);
      __syncthreads();
      continue;
    }
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
    const double2 v = (i > jj) ? make_double2(0.0, 0.0) : G[t];
    Gg[t] = failed ? make_double2(NAN, NAN) : v;
  }
}

// Columns flagged deficient get fresh pseudo-random entries (SplitMix64 of seed, index).
__global__ void refresh_columns_kernel(double2* V, int64_t ldv, int64_t n, int nu,
                                       const int* deficient, uint64_t seed) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * nu) return;
  const int c = (int)(t / n);
  if (!deficient[c]) return;
  const int64_t r = t % n;
  uint64_t a = seed + (2 * (uint64_t)t + 1) * 0x9E3779B97F4A7C15ull;
  uint64_t b = seed + (2 * (uint64_t)t + 2) * 0x9E3779B97F4A7C15ull;
  a = (a ^ (a >> 30)) * 0xBF58476D1CE4E5B9ull; a = (a ^ (a >> 27)) * 0x94D049BB133111EBull; a ^= a >> 31;
  b = (b ^ (b >> 30)) * 0xBF58476D1CE4E5B9ull; b = (b ^ (b >> 27)) * 0x94D049BB133111EBull; b ^= b >> 31;
  V[(int64_t)c * ldv + r] = make_double2((double)(a >> 11) * 0x1.0p-52 - 1.0,
                                         (double)(b >> 11) * 0x1.0p-52 - 1.0);
}

constexpr int kGT = 32;   // Gram output tile

// Partial Gram matrices: block (tile, r) sums conj(V[i][a]) V[i][b] over its row range.
__global__ void __launch_bounds__(256)
gram_partial_kernel(const double2* __restrict__ V, int64_t ldv, int64_t n, int nu,
                    int64_t rows_per_part, double2* __restrict__ part, const int* gate) {
  if (gate && *gate == 0) return;
  __shared__ double2 sX[kGT][kGT + 1];
  __shared__ double2 sY[kGT][kGT + 1];
  const int tiles_a = (nu + kGT - 1) / kGT;
  const int ta = blockIdx.x % tiles_a, tb = blockIdx.x / tiles_a;
  const int64_t r_begin = (int64_t)blockIdx.y * rows_per_part;
  const int64_t r_end = min(n, r_begin + rows_per_part);
  const int tid = threadIdx.x;
  const int oa = tid % kGT, ob0 = tid / kGT;
  double2 acc[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) acc[m] = make_double2(0.0, 0.0);
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kGT) {
    __syncthreads();
    for (int x = tid; x < kGT * kGT; x += 256) {
      const int rr = x % kGT, cc = x / kGT;
      const int64_t r = r0 + rr;
      const int a = ta * kGT + cc, b = tb * kGT + cc;
      sX[rr][cc] = (r < r_end && a < nu) ? V[(int64_t)a * ldv + r] : make_double2(0.0, 0.0);
      sY[rr][cc] = (r < r_end && b < nu) ? V[(int64_t)b * ldv + r] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < kGT; ++rr) {
      const double2 x = sX[rr][oa];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const double2 y = sY[rr][ob0 + 8 * m];
        acc[m].x = fma(x.x, y.x, fma(x.y, y.y, acc[m].x));
        acc[m].y = fma(x.x, y.y, fma(-x.y, y.x, acc[m].y));
      }
    }
  }
  const int a = ta * kGT + oa;
  if (a < nu) {
    double2* P = part + (int64_t)blockIdx.y * nu * nu;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int b = tb * kGT + ob0 + 8 * m;
      if (b < nu) P[(int64_t)b * nu + a] = acc[m];
    }
  }
}

// G = sum of the partials in part order (deterministic).
__global__ void sum_parts_kernel(const double2* __restrict__ part, int parts, int64_t count,
                                 double2* __restrict__ G, const int* gate) {
  if (gate && *gate == 0) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  double2 s = make_double2(0.0, 0.0);
  for (int r = 0; r < parts; ++r) {
    const double2 v = part[(int64_t)r * count + t];
    s.x += v.x;
    s.y += v.y;
  }
  G[t] = s;
}

// Rinv = R^{-1} for upper-triangular R: one block per column j, back substitution
// x_i = (delta_ij - sum_{m=i+1..j} R_im x_m) / R_ii for i = j..0, each sum split over the
// block's threads and combined in a fixed order (deterministic). The column lives in
// shared memory; R is read through the cache.
__global__ void __launch_bounds__(128)
triangular_inverse_kernel(const double2* __restrict__ R, int nu, double2* __restrict__ Rinv,
                          const int* gate) {
  if (gate && *gate == 0) return;
  __shared__ double2 x[kMaxNu];
  __shared__ double2 red[4];
  const int j = blockIdx.x;
  const int tid = threadIdx.x, lane = tid % 32, w = tid / 32;
  for (int i = tid; i < nu; i += blockDim.x) x[i] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int i = j; i >= 0; --i) {
    double2 acc = make_double2(0.0, 0.0);
    for (int m = i + 1 + tid; m <= j; m += blockDim.x) {
      const double2 r = R[(int64_t)m * nu + i];
      const double2 xm = x[m];
      acc.x += r.x * xm.x - r.y * xm.y;
      acc.y += r.x * xm.y + r.y * xm.x;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    if (lane == 0) red[w] = acc;
    __syncthreads();
    if (tid == 0) {
      double2 s = make_double2(i == j ? 1.0 : 0.0, 0.0);
      for (int k = 0; k < 4; ++k) {
        s.x -= red[k].x;
        s.y -= red[k].y;
      }
      const double d = R[(int64_t)i * nu + i].x;   // real positive
      x[i] = make_double2(s.x / d, s.y / d);
    }
    __syncthreads();
  }
  for (int i = tid; i < nu; i += blockDim.x) Rinv[(int64_t)j * nu + i] = x[i];
}

constexpr int kRows = 8;

// V <- V * M in place, M nu x nu upper triangular (column-major); each block owns kRows
// rows of V.
// gate: skip unless *gate == 1; skip_if: skip when *skip_if != 0
__global__ void __launch_bounds__(256)
right_multiply_kernel(double2* V, int64_t ldv, int64_t n, int nu, const double2* __restrict__ M,
                      const int* gate, const int* skip_if) {
  if ((gate && *gate == 0) || (skip_if && *skip_if != 0)) return;
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
    for (int k = 0; k <= c; ++k) {
      const double2 a = sV[rr][k];
      const double2 b = M[(int64_t)c * nu + k];
      acc.x += a.x * b.x - a.y * b.y;
      acc.y += a.x * b.y + a.y * b.x;
    }
    if (r < n) V[(int64_t)c * ldv + r] = acc;
  }
}

// ---- FP32 first pass (nu <= 128): Gram, Cholesky and triangular inverse in FP32 ----

__global__ void __launch_bounds__(256)
gram_partial32_kernel(const double2* __restrict__ V, int64_t ldv, int64_t n, int nu,
                      int64_t rows_per_part, double2* __restrict__ part) {
  __shared__ float2 sX[kGT][kGT + 1];
  __shared__ float2 sY[kGT][kGT + 1];
  const int tiles_a = (nu + kGT - 1) / kGT;
  const int ta = blockIdx.x % tiles_a, tb = blockIdx.x / tiles_a;
  const int64_t r_begin = (int64_t)blockIdx.y * rows_per_part;
  const int64_t r_end = min(n, r_begin + rows_per_part);
  const int tid = threadIdx.x;
  const int oa = tid % kGT, ob0 = tid / kGT;
  float2 acc[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) acc[m] = make_float2(0.f, 0.f);
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kGT) {
    __syncthreads();
    for (int x = tid; x < kGT * kGT; x += 256) {
      const int rr = x % kGT, cc = x / kGT;
      const int64_t r = r0 + rr;
      const int a = ta * kGT + cc, b = tb * kGT + cc;
      double2 va = make_double2(0.0, 0.0), vb = va;
      if (r < r_end && a < nu) va = V[(int64_t)a * ldv + r];
      if (r < r_end && b < nu) vb = V[(int64_t)b * ldv + r];
      sX[rr][cc] = make_float2((float)va.x, (float)va.y);
      sY[rr][cc] = make_float2((float)vb.x, (float)vb.y);
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < kGT; ++rr) {
      const float2 x = sX[rr][oa];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float2 y = sY[rr][ob0 + 8 * m];
        acc[m].x = fmaf(x.x, y.x, fmaf(x.y, y.y, acc[m].x));
        acc[m].y = fmaf(x.x, y.y, fmaf(-x.y, y.x, acc[m].y));
      }
    }
  }
  const int a = ta * kGT + oa;
  if (a < nu) {
    double2* P = part + (int64_t)blockIdx.y * nu * nu;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int b = tb * kGT + ob0 + 8 * m;
      if (b < nu) P[(int64_t)b * nu + a] = make_double2(acc[m].x, acc[m].y);
    }
  }
}

// FP32 Cholesky in shared memory (nu <= 128); output R (upper, as double2), lower zeroed.
// A pivot below 1e-6 of the largest diagonal entry (V too ill-conditioned for an FP32
// first pass) sets *fallback: the pass then leaves V alone and an FP64 pass is added.
__global__ void __launch_bounds__(1024) cholesky32_kernel(double2* Gg, int nu, int* fallback) {
  extern __shared__ float2 sG32[];
  __shared__ float rkk, dmax;
  const int tid = threadIdx.x;
  for (int t = tid; t < nu * nu; t += blockDim.x) sG32[t] = make_float2((float)Gg[t].x, (float)Gg[t].y);
  __syncthreads();
  if (tid == 0) {
    dmax = 0.f;
    for (int k = 0; k < nu; ++k) dmax = fmaxf(dmax, sG32[k * nu + k].x);
  }
  __syncthreads();
  bool failed = false;
  for (int k = 0; k < nu; ++k) {
    if (tid == 0) {
      const float d = sG32[k * nu + k].x;
      if (!(d > 1e-6f * dmax) || !isfinite(d)) {
        *fallback = 1;
        rkk = 0.f;
      } else {
        rkk = sqrtf(d);
      }
      sG32[k * nu + k] = make_float2(rkk, 0.f);
    }
    __syncthreads();
    if (rkk == 0.f) {
      failed = true;
      break;
    }
    for (int jj = k + 1 + tid; jj < nu; jj += blockDim.x) {
      const float2 g = sG32[jj * nu + k];
      sG32[jj * nu + k] = make_float2(g.x / rkk, g.y / rkk);
    }
    __syncthreads();
    const int m = nu - k - 1;
    for (int t = tid; t < m * m; t += blockDim.x) {
      const int i = k + 1 + t % m, jj = k + 1 + t / m;
      if (i > jj) continue;
      const float2 a = sG32[i * nu + k], b = sG32[jj * nu + k];
      float2 g = sG32[jj * nu + i];
      g.x -= a.x * b.x + a.y * b.y;
      g.y -= a.x * b.y - a.y * b.x;
      sG32[jj * nu + i] = g;
    }
    __syncthreads();
  }
  for (int t = tid; t < nu * nu; t += blockDim.x) {
    const int i = t % nu, jj = t / nu;
    const float2 v = (i > jj) ? make_float2(0.f, 0.f) : sG32[t];
    Gg[t] = failed ? make_double2(NAN, NAN) : make_double2(v.x, v.y);
  }
}

// FP32 triangular inverse, one block per column (as triangular_inverse_kernel).
__global__ void __launch_bounds__(128)
triangular_inverse32_kernel(const double2* __restrict__ R, int nu, double2* __restrict__ Rinv,
                            const int* skip_if) {
  if (*skip_if != 0) return;
  __shared__ float2 x[kMaxNu];
  __shared__ float2 red[4];
  const int j = blockIdx.x;
  const int tid = threadIdx.x, lane = tid % 32, w = tid / 32;
  for (int i = tid; i < nu; i += blockDim.x) x[i] = make_float2(0.f, 0.f);
  __syncthreads();
  for (int i = j; i >= 0; --i) {
    float2 acc = make_float2(0.f, 0.f);
    for (int m = i + 1 + tid; m <= j; m += blockDim.x) {
      const double2 rd = R[(int64_t)m * nu + i];
      const float2 r = make_float2((float)rd.x, (float)rd.y);
      const float2 xm = x[m];
      acc.x += r.x * xm.x - r.y * xm.y;
      acc.y += r.x * xm.y + r.y * xm.x;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    if (lane == 0) red[w] = acc;
    __syncthreads();
    if (tid == 0) {
      float2 sum = make_float2(i == j ? 1.f : 0.f, 0.f);
      for (int k = 0; k < 4; ++k) {
        sum.x -= red[k].x;
        sum.y -= red[k].y;
      }
      const float d = (float)R[(int64_t)i * nu + i].x;
      x[i] = make_float2(sum.x / d, sum.y / d);
    }
    __syncthreads();
  }
  for (int i = tid; i < nu; i += blockDim.x) Rinv[(int64_t)j * nu + i] = make_double2(x[i].x, x[i].y);
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

size_t cholqr2_work_bytes(bem_ctx* ctx, int64_t n, int nu) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  const int tiles = ((nu + kGT - 1) / kGT) * ((nu + kGT - 1) / kGT);
  int64_t parts = std::max<int64_t>(1, std::min<int64_t>((n + 63) / 64,
                                                         (2 * (int64_t)sms + tiles - 1) / tiles));
  const int64_t rows_per_part = (n + parts - 1) / parts;
  parts = (n + rows_per_part - 1) / rows_per_part;
  return (4 + (size_t)parts) * (size_t)nu * nu * sizeof(double2) + 257 * sizeof(int);
}

// CholeskyQR2 of V (n x nu, ld ldv) with caller-provided work (cholqr2_work_bytes);
// asynchronous; a Gram matrix that is not positive definite is flagged in the context's
// status word.
bem_status cholqr2_impl(bem_ctx* ctx, double* V_dev, int64_t n, int64_t ldv, int nu,
                        double* R_dev, void* work, cudaStream_t s, uint64_t refresh_seed) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  const int tiles = ((nu + kGT - 1) / kGT) * ((nu + kGT - 1) / kGT);
  int64_t parts = std::max<int64_t>(1, std::min<int64_t>((n + 63) / 64,
                                                         (2 * (int64_t)sms + tiles - 1) / tiles));
  const int64_t rows_per_part = (n + parts - 1) / parts;
  parts = (n + rows_per_part - 1) / rows_per_part;
  double2* G = reinterpret_cast<double2*>(work);
  double2* Rinv = G + (size_t)nu * nu;
  double2* R1 = Rinv + (size_t)nu * nu;
  double2* R2 = R1 + (size_t)nu * nu;
  double2* part = R2 + (size_t)nu * nu;
  int* deficient = reinterpret_cast<int*>(part + (size_t)parts * nu * nu);
  bem_status st = BEM_OK;
  const size_t chol_smem = nu <= 64 ? (size_t)nu * nu * sizeof(double2) : 0;
  if (chol_smem > 48 * 1024) {
    st = cuda_check(ctx, cudaFuncSetAttribute(cholesky_kernel,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)chol_smem),
                    "cholqr attribute");
    if (st != BEM_OK) return st;
  }
  // first pass in FP32 when its factor is not needed: it only has to make V well
  // conditioned; the FP64 second pass sets the final orthogonality. If V is too ill-
  // conditioned for FP32 the FP32 pass leaves V alone (device flag) and a third, FP64,
  // pass runs in its place (its kernels return at once otherwise).
  const bool fp32_first = R_dev == nullptr && refresh_seed == 0 && nu <= 128;
  int* fallback = deficient + 256;
  if (fp32_first) {
    st = cuda_check(ctx, cudaFuncSetAttribute(cholesky32_kernel,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)(nu * nu * sizeof(float2))),
                    "cholqr attribute");
    if (st != BEM_OK) return st;
    st = cuda_check(ctx, cudaMemsetAsync(fallback, 0, sizeof(int), s), "cholqr flag");
    if (st != BEM_OK) return st;
  }
  const int passes = fp32_first ? 3 : 2;
  for (int pass = 0; pass < passes; ++pass) {
    // FP32 pass (fp32_first, pass 0); FP64 passes; the third pass only if flagged
    double2* R = pass == 0 ? R1 : R2;
    const bool low = fp32_first && pass == 0;
    const int* gate = (fp32_first && pass == 2) ? fallback : nullptr;
    const dim3 ggrid((unsigned)tiles, (unsigned)parts);
    if (low)
      gram_partial32_kernel<<<ggrid, 256, 0, s>>>(reinterpret_cast<const double2*>(V_dev), ldv, n,
                                                  nu, rows_per_part, part);
    else
      gram_partial_kernel<<<ggrid, 256, 0, s>>>(reinterpret_cast<const double2*>(V_dev), ldv, n,
                                                nu, rows_per_part, part, gate);
    sum_parts_kernel<<<(unsigned)(((int64_t)nu * nu + 255) / 256), 256, 0, s>>>(
        part, (int)parts, (int64_t)nu * nu, R, gate);
    const bool refresh = refresh_seed != 0 && pass == 0;
    if (low) {
      cholesky32_kernel<<<1, 1024, nu * nu * sizeof(float2), s>>>(R, nu, fallback);
      triangular_inverse32_kernel<<<nu, 128, 0, s>>>(R, nu, Rinv, fallback);
    } else {
      cholesky_kernel<<<1, 1024, chol_smem, s>>>(R, nu, ctx->d_status,
                                                 refresh ? deficient : nullptr, gate);
      triangular_inverse_kernel<<<nu, 128, 0, s>>>(R, nu, Rinv, gate);
    }
    right_multiply_kernel<<<(unsigned)((n + kRows - 1) / kRows), 256, 0, s>>>(
        reinterpret_cast<double2*>(V_dev), ldv, n, nu, Rinv, gate, low ? fallback : nullptr);
    ctx->launches += 5;
    if (refresh) {
      refresh_columns_kernel<<<(unsigned)((n * nu + 255) / 256), 256, 0, s>>>(
          reinterpret_cast<double2*>(V_dev), ldv, n, nu, deficient, refresh_seed);
      ctx->launches++;
    }
    st = cuda_check(ctx, cudaGetLastError(), "cholqr kernels");
    if (st != BEM_OK) return st;
  }
  if (R_dev) {
    upper_product_kernel<<<1, 256, 0, s>>>(R2, R1, nu, reinterpret_cast<double2*>(R_dev));
    ctx->launches++;
    st = cuda_check(ctx, cudaGetLastError(), "cholqr kernels");
  }
  (void)G;
  return st;
}

}  // namespace bem

using namespace bem;

extern "C" bem_status bem_cholqr2(bem_ctx* ctx, double* V_dev, int64_t n, int64_t ldv, int nu,
                                  double* R_dev, void* stream) {
  if (!ctx) return BEM_EINVAL;
  if (!V_dev || n < 1 || nu < 1 || nu > kMaxNu || ldv < n || nu > n)
    return fail(ctx, BEM_EINVAL, "bem_cholqr2: need V, 1 <= nu <= min(n, 256), ldv >= n");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  bem_status st = ensure_small(ctx, cholqr2_work_bytes(ctx, n, nu));
  if (st != BEM_OK) return st;
  st = cholqr2_impl(ctx, V_dev, n, ldv, nu, R_dev, ctx->d_small, s, 0);
  if (st != BEM_OK) return st;
  return take_status(ctx, s, "bem_cholqr2");
}
