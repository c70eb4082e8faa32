// The reduced linearised eigenproblem (Section 3.1) and the Ritz vectors.
//
// With B^_j the weighted projected matrices (bem_project), the reduced Cauchy problem
// sum_j B^_j y / (lambda - z_j) = 0 is linearised (Eq. EVP_red, Eq. sc1_cauchy_red) as
// A w = lambda M w, w = [v_0; ..; v_{N-1}; y], v_j = y / (lambda - z_j). Shift-and-invert
// about s (Eq. sc2) turns it into H w = mu w, mu = 1 / (lambda - s),
// H = (A - s M)^{-1} M, applied through the Schur complement of the block system
// (Eq. sc3 - sc5): with C_j = B^_j / (z_j - s) and S = sum_j C_j,
//     u' = S^{-1} sum_j C_j v_j,   v_j' = (v_j - u') / (z_j - s).
// The eigenvalues nearest the contour's centre are the dominant mu, so a block of p
// vectors is iterated with H (subspace iteration, the paper's suggestion for the reduced
// problem when dense methods are too costly), orthonormalised by CholeskyQR2 after every
// application, and a Rayleigh-Ritz step W^H H W = Z diag(mu) Z^-1 (small dense
// eigensolver, small_eig.h) gives the eigenvalues lambda = s + 1/mu and the y-parts of
// the eigenvectors, y = S^{-1} C (W z) / mu.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "small_eig.h"

namespace bem {
namespace {

__device__ __forceinline__ double2 zmul_(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zdiv_(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// C_j = Bhat_j / (z_j - s) for all j, and S = sum_j C_j (fixed order).
__global__ void reduced_setup_kernel(const double2* __restrict__ Bhat, const double2* __restrict__ z,
                                     double2 shift, int N, int nu, double2* __restrict__ C,
                                     double2* __restrict__ S) {
  const int64_t per = (int64_t)nu * nu;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= per) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int j = 0; j < N; ++j) {
    const double2 d = make_double2(z[j].x - shift.x, z[j].y - shift.y);
    const double2 c = zdiv_(Bhat[(int64_t)j * per + t], d);
    C[(int64_t)j * per + t] = c;
    acc.x += c.x;
    acc.y += c.y;
  }
  S[t] = acc;
}

// Minv = M^{-1} by Gauss-Jordan elimination with partial pivoting (one block, nu <= 256;
// M is destroyed). A zero pivot flags the status word.
__global__ void __launch_bounds__(1024) gauss_jordan_kernel(double2* M, double2* Minv, int nu,
                                                            int* status) {
  __shared__ int piv;
  __shared__ double best[32];
  __shared__ int besti[32];
  const int tid = threadIdx.x;
  for (int64_t t = tid; t < (int64_t)nu * nu; t += blockDim.x)
    Minv[t] = make_double2((t % nu) == (t / nu) ? 1.0 : 0.0, 0.0);
  __syncthreads();
  for (int c = 0; c < nu; ++c) {
    // pivot: largest |M(r, c)|, r >= c (ties: smallest r)
    double bv = -1.0;
    int bi = c;
    for (int r = c + tid; r < nu; r += blockDim.x) {
      const double2 v = M[(int64_t)c * nu + r];
      const double a = v.x * v.x + v.y * v.y;
      if (a > bv) { bv = a; bi = r; }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, bv, off);
      const int oi = __shfl_down_sync(0xffffffffu, bi, off);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (tid % 32 == 0) { best[tid / 32] = bv; besti[tid / 32] = bi; }
    __syncthreads();
    if (tid == 0) {
      double b = -1.0;
      int bi2 = c;
      for (int w = 0; w < (int)((blockDim.x + 31) / 32); ++w)
        if (best[w] > b || (best[w] == b && besti[w] < bi2)) { b = best[w]; bi2 = besti[w]; }
      piv = bi2;
      if (!(b > 0.0)) atomicOr(status, kStatusNotSPD);
    }
    __syncthreads();
    const int r = piv;
    if (r != c)
      for (int k = tid; k < nu; k += blockDim.x) {
        double2 a = M[(int64_t)k * nu + c], b = M[(int64_t)k * nu + r];
        M[(int64_t)k * nu + c] = b; M[(int64_t)k * nu + r] = a;
        a = Minv[(int64_t)k * nu + c]; b = Minv[(int64_t)k * nu + r];
        Minv[(int64_t)k * nu + c] = b; Minv[(int64_t)k * nu + r] = a;
      }
    __syncthreads();
    const double2 pv = M[(int64_t)c * nu + c];
    const double2 inv = zdiv_(make_double2(1.0, 0.0), pv);
    __syncthreads();
    for (int k = tid; k < nu; k += blockDim.x) {
      M[(int64_t)k * nu + c] = zmul_(M[(int64_t)k * nu + c], inv);
      Minv[(int64_t)k * nu + c] = zmul_(Minv[(int64_t)k * nu + c], inv);
    }
    __syncthreads();
    // eliminate column c from every other row: row_i -= M(i, c) row_c
    for (int64_t t = tid; t < (int64_t)nu * 2 * nu; t += blockDim.x) {
      const int i = (int)(t % nu);
      const int k = (int)(t / nu);   // 0 .. 2nu-1: columns of [M | Minv]
      if (i == c) continue;
      const double2 f = M[(int64_t)c * nu + i];
      if (k < nu) {
        if (k == c) continue;   // column c itself is cleared below
        const double2 rc = M[(int64_t)k * nu + c];
        double2 v = M[(int64_t)k * nu + i];
        const double2 pr = zmul_(f, rc);
        M[(int64_t)k * nu + i] = make_double2(v.x - pr.x, v.y - pr.y);
      } else {
        const int kk = k - nu;
        const double2 rc = Minv[(int64_t)kk * nu + c];
        double2 v = Minv[(int64_t)kk * nu + i];
        const double2 pr = zmul_(f, rc);
        Minv[(int64_t)kk * nu + i] = make_double2(v.x - pr.x, v.y - pr.y);
      }
    }
    __syncthreads();
    for (int i = tid; i < nu; i += blockDim.x)
      if (i != c) M[(int64_t)c * nu + i] = make_double2(0.0, 0.0);
    __syncthreads();
  }
}

constexpr int kZT = 32;
// C = A B (complex FP64): A m x k (lda), B k x n (ldb), C m x n (ldc); 32 x 32 tiles,
// fixed-order sums.
// With gridDim.z > 1 block z sums the k-range [z kc, (z + 1) kc) and writes its partial
// product at C + z * ldc * n (the caller sums the partials in z order).
__global__ void __launch_bounds__(256)
zgemm_kernel(int m, int n, int k, const double2* __restrict__ A, int64_t lda,
             const double2* __restrict__ B, int64_t ldb, double2* __restrict__ C, int64_t ldc,
             int kc) {
  __shared__ double2 sA[kZT][kZT + 1];
  __shared__ double2 sB[kZT][kZT + 1];
  const int i0 = blockIdx.x * kZT, j0 = blockIdx.y * kZT;
  const int ti = threadIdx.x % kZT, tj0 = threadIdx.x / kZT;   // rows ti, columns tj0 + 8 q
  double2 acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] = make_double2(0.0, 0.0);
  const int kb = blockIdx.z * kc, ke = min(k, kb + kc);
  C += (int64_t)blockIdx.z * ldc * n;
  for (int k0 = kb; k0 < ke; k0 += kZT) {
    __syncthreads();
    for (int t = threadIdx.x; t < kZT * kZT; t += 256) {
      const int r = t % kZT, c = t / kZT;
      sA[r][c] = (i0 + r < m && k0 + c < ke) ? A[(int64_t)(k0 + c) * lda + i0 + r] : make_double2(0.0, 0.0);
      sB[r][c] = (k0 + r < ke && j0 + c < n) ? B[(int64_t)(j0 + c) * ldb + k0 + r] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kZT; ++kk) {
      const double2 a = sA[ti][kk];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double2 b = sB[kk][tj0 + 8 * q];
        acc[q].x = fma(a.x, b.x, fma(-a.y, b.y, acc[q].x));
        acc[q].y = fma(a.x, b.y, fma(a.y, b.x, acc[q].y));
      }
    }
  }
  if (i0 + ti < m)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + tj0 + 8 * q;
      if (j < n) C[(int64_t)j * ldc + i0 + ti] = acc[q];
    }
}

// HW_j = (W_j - U) / (z_j - s): W, HW (N nu) x p with ld N nu, U nu x p.
__global__ void reduced_update_kernel(const double2* __restrict__ W, const double2* __restrict__ U,
                                      const double2* __restrict__ z, double2 shift, int N, int nu,
                                      int p, double2* __restrict__ HW) {
  const int64_t rows = (int64_t)N * nu;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= rows * p) return;
  const int64_t r = t % rows;
  const int c = (int)(t / rows);
  const int j = (int)(r / nu), k = (int)(r % nu);
  const double2 w = W[t], u = U[(int64_t)c * nu + k];
  const double2 d = make_double2(z[j].x - shift.x, z[j].y - shift.y);
  HW[t] = zdiv_(make_double2(w.x - u.x, w.y - u.y), d);
}

// Deterministic pseudo-random start block: SplitMix64 of (seed, index), uniform in [-1, 1).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__global__ void random_block_kernel(double2* W, int64_t count, uint64_t seed) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const uint64_t a = mix64(seed + (2 * (uint64_t)t + 1) * 0x9E3779B97F4A7C15ull);
  const uint64_t b = mix64(seed + (2 * (uint64_t)t + 2) * 0x9E3779B97F4A7C15ull);
  W[t] = make_double2((double)(a >> 11) * 0x1.0p-52 - 1.0, (double)(b >> 11) * 0x1.0p-52 - 1.0);
}

// Y(:, i) *= 1 / mu_i
__global__ void scale_columns_kernel(double2* Y, int64_t rows, int cols, const double2* mu) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= rows * cols) return;
  const int c = (int)(t / rows);
  Y[t] = zdiv_(Y[t], mu[c]);
}

// Reduced residuals ||sum_j B^_j y_i / (lambda_i - z_j)|| / (||y_i|| sum_j ||B^_j||_1 /
// |lambda_i - z_j|), one block per column i (fixed-order sums).
// bnorm[j] = max column sum of |B^_j| (the size of B^_j in the residual's scale), one block
// per node, fixed-order sums
__global__ void bnorm_kernel(const double2* __restrict__ Bhat, int nu, double* __restrict__ bnorm) {
  __shared__ double red[256];
  const double2* B = Bhat + (int64_t)blockIdx.x * nu * nu;
  double mx = 0.0;
  for (int k = threadIdx.x; k < nu; k += blockDim.x) {
    double cs = 0.0;
    for (int a = 0; a < nu; ++a) cs += hypot(B[(int64_t)k * nu + a].x, B[(int64_t)k * nu + a].y);
    mx = fmax(mx, cs);
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) bnorm[blockIdx.x] = red[0];
}

// ||sum_j B^_j y / (lambda - z_j)|| / (||y|| sum_j ||B^_j|| / |lambda - z_j|) per Ritz pair,
// one block per pair; bnorm from bnorm_kernel.
__global__ void reduced_residual_kernel(const double2* __restrict__ Bhat, const double2* __restrict__ z,
                                        const double2* __restrict__ lam, const double2* __restrict__ Y,
                                        int N, int nu, const double* __restrict__ bnorm,
                                        double* __restrict__ res) {
  __shared__ double red[256], ry[256];
  const int i = blockIdx.x;
  const double2 l = lam[i];
  const double2* y = Y + (int64_t)i * nu;
  double part = 0.0, yn = 0.0;
  for (int a = threadIdx.x; a < nu; a += blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int j = 0; j < N; ++j) {
      double2 s = make_double2(0.0, 0.0);
      const double2* B = Bhat + (int64_t)j * nu * nu;
      for (int k = 0; k < nu; ++k) {
        const double2 pr = zmul_(B[(int64_t)k * nu + a], y[k]);
        s.x += pr.x;
        s.y += pr.y;
      }
      const double2 q = zdiv_(s, make_double2(l.x - z[j].x, l.y - z[j].y));
      acc.x += q.x;
      acc.y += q.y;
    }
    part += acc.x * acc.x + acc.y * acc.y;
    yn += y[a].x * y[a].x + y[a].y * y[a].y;
  }
  red[threadIdx.x] = part;
  ry[threadIdx.x] = yn;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      red[threadIdx.x] += red[threadIdx.x + w];
      ry[threadIdx.x] += ry[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double den = 0.0;
    for (int j = 0; j < N; ++j) den += bnorm[j] / hypot(l.x - z[j].x, l.y - z[j].y);
    const double sden = den * sqrt(ry[0]);
    res[i] = sden > 0.0 ? sqrt(red[0]) / sden : INFINITY;
  }
}

__global__ void small_eig_kernel(int m, double2* A, double2* w, double2* V, double2* Z,
                                 int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int rc = small::eig(m, reinterpret_cast<small::zc*>(A), reinterpret_cast<small::zc*>(w),
                            reinterpret_cast<small::zc*>(V), reinterpret_cast<small::zc*>(Z));
  if (rc != 0) atomicOr(status, kStatusNonFinite);
}

// ---- Chebyshev variant (Eq. Chebyshev, Eq. sc1_chebyshev_red, Algorithm 2's setting) ----
//
// With projected samples P_k = V^H T(x_k) V at the Chebyshev points of [c - a, c + a], the
// reduced interpolant is sum_i B^_i T_i(zeta), zeta = (z - c) / a, and its colleague
// linearisation A w = zeta M w, w = [v_0; ..; v_{m-1}], v_i = T_i(zeta) y. Shift-and-invert
// about sigma (zeta units): (A - sigma M) w' = M w is solved by the three-term recurrence
// of the first m - 1 block rows, v'_i = e_i + T_i(sigma) u with e_0 = 0, e_1 = y_0,
// e_{i+1} = y_i - e_{i-1} + 2 sigma e_i (y = M w), and the last block row, which leaves the
// nu x nu system G u = b, G = sum_i T_i(sigma) L_i, b = y_{m-1} - sum_i L_i e_i, where
// L_i = -B^_i (i <= m-3), L_{m-2} = B^_m - B^_{m-2}, L_{m-1} = -B^_{m-1} - 2 sigma B^_m.
// (Algorithm 2 is this solve at sigma = 0.)

// table[i N + k] = (2 - delta_i0) / N cos(i pi (k + 1/2) / N)
__global__ void cheb_table_kernel(int N, double* table) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * N) return;
  const int i = t / N, k = t % N;
  table[t] = (i == 0 ? 1.0 : 2.0) / N * cospi((double)i * (k + 0.5) / N);
}

// B_i = sum_k table[i N + k] P_k (fixed order), P_k and B_i nu x nu.
__global__ void cheb_coeff_kernel(const double2* __restrict__ P, const double* __restrict__ table,
                                  int N, int64_t nn, double2* __restrict__ B) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)N * nn) return;
  const int i = (int)(t / nn);
  const int64_t e = t % nn;
  double2 acc = make_double2(0.0, 0.0);
  for (int k = 0; k < N; ++k) {
    const double c = table[i * N + k];
    const double2 p = P[(int64_t)k * nn + e];
    acc.x += c * p.x;
    acc.y += c * p.y;
  }
  B[t] = acc;
}

// L = [L_0 .. L_{m-1}] (nu x m nu, ld nu) and G = sum_i s_i L_i, s_i = T_i(sigma).
__global__ void cheb_setup_kernel(const double2* __restrict__ B, int m, int nu, double2 sigma,
                                  const double2* __restrict__ sT, double2* __restrict__ L,
                                  double2* __restrict__ G) {
  const int64_t nn = (int64_t)nu * nu;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nn) return;
  double2 g = make_double2(0.0, 0.0);
  for (int i = 0; i < m; ++i) {
    double2 l;
    if (i <= m - 3) {
      l = make_double2(-B[i * nn + e].x, -B[i * nn + e].y);
    } else if (i == m - 2) {
      l = make_double2(B[m * nn + e].x - B[(m - 2) * nn + e].x, B[m * nn + e].y - B[(m - 2) * nn + e].y);
    } else {
      const double2 bm = zmul_(make_double2(2.0 * sigma.x, 2.0 * sigma.y), B[m * nn + e]);
      l = make_double2(-B[(m - 1) * nn + e].x - bm.x, -B[(m - 1) * nn + e].y - bm.y);
    }
    L[i * nn + e] = l;
    const double2 sl = zmul_(sT[i], l);
    g.x += sl.x;
    g.y += sl.y;
  }
  G[e] = g;
}

// E = the u-independent parts e_0..e_{m-1} of the solve, from W (y = M W on the fly; the
// last block row is handled separately). One thread per (row of a block, column).
__global__ void cheb_recur_kernel(const double2* __restrict__ W, int m, int nu, int p,
                                  double2 sigma, double2* __restrict__ E) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nu * p) return;
  const int r = (int)(t % nu), c = (int)(t / nu);
  const int64_t ld = (int64_t)m * nu;
  const double2* w = W + (int64_t)c * ld + r;
  double2* e = E + (int64_t)c * ld + r;
  double2 em1 = make_double2(0.0, 0.0);     // e_{i-1}
  double2 ei = w[0];                         // e_1 = y_0 = w_0
  e[0] = em1;                                // e_0 = 0
  if (m > 1) e[nu] = ei;
  for (int i = 1; i + 1 < m; ++i) {
    const double2 yi = make_double2(2.0 * w[(int64_t)i * nu].x, 2.0 * w[(int64_t)i * nu].y);
    const double2 se = zmul_(make_double2(2.0 * sigma.x, 2.0 * sigma.y), ei);
    const double2 en = make_double2(yi.x - em1.x + se.x, yi.y - em1.y + se.y);
    e[(int64_t)(i + 1) * nu] = en;
    em1 = ei;
    ei = en;
  }
}

// HW_i = E_i + s_i U, U nu x p; HW and E are (m nu) x p.
__global__ void cheb_combine_kernel(const double2* __restrict__ E, const double2* __restrict__ U,
                                    const double2* __restrict__ sT, int m, int nu, int p,
                                    double2* __restrict__ HW) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t rows = (int64_t)m * nu;
  if (t >= rows * p) return;
  const int64_t r = t % rows;
  const int c = (int)(t / rows);
  const int i = (int)(r / nu), a = (int)(r % nu);
  const double2 su = zmul_(sT[i], U[(int64_t)c * nu + a]);
  HW[t] = make_double2(E[t].x + su.x, E[t].y + su.y);
}

// rhs = y_{m-1} - L E = 2 BW - LE, given BW = B_m w_{m-1} and LE = L E (nu x p each)
__global__ void cheb_rhs_kernel(const double2* __restrict__ BW, const double2* __restrict__ LE,
                                int64_t count, double2* __restrict__ rhs) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  rhs[t] = make_double2(2.0 * BW[t].x - LE[t].x, 2.0 * BW[t].y - LE[t].y);
}

// ||sum_i T_i(zeta) B_i y|| / (||y|| sum_i |T_i(zeta)| ||B_i||_1), one block per Ritz pair;
// zeta[i] in zeta units.
__global__ void cheb_residual_kernel(const double2* __restrict__ B, const double2* __restrict__ zeta,
                                     const double2* __restrict__ Y, int N, int nu,
                                     double* __restrict__ res) {
  __shared__ double red[256];
  const int q = blockIdx.x;
  const double2 zt = zeta[q];
  const double2* y = Y + (int64_t)q * nu;
  const int64_t nn = (int64_t)nu * nu;
  double part = 0.0;
  for (int a = threadIdx.x; a < nu; a += blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    double2 tm1 = make_double2(1.0, 0.0), ti = zt;
    for (int i = 0; i < N; ++i) {
      const double2 T = i == 0 ? tm1 : ti;
      double2 s = make_double2(0.0, 0.0);
      for (int k = 0; k < nu; ++k) {
        const double2 pr = zmul_(B[i * nn + (int64_t)k * nu + a], y[k]);
        s.x += pr.x;
        s.y += pr.y;
      }
      const double2 ts = zmul_(T, s);
      acc.x += ts.x;
      acc.y += ts.y;
      if (i >= 1) {   // advance T_i -> T_{i+1}
        const double2 z2t = zmul_(make_double2(2.0 * zt.x, 2.0 * zt.y), ti);
        const double2 tn = make_double2(z2t.x - tm1.x, z2t.y - tm1.y);
        tm1 = ti;
        ti = tn;
      }
    }
    part += acc.x * acc.x + acc.y * acc.y;
  }
  red[threadIdx.x] = part;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double yn = 0.0, den = 0.0;
    for (int k = 0; k < nu; ++k) yn += y[k].x * y[k].x + y[k].y * y[k].y;
    double2 tm = make_double2(1.0, 0.0), tc = zt;
    for (int i = 0; i < N; ++i) {
      const double2 T = i == 0 ? tm : tc;
      double bmax = 0.0;
      for (int k = 0; k < nu; ++k) {
        double cs = 0.0;
        for (int a = 0; a < nu; ++a) cs += hypot(B[i * nn + (int64_t)k * nu + a].x, B[i * nn + (int64_t)k * nu + a].y);
        bmax = fmax(bmax, cs);
      }
      den += bmax * hypot(T.x, T.y);
      if (i >= 1) {
        const double2 z2t = zmul_(make_double2(2.0 * zt.x, 2.0 * zt.y), tc);
        const double2 tn = make_double2(z2t.x - tm.x, z2t.y - tm.y);
        tm = tc;
        tc = tn;
      }
    }
    const double d = den * sqrt(yn);
    res[q] = d > 0.0 ? sqrt(red[0]) / d : INFINITY;
  }
}

}  // namespace

// C = sum_z P_z (m x n each, packed with leading dimension m), fixed order
__global__ void zsum_parts_kernel(const double2* __restrict__ P, int parts, int m, int n,
                                  double2* __restrict__ C, int64_t ldc) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * n) return;
  const int i = (int)(t % m), j = (int)(t / m);
  double2 acc = make_double2(0.0, 0.0);
  for (int z = 0; z < parts; ++z) {
    const double2 v = P[(int64_t)z * m * n + t];
    acc.x += v.x;
    acc.y += v.y;
  }
  C[(int64_t)j * ldc + i] = acc;
}

cudaError_t launch_zgemm(bem_ctx* ctx, int m, int n, int k, const double* A, int64_t lda,
                         const double* B, int64_t ldb, double* C, int64_t ldc, cudaStream_t s) {
  dim3 grid((unsigned)((m + kZT - 1) / kZT), (unsigned)((n + kZT - 1) / kZT));
  // few output tiles and a long k (the reduced problem's [C_0 .. C_{N-1}] W, k = N nu):
  // split k so that the device fills, partial products summed in a fixed order
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  const int tiles = (int)(grid.x * grid.y);
  int parts = 1;
  if (tiles < 2 * sms && k >= 8 * kZT)
    parts = std::min((2 * sms + tiles - 1) / tiles, k / (4 * kZT));
  if (parts > 1) {
    const int kc = ((k + parts - 1) / parts + kZT - 1) / kZT * kZT;
    parts = (k + kc - 1) / kc;
    const size_t bytes = (size_t)parts * m * n * sizeof(double2);
    if (bytes > ctx->zgemm_bytes) {
      cudaFree(ctx->d_zgemm);
      ctx->d_zgemm = nullptr;
      ctx->zgemm_bytes = 0;
      cudaError_t e = cudaMalloc(&ctx->d_zgemm, bytes);
      if (e != cudaSuccess) return e;
      ctx->zgemm_bytes = bytes;
    }
    grid.z = (unsigned)parts;
    zgemm_kernel<<<grid, 256, 0, s>>>(m, n, k, reinterpret_cast<const double2*>(A), lda,
                                      reinterpret_cast<const double2*>(B), ldb,
                                      reinterpret_cast<double2*>(ctx->d_zgemm), m, kc);
    zsum_parts_kernel<<<(unsigned)(((int64_t)m * n + 255) / 256), 256, 0, s>>>(
        reinterpret_cast<const double2*>(ctx->d_zgemm), parts, m, n,
        reinterpret_cast<double2*>(C), ldc);
    ctx->launches += 2;
    return cudaGetLastError();
  }
  zgemm_kernel<<<grid, 256, 0, s>>>(m, n, k, reinterpret_cast<const double2*>(A), lda,
                                    reinterpret_cast<const double2*>(B), ldb,
                                    reinterpret_cast<double2*>(C), ldc, k);
  ctx->launches++;
  return cudaGetLastError();
}

}  // namespace bem

using namespace bem;

extern "C" bem_status bem_solve_reduced(bem_ctx* ctx, const double* Bhat_dev, int nu,
                                        double shift_re, double shift_im, int p, int max_iter,
                                        double tol, double* lam_host, double* Y_dev,
                                        double* res_host, int* iters_done, void* stream) {
  if (!ctx) return BEM_EINVAL;
  if (ctx->con.N == 0) return fail(ctx, BEM_ESTATE, "bem_solve_reduced: no contour set");
  if (ctx->con.kind == BEM_CONTOUR_CHEBYSHEV)
    return fail(ctx, BEM_ESTATE, "bem_solve_reduced: a Chebyshev interval needs bem_solve_chebyshev");
  const int N = ctx->con.N;
  const int64_t rows = (int64_t)N * nu;
  if (!Bhat_dev || !lam_host || !Y_dev || !res_host || nu < 1 || nu > kMaxNu || p < 1 ||
      p > 256 || p > rows || max_iter < 1 || !(tol > 0.0))
    return fail(ctx, BEM_EINVAL,
                "bem_solve_reduced: need Bhat, outputs, 1 <= nu <= 256, 1 <= p <= min(256, N nu)");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const double2 shift = make_double2(shift_re, shift_im);
  const size_t z2 = sizeof(double2);
  // work layout in the scratch buffer
  const size_t nC = (size_t)N * nu * nu, nS = (size_t)nu * nu, nW = (size_t)rows * p,
               nT = (size_t)nu * p, nG = (size_t)p * p;
  const size_t cq = cholqr2_work_bytes(ctx, rows, p);
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
  const size_t oC = take(nC * z2), oS = take(nS * z2), oSi = take(nS * z2), oW = take(nW * z2),
               oHW = take(nW * z2), oT = take(nT * z2), oU = take(nT * z2), oG = take(nG * z2),
               oZ = take(nG * z2), oVs = take(nG * z2), oMu = take((size_t)p * z2),
               oRes = take((size_t)p * sizeof(double)), oBn = take((size_t)N * sizeof(double)),
               oCq = take(cq);
  bem_status st = ensure_scratch(ctx, off);
  if (st != BEM_OK) return st;
  unsigned char* base = reinterpret_cast<unsigned char*>(ctx->d_scratch);
  double2* C = reinterpret_cast<double2*>(base + oC);
  double2* S = reinterpret_cast<double2*>(base + oS);
  double2* Si = reinterpret_cast<double2*>(base + oSi);
  double2* W = reinterpret_cast<double2*>(base + oW);
  double2* HW = reinterpret_cast<double2*>(base + oHW);
  double2* T = reinterpret_cast<double2*>(base + oT);
  double2* U = reinterpret_cast<double2*>(base + oU);
  double2* G = reinterpret_cast<double2*>(base + oG);
  double2* Zm = reinterpret_cast<double2*>(base + oZ);
  double2* Vs = reinterpret_cast<double2*>(base + oVs);
  double2* mu = reinterpret_cast<double2*>(base + oMu);
  double* res = reinterpret_cast<double*>(base + oRes);
  double* bnorm = reinterpret_cast<double*>(base + oBn);
  void* cqw = base + oCq;
  const double2* z = reinterpret_cast<const double2*>(ctx->con.z);

  reduced_setup_kernel<<<(unsigned)((nS + 255) / 256), 256, 0, s>>>(
      reinterpret_cast<const double2*>(Bhat_dev), z, shift, N, nu, C, S);
  gauss_jordan_kernel<<<1, 1024, 0, s>>>(S, Si, nu, ctx->d_status);
  random_block_kernel<<<(unsigned)((nW + 255) / 256), 256, 0, s>>>(W, (int64_t)nW, 20190609ull);
  bnorm_kernel<<<N, 256, 0, s>>>(reinterpret_cast<const double2*>(Bhat_dev), nu, bnorm);
  ctx->launches += 4;
  st = cuda_check(ctx, cudaGetLastError(), "reduced setup");
  if (st != BEM_OK) return st;
  st = cholqr2_impl(ctx, reinterpret_cast<double*>(W), rows, rows, p, nullptr, cqw, s, 77);
  if (st != BEM_OK) return st;

  // apply H to the block W: T = [C_0 .. C_{N-1}] W, U = S^{-1} T, HW_j = (W_j - U)/(z_j - s)
  auto apply_H = [&]() -> bem_status {
    if (launch_zgemm(ctx, nu, p, (int)rows, reinterpret_cast<double*>(C), nu,
                     reinterpret_cast<double*>(W), rows, reinterpret_cast<double*>(T), nu, s) != cudaSuccess ||
        launch_zgemm(ctx, nu, p, nu, reinterpret_cast<double*>(Si), nu,
                     reinterpret_cast<double*>(T), nu, reinterpret_cast<double*>(U), nu, s) != cudaSuccess)
      return fail(ctx, BEM_ECUDA, "reduced apply");
    reduced_update_kernel<<<(unsigned)((nW + 255) / 256), 256, 0, s>>>(W, U, z, shift, N, nu, p, HW);
    ctx->launches++;
    return cuda_check(ctx, cudaGetLastError(), "reduced apply");
  };

  std::vector<double> hmu(2 * p), hres(p);
  const int check_every = 5;
  int it = 0;
  bool done = false;
  while (!done) {
    // Rayleigh-Ritz on the current block
    const bool rr = (it > 0 && it % check_every == 0) || it >= max_iter;
    st = apply_H();
    if (st != BEM_OK) return st;
    if (rr) {
      st = cuda_check(ctx, launch_xhy_fp64(ctx, reinterpret_cast<double*>(W), rows, p,
                                           reinterpret_cast<double*>(HW), rows, 0, p, rows, 1,
                                           nullptr, reinterpret_cast<double*>(G), s),
                      "reduced rayleigh-ritz");
      if (st != BEM_OK) return st;
      small_eig_kernel<<<1, 32, 0, s>>>(p, G, mu, Vs, Zm, ctx->d_status);
      ctx->launches++;
      // Y = U Vs diag(1/mu): the y-parts of the Ritz vectors (U = S^{-1} C W)
      if (launch_zgemm(ctx, nu, p, p, reinterpret_cast<double*>(U), nu,
                       reinterpret_cast<double*>(Vs), p, Y_dev, nu, s) != cudaSuccess)
        return fail(ctx, BEM_ECUDA, "reduced ritz vectors");
      scale_columns_kernel<<<(unsigned)((nT + 255) / 256), 256, 0, s>>>(
          reinterpret_cast<double2*>(Y_dev), nu, p, mu);
      ctx->launches++;
      // lambda = s + 1/mu, computed on the host from mu; residuals need lambda on device:
      // store lambda into mu's buffer after reading mu
      st = cuda_check(ctx, cudaMemcpyAsync(hmu.data(), mu, 2 * p * sizeof(double),
                                           cudaMemcpyDeviceToHost, s), "reduced copy");
      if (st == BEM_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), "reduced sync");
      if (st != BEM_OK) return st;
      for (int i = 0; i < p; ++i) {
        const double mr = hmu[2 * i], mi = hmu[2 * i + 1];
        const double d = mr * mr + mi * mi;
        lam_host[2 * i] = d > 0.0 ? shift_re + mr / d : INFINITY;
        lam_host[2 * i + 1] = d > 0.0 ? shift_im - mi / d : INFINITY;
      }
      st = cuda_check(ctx, cudaMemcpyAsync(mu, lam_host, 2 * p * sizeof(double),
                                           cudaMemcpyHostToDevice, s), "reduced copy");
      if (st != BEM_OK) return st;
      reduced_residual_kernel<<<p, 256, 0, s>>>(reinterpret_cast<const double2*>(Bhat_dev), z, mu,
                                                reinterpret_cast<const double2*>(Y_dev), N, nu,
                                                bnorm, res);
      ctx->launches++;
      st = cuda_check(ctx, cudaMemcpyAsync(hres.data(), res, p * sizeof(double),
                                           cudaMemcpyDeviceToHost, s), "reduced copy");
      if (st == BEM_OK) st = take_status(ctx, s, "bem_solve_reduced");
      if (st != BEM_OK) return st;
      // converged when every Ritz value inside the contour among the dominant half
      // (largest |mu|, i.e. nearest the shift) has a small reduced residual; the others
      // include the refreshed random directions and are not waited for
      const Contour& c = ctx->con;
      std::vector<int> order(p);
      for (int i = 0; i < p; ++i) order[i] = i;
      std::sort(order.begin(), order.end(), [&](int a, int b) {
        return hmu[2 * a] * hmu[2 * a] + hmu[2 * a + 1] * hmu[2 * a + 1] >
               hmu[2 * b] * hmu[2 * b] + hmu[2 * b + 1] * hmu[2 * b + 1];
      });
      bool all = true;
      for (int r = 0; r < p; ++r) {
        const int i = order[r];
        res_host[i] = hres[i];
        if (r >= (p + 1) / 2) continue;
        const double xr = (lam_host[2 * i] - c.c_re) / c.a, xi = (lam_host[2 * i + 1] - c.c_im) / c.b;
        if (xr * xr + xi * xi < 1.0 && !(hres[i] <= tol)) all = false;
      }
      if (all || it >= max_iter) done = true;
    }
    if (done) break;
    // W <- orth(H W)
    std::swap(W, HW);
    // directions H annihilates (numerically) are refilled at random, so the block keeps
    // full rank when p exceeds the number of non-negligible eigenvalues mu
    st = cholqr2_impl(ctx, reinterpret_cast<double*>(W), rows, rows, p, nullptr, cqw, s,
                      1000003ull * (it + 1));
    if (st != BEM_OK) return st;
    ++it;
  }
  if (iters_done) *iters_done = it;
  return BEM_OK;
}

extern "C" bem_status bem_ritz_vectors(bem_ctx* ctx, const double* V_dev, int64_t ldv, int nu,
                                       const double* Y_dev, int k, double* X_dev, int64_t ldx,
                                       void* stream) {
  if (!ctx) return BEM_EINVAL;
  const int64_t n = ctx->geo.n;
  if (n == 0) return fail(ctx, BEM_ESTATE, "bem_ritz_vectors: no mesh set");
  if (!V_dev || !Y_dev || !X_dev || nu < 1 || k < 1 || ldv < n || ldx < n)
    return fail(ctx, BEM_EINVAL, "bem_ritz_vectors: bad arguments");
  cudaSetDevice(ctx->device);
  return cuda_check(ctx, launch_zgemm(ctx, (int)n, k, nu, V_dev, ldv, Y_dev, nu, X_dev, ldx,
                                      (cudaStream_t)stream),
                    "bem_ritz_vectors");
}

extern "C" bem_status bem_chebyshev_coeffs(bem_ctx* ctx, const double* P_dev, int nu, double* B_dev,
                                           void* stream) {
  if (!ctx) return BEM_EINVAL;
  if (ctx->con.N == 0 || ctx->con.kind != BEM_CONTOUR_CHEBYSHEV)
    return fail(ctx, BEM_ESTATE, "bem_chebyshev_coeffs: the contour must be a Chebyshev interval");
  if (!P_dev || !B_dev || nu < 1 || nu > kMaxNu)
    return fail(ctx, BEM_EINVAL, "bem_chebyshev_coeffs: need P, B and 1 <= nu <= 256");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int N = ctx->con.N;
  bem_status st = ensure_small(ctx, (size_t)N * N * sizeof(double));
  if (st != BEM_OK) return st;
  cheb_table_kernel<<<(N * N + 255) / 256, 256, 0, s>>>(N, ctx->d_small);
  const int64_t nn = (int64_t)nu * nu;
  cheb_coeff_kernel<<<(unsigned)((N * nn + 255) / 256), 256, 0, s>>>(
      reinterpret_cast<const double2*>(P_dev), ctx->d_small, N, nn, reinterpret_cast<double2*>(B_dev));
  ctx->launches += 2;
  return cuda_check(ctx, cudaGetLastError(), "bem_chebyshev_coeffs");
}

namespace {

// Work of the Chebyshev shift-and-invert operator for p columns (in the context's scratch).
struct ChebOp {
  int m = 0, nu = 0, p = 0;
  int64_t rows = 0;
  double2 sigma{};
  const double2* B = nullptr;
  double2 *L, *G, *Gi, *W, *E, *HW, *Y2, *LE, *U, *R, *Sm, *Zm, *Vs, *mu, *dsT;
  double* res;
  void* cqw;
};

bem_status cheb_prepare(bem_ctx* ctx, const double* B_dev, int nu, double2 sigma, int p,
                        ChebOp& op, cudaStream_t s) {
  const int N = ctx->con.N, m = N - 1;
  op.m = m;
  op.nu = nu;
  op.p = p;
  op.rows = (int64_t)m * nu;
  op.sigma = sigma;
  op.B = reinterpret_cast<const double2*>(B_dev);
  // T_i(sigma), i < m, on the host (three-term recurrence)
  std::vector<double> sT(2 * m);
  {
    double pr = 1.0, pi = 0.0, qr = sigma.x, qi = sigma.y;
    for (int i = 0; i < m; ++i) {
      if (i == 0) { sT[0] = 1.0; sT[1] = 0.0; continue; }
      sT[2 * i] = qr;
      sT[2 * i + 1] = qi;
      const double nr = 2.0 * (sigma.x * qr - sigma.y * qi) - pr;
      const double ni = 2.0 * (sigma.x * qi + sigma.y * qr) - pi;
      pr = qr; pi = qi; qr = nr; qi = ni;
    }
  }
  const size_t z2 = sizeof(double2);
  const size_t nn = (size_t)nu * nu, nW = (size_t)op.rows * p, nT = (size_t)nu * p, nG = (size_t)p * p;
  const size_t cq = cholqr2_work_bytes(ctx, op.rows, p);
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
  const size_t oL = take((size_t)m * nn * z2), oG = take(nn * z2), oGi = take(nn * z2),
               oW = take(nW * z2), oE = take(nW * z2), oHW = take(nW * z2), oY2 = take(nT * z2),
               oLE = take(nT * z2), oU = take(nT * z2), oR = take(nT * z2), oS = take(nG * z2),
               oZ = take(nG * z2), oVs = take(nG * z2), oMu = take((size_t)p * z2),
               oRes = take((size_t)p * sizeof(double)), oST = take((size_t)m * z2), oCq = take(cq);
  bem_status st = ensure_scratch(ctx, off);
  if (st != BEM_OK) return st;
  unsigned char* base = reinterpret_cast<unsigned char*>(ctx->d_scratch);
  auto at = [&](size_t o) { return reinterpret_cast<double2*>(base + o); };
  op.L = at(oL); op.G = at(oG); op.Gi = at(oGi); op.W = at(oW); op.E = at(oE); op.HW = at(oHW);
  op.Y2 = at(oY2); op.LE = at(oLE); op.U = at(oU); op.R = at(oR); op.Sm = at(oS); op.Zm = at(oZ);
  op.Vs = at(oVs); op.mu = at(oMu); op.dsT = at(oST);
  op.res = reinterpret_cast<double*>(base + oRes);
  op.cqw = base + oCq;
  st = cuda_check(ctx, cudaMemcpyAsync(op.dsT, sT.data(), 2 * m * sizeof(double),
                                       cudaMemcpyHostToDevice, s), "chebyshev copy");
  if (st != BEM_OK) return st;
  cheb_setup_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(op.B, m, nu, sigma, op.dsT, op.L, op.G);
  gauss_jordan_kernel<<<1, 1024, 0, s>>>(op.G, op.Gi, nu, ctx->d_status);
  ctx->launches += 2;
  return cuda_check(ctx, cudaGetLastError(), "chebyshev setup");
}

// HW = (A - sigma M)^{-1} M W for the op's p columns (W, HW: rows x p, leading dim rows)
bem_status cheb_apply(bem_ctx* ctx, const ChebOp& op, const double2* W, double2* HW, cudaStream_t s) {
  const int m = op.m, nu = op.nu, p = op.p;
  const int64_t rows = op.rows;
  const size_t nn = (size_t)nu * nu, nT = (size_t)nu * p, nW = (size_t)rows * p;
  const double2* Bm = op.B + (size_t)m * nn;
  const double2* wlast = W + (size_t)(m - 1) * nu;
  cheb_recur_kernel<<<(unsigned)((nT + 255) / 256), 256, 0, s>>>(W, m, nu, p, op.sigma, op.E);
  ctx->launches++;
  if (launch_zgemm(ctx, nu, p, nu, reinterpret_cast<const double*>(Bm), nu,
                   reinterpret_cast<const double*>(wlast), rows, reinterpret_cast<double*>(op.Y2), nu,
                   s) != cudaSuccess ||
      launch_zgemm(ctx, nu, p, (int)rows, reinterpret_cast<const double*>(op.L), nu,
                   reinterpret_cast<const double*>(op.E), rows, reinterpret_cast<double*>(op.LE), nu,
                   s) != cudaSuccess)
    return fail(ctx, BEM_ECUDA, "chebyshev apply");
  // rhs = 2 B_m w_{m-1} - L E (Y2 holds B_m w_{m-1})
  cheb_rhs_kernel<<<(unsigned)((nT + 255) / 256), 256, 0, s>>>(op.Y2, op.LE, (int64_t)nT, op.R);
  ctx->launches++;
  if (launch_zgemm(ctx, nu, p, nu, reinterpret_cast<const double*>(op.Gi), nu,
                   reinterpret_cast<const double*>(op.R), nu, reinterpret_cast<double*>(op.U), nu,
                   s) != cudaSuccess)
    return fail(ctx, BEM_ECUDA, "chebyshev apply");
  cheb_combine_kernel<<<(unsigned)((nW + 255) / 256), 256, 0, s>>>(op.E, op.U, op.dsT, m, nu, p, HW);
  ctx->launches++;
  return cuda_check(ctx, cudaGetLastError(), "chebyshev apply");
}

bem_status cheb_check_args(bem_ctx* ctx, const char* who) {
  if (ctx->con.N == 0 || ctx->con.kind != BEM_CONTOUR_CHEBYSHEV)
    return fail(ctx, BEM_ESTATE, std::string(who) + ": the contour must be a Chebyshev interval");
  if (ctx->con.N < 4) return fail(ctx, BEM_EINVAL, std::string(who) + ": need N >= 4 coefficients");
  return BEM_OK;
}

}  // namespace

extern "C" bem_status bem_chebyshev_apply(bem_ctx* ctx, const double* B_dev, int nu,
                                          double shift_re, double shift_im, const double* W_dev,
                                          int p, double* HW_dev, void* stream) {
  if (!ctx) return BEM_EINVAL;
  bem_status st = cheb_check_args(ctx, "bem_chebyshev_apply");
  if (st != BEM_OK) return st;
  const int64_t rows = (int64_t)(ctx->con.N - 1) * nu;
  if (!B_dev || !W_dev || !HW_dev || nu < 1 || nu > kMaxNu || p < 1 || p > 256 || p > rows)
    return fail(ctx, BEM_EINVAL, "bem_chebyshev_apply: bad arguments");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const Contour& con = ctx->con;
  ChebOp op;
  st = cheb_prepare(ctx, B_dev, nu, make_double2((shift_re - con.c_re) / con.a,
                                                 (shift_im - con.c_im) / con.a), p, op, s);
  if (st != BEM_OK) return st;
  st = cheb_apply(ctx, op, reinterpret_cast<const double2*>(W_dev), reinterpret_cast<double2*>(HW_dev), s);
  if (st != BEM_OK) return st;
  return take_status(ctx, s, "bem_chebyshev_apply");
}

extern "C" bem_status bem_solve_chebyshev(bem_ctx* ctx, const double* B_dev, int nu,
                                          double shift_re, double shift_im, int p, int max_iter,
                                          double tol, double* lam_host, double* Y_dev,
                                          double* res_host, int* iters_done, void* stream) {
  if (!ctx) return BEM_EINVAL;
  bem_status st = cheb_check_args(ctx, "bem_solve_chebyshev");
  if (st != BEM_OK) return st;
  const int N = ctx->con.N;
  const int64_t rows = (int64_t)(N - 1) * nu;
  if (!B_dev || !lam_host || !Y_dev || !res_host || nu < 1 || nu > kMaxNu || p < 1 ||
      p > 256 || p > rows || max_iter < 1 || !(tol > 0.0))
    return fail(ctx, BEM_EINVAL,
                "bem_solve_chebyshev: need outputs, 1 <= nu <= 256, 1 <= p <= min(256, (N - 1) nu)");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const Contour& con = ctx->con;
  const double cc = con.c_re, ci = con.c_im, ha = con.a;
  const double2 sigma = make_double2((shift_re - cc) / ha, (shift_im - ci) / ha);
  ChebOp op;
  st = cheb_prepare(ctx, B_dev, nu, sigma, p, op, s);
  if (st != BEM_OK) return st;
  double2* W = op.W;
  double2* HW = op.HW;
  const size_t nW = (size_t)rows * p;
  random_block_kernel<<<(unsigned)((nW + 255) / 256), 256, 0, s>>>(W, (int64_t)nW, 20190609ull);
  ctx->launches++;
  st = cholqr2_impl(ctx, reinterpret_cast<double*>(W), rows, rows, p, nullptr, op.cqw, s, 77);
  if (st != BEM_OK) return st;

  std::vector<double> hmu(2 * p), hres(p), zeta(2 * p);
  const int check_every = 5;
  int it = 0;
  bool done = false;
  while (!done) {
    const bool rr = (it > 0 && it % check_every == 0) || it >= max_iter;
    st = cheb_apply(ctx, op, W, HW, s);
    if (st != BEM_OK) return st;
    if (rr) {
      st = cuda_check(ctx, launch_xhy_fp64(ctx, reinterpret_cast<double*>(W), rows, p,
                                           reinterpret_cast<double*>(HW), rows, 0, p, rows, 1,
                                           nullptr, reinterpret_cast<double*>(op.Sm), s),
                      "chebyshev rayleigh-ritz");
      if (st != BEM_OK) return st;
      small_eig_kernel<<<1, 32, 0, s>>>(p, op.Sm, op.mu, op.Vs, op.Zm, ctx->d_status);
      ctx->launches++;
      // y-parts of the Ritz vectors: the first block of W Vs (v_0 = T_0 y = y)
      if (launch_zgemm(ctx, nu, p, p, reinterpret_cast<double*>(W), rows,
                       reinterpret_cast<double*>(op.Vs), p, Y_dev, nu, s) != cudaSuccess)
        return fail(ctx, BEM_ECUDA, "chebyshev ritz vectors");
      st = cuda_check(ctx, cudaMemcpyAsync(hmu.data(), op.mu, 2 * p * sizeof(double),
                                           cudaMemcpyDeviceToHost, s), "chebyshev copy");
      if (st == BEM_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), "chebyshev sync");
      if (st != BEM_OK) return st;
      for (int i = 0; i < p; ++i) {   // zeta = sigma + 1 / mu, lambda = c + a zeta
        const double mr = hmu[2 * i], mi = hmu[2 * i + 1];
        const double d = mr * mr + mi * mi;
        zeta[2 * i] = d > 0.0 ? sigma.x + mr / d : INFINITY;
        zeta[2 * i + 1] = d > 0.0 ? sigma.y - mi / d : INFINITY;
        lam_host[2 * i] = cc + ha * zeta[2 * i];
        lam_host[2 * i + 1] = ci + ha * zeta[2 * i + 1];
      }
      st = cuda_check(ctx, cudaMemcpyAsync(op.mu, zeta.data(), 2 * p * sizeof(double),
                                           cudaMemcpyHostToDevice, s), "chebyshev copy");
      if (st != BEM_OK) return st;
      cheb_residual_kernel<<<p, 256, 0, s>>>(op.B, op.mu, reinterpret_cast<const double2*>(Y_dev), N,
                                             nu, op.res);
      ctx->launches++;
      st = cuda_check(ctx, cudaMemcpyAsync(hres.data(), op.res, p * sizeof(double),
                                           cudaMemcpyDeviceToHost, s), "chebyshev copy");
      if (st == BEM_OK) st = take_status(ctx, s, "bem_solve_chebyshev");
      if (st != BEM_OK) return st;
      // converged when the dominant half holds at least one Ritz value near the interval
      // (|Re zeta| < 1, |Im zeta| < 0.25) and every such value has a small reduced residual.
      // The colleague operator is far from normal, so the first Rayleigh-Ritz values of a
      // poorly converged block can all be spurious: an empty set is not taken as converged.
      std::vector<int> order(p);
      for (int i = 0; i < p; ++i) order[i] = i;
      std::sort(order.begin(), order.end(), [&](int a, int b) {
        return hmu[2 * a] * hmu[2 * a] + hmu[2 * a + 1] * hmu[2 * a + 1] >
               hmu[2 * b] * hmu[2 * b] + hmu[2 * b + 1] * hmu[2 * b + 1];
      });
      bool all = true;
      int inside = 0;
      for (int r = 0; r < p; ++r) {
        const int i = order[r];
        res_host[i] = hres[i];
        if (r >= (p + 1) / 2) continue;
        if (fabs(zeta[2 * i]) < 1.0 && fabs(zeta[2 * i + 1]) < 0.25) {
          ++inside;
          if (!(hres[i] <= tol)) all = false;
        }
      }
      if ((all && inside > 0) || it >= max_iter) done = true;
    }
    if (done) break;
    std::swap(W, HW);
    st = cholqr2_impl(ctx, reinterpret_cast<double*>(W), rows, rows, p, nullptr, op.cqw, s,
                      1000003ull * (it + 1));
    if (st != BEM_OK) return st;
    ++it;
  }
  if (iters_done) *iters_done = it;
  return BEM_OK;
}
