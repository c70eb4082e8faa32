// CholeskyQR2 orthonormalisation of the Ritz basis.
//
// The paper orthonormalises the basis U before the Rayleigh-Ritz projection (Section 4,
// Example 1). CholeskyQR2: G = V^H V, G = R^H R (R upper, positive diagonal),
// V <- V R^{-1}, and the same once more, which restores orthogonality to working
// precision for well-conditioned V. All steps are deterministic (fixed-order sums).
// FP64 runs at a small fraction of the FP32 rate on this part, so the FP64 work is kept to
// the Gram matrix and the multiplication by the inverse factor: the first pass factors in
// FP32, and the second pass, whose Gram matrix is then near the identity, obtains its
// inverse factor from a few small products instead of a sequential factorisation.
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
constexpr int kGR = 16;   // rows of V staged at a time by the FP64 Gram kernel

// Tile pair (ta, tb), ta <= tb, of the idx-th upper tile: tb = 0, 1, ..., ta = 0..tb.
__device__ __forceinline__ void upper_tile(int idx, int& ta, int& tb) {
  int b = 0;
  while ((b + 1) * (b + 2) / 2 <= idx) ++b;
  tb = b;
  ta = idx - b * (b + 1) / 2;
}

// Partial Gram matrices, FP64: block (tile, r) sums conj(V[i][a]) V[i][b] over its row
// range for the upper tiles only (the Gram matrix is Hermitian; every consumer reads the
// upper triangle). Three real products per complex term: with x = V[i][a], y = V[i][b],
// conj(x) y = (S1 + S2) + i (S3 - S1 + S2), S1 = x.re y.re, S2 = x.im y.im,
// S3 = (x.re - x.im)(y.re + y.im); the sums of the parts are formed once per staged element.
__global__ void __launch_bounds__(256)
gram_partial_kernel(const double2* __restrict__ V, int64_t ldv, int64_t n, int nu,
                    int64_t rows_per_part, double2* __restrict__ part, const int* gate) {
  if (gate && *gate == 0) return;
  __shared__ double xr[kGR][kGT + 1], xi[kGR][kGT + 1], xd[kGR][kGT + 1];
  __shared__ double yr[kGR][kGT + 1], yi[kGR][kGT + 1], ys[kGR][kGT + 1];
  int ta, tb;
  upper_tile(blockIdx.x, ta, tb);
  const int64_t r_begin = (int64_t)blockIdx.y * rows_per_part;
  const int64_t r_end = min(n, r_begin + rows_per_part);
  const int tid = threadIdx.x;
  const int oa = tid % kGT, ob0 = tid / kGT;
  double s1[4], s2[4], s3[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) s1[m] = s2[m] = s3[m] = 0.0;
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kGR) {
    __syncthreads();
    for (int x = tid; x < kGR * kGT; x += 256) {
      const int rr = x % kGR, cc = x / kGR;
      const int64_t r = r0 + rr;
      const int a = ta * kGT + cc, b = tb * kGT + cc;
      const double2 va = (r < r_end && a < nu) ? V[(int64_t)a * ldv + r] : make_double2(0.0, 0.0);
      const double2 vb = (r < r_end && b < nu) ? V[(int64_t)b * ldv + r] : make_double2(0.0, 0.0);
      xr[rr][cc] = va.x;
      xi[rr][cc] = va.y;
      xd[rr][cc] = va.x - va.y;
      yr[rr][cc] = vb.x;
      yi[rr][cc] = vb.y;
      ys[rr][cc] = vb.x + vb.y;
    }
    __syncthreads();
    const int rows = (int)(r_end - r0 < kGR ? r_end - r0 : kGR);
    for (int rr = 0; rr < rows; ++rr) {
      const double ar = xr[rr][oa], ai = xi[rr][oa], ad = xd[rr][oa];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int cb = ob0 + 8 * m;
        s1[m] = fma(ar, yr[rr][cb], s1[m]);
        s2[m] = fma(ai, yi[rr][cb], s2[m]);
        s3[m] = fma(ad, ys[rr][cb], s3[m]);
      }
    }
  }
  const int a = ta * kGT + oa;
  if (a < nu) {
    double2* P = part + (int64_t)blockIdx.y * nu * nu;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int b = tb * kGT + ob0 + 8 * m;
      if (b < nu) P[(int64_t)b * nu + a] = make_double2(s1[m] + s2[m], s3[m] - s1[m] + s2[m]);
    }
  }
}

// Partial Gram matrices in FP32 (first pass), upper tiles; partial sums stored as double2.
__global__ void __launch_bounds__(256)
gram_partial32_kernel(const double2* __restrict__ V, int64_t ldv, int64_t n, int nu,
                      int64_t rows_per_part, double2* __restrict__ part) {
  __shared__ float2 sX[kGT][kGT + 1];
  __shared__ float2 sY[kGT][kGT + 1];
  int ta, tb;
  upper_tile(blockIdx.x, ta, tb);
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

// G = sum of the partials (deterministic): eight threads per element, thread q adding the
// parts q, q + 8, ... in order, then a fixed shuffle tree. Elements of lower tiles are not
// formed.
__global__ void __launch_bounds__(256)
sum_parts_kernel(const double2* __restrict__ part, int parts, int nu, double2* __restrict__ G,
                 const int* gate) {
  if (gate && *gate == 0) return;
  const int64_t count = (int64_t)nu * nu;
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t t = gt / 8;
  const int q = (int)(gt % 8);
  double2 sum = make_double2(0.0, 0.0);
  bool live = t < count;
  if (live) {
    const int a = (int)(t % nu), b = (int)(t / nu);
    live = a / kGT <= b / kGT;
  }
  if (live)
    for (int r = q; r < parts; r += 8) {
      const double2 v = part[(int64_t)r * count + t];
      sum.x += v.x;
      sum.y += v.y;
    }
#pragma unroll
  for (int off = 1; off < 8; off <<= 1) {
    sum.x += __shfl_xor_sync(0xffffffffu, sum.x, off);
    sum.y += __shfl_xor_sync(0xffffffffu, sum.y, off);
  }
  if (live && q == 0) G[t] = sum;
}

// FP32 first-pass factor: Z = R^{-1} for G = R^H R (nu <= 128), one block, by Gaussian
// elimination of [G | I] without pivoting: the left part becomes D L^H and the right part
// L^{-1} (G = L D L^H, L unit lower), so Z = L^{-H} D^{-1/2}. Shared memory holds G's
// trailing lower triangle (G[r][c], r >= c) and W = L^{-1} transposed in the strict upper
// triangle (W[c][r] at row r, column c); step k changes only columns c > k and reads
// column k, so one barrier per step suffices. A pivot below 1e-6 of the largest diagonal
// entry sets *fallback (V too ill-conditioned for an FP32 pass) and Z is not written.
template <int kSlots>   // ceil(nu^2 / 1024)
__global__ void __launch_bounds__(1024)
chol_inv32_kernel(const double2* __restrict__ Gg, int nu, double2* __restrict__ Z, int* fallback) {
  extern __shared__ float2 S[];
  __shared__ float dmax_s;
  const int tid = threadIdx.x;
  const int total = nu * nu;
  for (int e = tid; e < total; e += blockDim.x) {
    const int r = e % nu, c = e / nu;
    float2 v = make_float2(0.f, 0.f);
    if (r >= c) {
      const double2 g = Gg[(int64_t)r * nu + c];   // G[r][c] = conj(G[c][r]), upper stored
      v = make_float2((float)g.x, -(float)g.y);
    }
    S[e] = v;
  }
  if (tid < 32) {
    float m = 0.f;
    for (int k = tid; k < nu; k += 32) m = fmaxf(m, (float)Gg[(int64_t)k * nu + k].x);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (tid == 0) dmax_s = m;
  }
  __syncthreads();
  const float dmax = dmax_s;
  int sr[kSlots], sc[kSlots];
#pragma unroll
  for (int m = 0; m < kSlots; ++m) {
    const int e = tid + m * 1024;
    sr[m] = e < total ? e % nu : 0;
    sc[m] = e < total ? e / nu : -1;
  }
  for (int k = 0; k < nu; ++k) {
    const float d = S[k * nu + k].x;
    if (!(d > 1e-6f * dmax) || !isfinite(d)) {
      if (tid == 0) *fallback = 1;
      return;   // d is the same for every thread: the whole block leaves
    }
    const float rd = 1.f / d;
#pragma unroll
    for (int m = 0; m < kSlots; ++m) {
      const int r = sr[m], c = sc[m];
      if (c <= k) continue;
      if (r >= c) {
        // G[r][c] -= G[r][k] conj(G[c][k]) / d
        const float2 a = S[k * nu + r], b = S[k * nu + c];
        float2 g = S[c * nu + r];
        g.x -= (a.x * b.x + a.y * b.y) * rd;
        g.y -= (a.y * b.x - a.x * b.y) * rd;
        S[c * nu + r] = g;
      } else if (r <= k) {
        // W[c][r] -= (G[c][k] / d) W[k][r], W[k][k] = 1
        const float2 l = S[k * nu + c];
        const float2 w = (r == k) ? make_float2(1.f, 0.f) : S[k * nu + r];
        float2 g = S[c * nu + r];
        g.x -= (l.x * w.x - l.y * w.y) * rd;
        g.y -= (l.x * w.y + l.y * w.x) * rd;
        S[c * nu + r] = g;
      }
    }
    __syncthreads();
  }
  // Z[c][k] = conj(W[k][c]) / sqrt(d_k) for c <= k, zero below the diagonal
  for (int e = tid; e < total; e += blockDim.x) {
    const int c = e % nu, k = e / nu;
    double2 out = make_double2(0.0, 0.0);
    if (c <= k) {
      const float inv = 1.f / sqrtf(S[k * nu + k].x);
      if (c == k) {
        out = make_double2(inv, 0.0);
      } else {
        const float2 w = S[k * nu + c];
        out = make_double2(w.x * inv, -w.y * inv);
      }
    }
    Z[e] = out;
  }
}

// ---- second pass near the identity ----
//
// After a first pass G = V^H V = I + E with ||E|| small. The inverse factor Z = R^{-1} is
// I + Y with Y upper triangular with a real diagonal, and Z^H G Z = I reads
// Y + Y^H = -H(Y), H(Y) = E + Y^H E + E Y + Y^H Y + Y^H E Y. The fixed point
// Y <- -U(H(Y)) (U keeps the strict upper triangle and half the diagonal) gains one order
// of ||E|| per step: Y0 = -U(E) is exact to O(||E||^2), Y1 (without the cubic term) to
// O(||E||^3) and Y2 to O(||E||^4). Only small products are needed, spread over many
// blocks, instead of a sequential Cholesky factorisation and triangular inverse.

// E entry (m, j) from the upper triangle of G.
__device__ __forceinline__ double2 e_entry(const double2* G, int nu, int m, int j) {
  if (m <= j) {
    const double2 g = G[(int64_t)j * nu + m];
    return make_double2(g.x - (m == j ? 1.0 : 0.0), m == j ? 0.0 : g.y);
  }
  const double2 g = G[(int64_t)m * nu + j];
  return make_double2(g.x, -g.y);
}

// Y entry (m, i), m <= i: explicit (Yx non-null) or Y0 = -U(E) from G.
__device__ __forceinline__ double2 y_entry(const double2* G, const double2* Yx, int nu, int m, int i) {
  if (Yx) return Yx[(int64_t)i * nu + m];
  const double2 g = G[(int64_t)i * nu + m];
  return m < i ? make_double2(-g.x, -g.y) : make_double2(-0.5 * (g.x - 1.0), 0.0);
}

constexpr int kNT = 8;     // output tile of the near-identity products (kNT x kNT per block)
constexpr int kNM = 16;    // inner-dimension chunk staged in shared memory

// Tiled small products of the near-identity factor; one 8 x 8 output tile per block of 64
// threads, the inner dimension staged 16 at a time in shared memory.
//  kMode 0: P = Y0^H E (all entries), Q = Y0^H Y0 (upper), Y0 = -U(E) formed from G, and
//           the block sums of |E_ij|^2 (upper triangle, off-diagonal entries twice);
//  kMode 1: P = Y^H E, Q = Y^H Y for the explicit Y;
//  kMode 2: Z = I + Y2, Y2 = -U(E + P + P^H + Q + P Y) (P, Q, Y of mode 1).
template <int kMode>
__global__ void __launch_bounds__(64)
near_tile_kernel(const double2* __restrict__ G, const double2* __restrict__ Y,
                 const double2* __restrict__ Pin, const double2* __restrict__ Qin, int nu,
                 double2* __restrict__ P, double2* __restrict__ Q, double2* __restrict__ Z,
                 float* epsp, const int* gate, const int* skip_if) {
  if ((gate && *gate == 0) || (skip_if && *skip_if != 0)) return;
  __shared__ double2 sA[kNM][kNT], sB[kNM][kNT], sC[kNM][kNT];
  __shared__ float red[64];
  const int tid = threadIdx.x;
  const int ti = tid % kNT, tj = tid / kNT;
  const int i0 = blockIdx.x * kNT, j0 = blockIdx.y * kNT;
  const int i = i0 + ti, j = j0 + tj;
  double2 p = make_double2(0.0, 0.0), q = p;
  // inner index m runs to the last row where the upper-triangular factor is non-zero
  const int mend = min(nu, (kMode == 2 ? j0 : i0) + kNT);
  for (int m0 = 0; m0 < mend; m0 += kNM) {
    __syncthreads();
    for (int x = tid; x < kNM * kNT; x += 64) {
      const int mm = x / kNT, cc = x % kNT;
      const int m = m0 + mm;
      const int ic = i0 + cc, jc = j0 + cc;
      const bool mv = m < nu;
      if (kMode == 2) {
        sA[mm][cc] = (mv && ic < nu) ? Pin[(int64_t)m * nu + ic] : make_double2(0.0, 0.0);   // P(i, m)
        sB[mm][cc] = (mv && jc < nu && m <= jc) ? Y[(int64_t)jc * nu + m] : make_double2(0.0, 0.0);
      } else {
        sA[mm][cc] = (mv && ic < nu && m <= ic) ? y_entry(G, kMode == 0 ? nullptr : Y, nu, m, ic)
                                                : make_double2(0.0, 0.0);
        sB[mm][cc] = (mv && jc < nu) ? e_entry(G, nu, m, jc) : make_double2(0.0, 0.0);
        sC[mm][cc] = (mv && jc < nu && m <= jc) ? y_entry(G, kMode == 0 ? nullptr : Y, nu, m, jc)
                                                : make_double2(0.0, 0.0);
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int mm = 0; mm < kNM; ++mm) {
      const double2 a = sA[mm][ti], b = sB[mm][tj];
      if (kMode == 2) {   // P(i, m) Y(m, j)
        p.x += a.x * b.x - a.y * b.y;
        p.y += a.x * b.y + a.y * b.x;
      } else {            // conj(Y(m, i)) E(m, j), conj(Y(m, i)) Y(m, j)
        const double2 c = sC[mm][tj];
        p.x += a.x * b.x + a.y * b.y;
        p.y += a.x * b.y - a.y * b.x;
        q.x += a.x * c.x + a.y * c.y;
        q.y += a.x * c.y - a.y * c.x;
      }
    }
  }
  const bool in = i < nu && j < nu;
  const int64_t t = (int64_t)j * nu + i;
  if (kMode == 2) {
    if (in) {
      if (i > j) {
        Z[t] = make_double2(0.0, 0.0);
      } else {
        double2 h = e_entry(G, nu, i, j);
        const double2 pp = Pin[t], pt = Pin[(int64_t)i * nu + j], qq = Qin[t];
        h.x += pp.x + pt.x + qq.x + p.x;
        h.y += pp.y - pt.y + qq.y + p.y;
        Z[t] = i < j ? make_double2(-h.x, -h.y) : make_double2(1.0 - 0.5 * h.x, 0.0);
      }
    }
    return;
  }
  if (in) {
    P[t] = p;
    if (i <= j) Q[t] = q;
  }
  if (kMode == 0) {
    float e2 = 0.f;
    if (in && i <= j) {
      const double2 e = e_entry(G, nu, i, j);
      e2 = (float)((e.x * e.x + e.y * e.y) * (i == j ? 1.0 : 2.0));
    }
    red[tid] = e2;
    __syncthreads();
    for (int s = 32; s > 0; s >>= 1) {
      if (tid < s) red[tid] += red[tid + s];
      __syncthreads();
    }
    if (tid == 0) epsp[blockIdx.y * gridDim.x + blockIdx.x] = red[0];
  }
}

// Y1 = -U(E + P + P^H + Q). Every block first sums the block sums of |E|^2 in order; if
// ||E||_F exceeds eps_max the near-identity route is abandoned (*classic = 1) and the
// classic Cholesky factorisation runs instead. *done = 1 tells the second step to skip.
__global__ void __launch_bounds__(64)
near_y1_kernel(const double2* __restrict__ G, const double2* __restrict__ P,
               const double2* __restrict__ Q, const float* __restrict__ epsp, int nparts,
               int nu, float eps_max, float eps_small, double2* __restrict__ Y,
               double2* __restrict__ Z, int* classic, int* done, const int* gate) {
  if (gate && *gate == 0) return;
  __shared__ float e2s;
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int b = 0; b < nparts; ++b) s += epsp[b];
    e2s = s;
  }
  __syncthreads();
  if (!(e2s <= eps_max * eps_max)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      *classic = 1;
      *done = 1;
    }
    return;
  }
  // ||E|| <= eps_small: Y1 is already exact to rounding (its error is O(||E||^3)), so
  // Z = I + Y1 is written here and the second step is skipped
  const bool small = e2s <= eps_small * eps_small;
  if (small && blockIdx.x == 0 && threadIdx.x == 0) *done = 1;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nu * nu) return;
  const int i = (int)(t % nu), j = (int)(t / nu);
  double2 y = make_double2(0.0, 0.0);
  if (i < j) {
    const double2 e = e_entry(G, nu, i, j), p = P[t], pt = P[(int64_t)i * nu + j], q = Q[t];
    y = make_double2(-(e.x + p.x + pt.x + q.x), -(e.y + p.y - pt.y + q.y));
  } else if (i == j) {
    const double2 e = e_entry(G, nu, i, i), p = P[t], q = Q[t];
    y = make_double2(-0.5 * (e.x + 2.0 * p.x + q.x), 0.0);
  }
  if (small)
    Z[t] = i == j ? make_double2(1.0 + y.x, 0.0) : y;
  else
    Y[t] = y;
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

constexpr int kRMRows = 8;    // rows of V per block
constexpr int kRMK = 16;      // k chunk of M staged at a time

size_t right_multiply_smem(int nu) {
  return (size_t)(3 * nu * kRMRows + 3 * kRMK * (nu + 1)) * sizeof(double);
}

// V <- V M in place, M nu x nu upper triangular (column-major, zero below the diagonal);
// each block owns kRMRows complete rows of V, staged in shared memory before any is
// overwritten. Three real products per complex term: a b = (S1 - S2) + i (S3 - S1 - S2),
// S1 = a.re b.re, S2 = a.im b.im, S3 = (a.re + a.im)(b.re + b.im).
// gate, need: skip unless *gate != 0 and *need != 0; skip_if: skip when *skip_if != 0.
__global__ void __launch_bounds__(256)
right_multiply_kernel(double2* V, int64_t ldv, int64_t n, int nu, const double2* __restrict__ M,
                      const int* gate, const int* skip_if, const int* need) {
  if ((gate && *gate == 0) || (need && *need == 0) || (skip_if && *skip_if != 0)) return;
  extern __shared__ double rm_smem[];
  double* vr = rm_smem;                  // [nu][kRMRows]
  double* vi = vr + nu * kRMRows;
  double* vs = vi + nu * kRMRows;
  double* mr = vs + nu * kRMRows;        // [kRMK][nu + 1]
  double* mi = mr + kRMK * (nu + 1);
  double* ms = mi + kRMK * (nu + 1);
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * kRMRows;
  for (int t = tid; t < kRMRows * nu; t += blockDim.x) {
    const int rr = t % kRMRows, c = t / kRMRows;
    const int64_t r = r0 + rr;
    const double2 v = (r < n) ? V[(int64_t)c * ldv + r] : make_double2(0.0, 0.0);
    vr[c * kRMRows + rr] = v.x;
    vi[c * kRMRows + rr] = v.y;
    vs[c * kRMRows + rr] = v.x + v.y;
  }
  constexpr int kOut = kMaxNu * kRMRows / 256;   // outputs per thread at nu = kMaxNu
  const int outs = kRMRows * nu;
  double s1[kOut], s2[kOut], s3[kOut];
#pragma unroll
  for (int m = 0; m < kOut; ++m) s1[m] = s2[m] = s3[m] = 0.0;
  for (int k0 = 0; k0 < nu; k0 += kRMK) {
    const int kn = min(kRMK, nu - k0);
    __syncthreads();
    for (int t = tid; t < kRMK * nu; t += blockDim.x) {
      const int kk = t % kRMK, c = t / kRMK;
      const double2 b = kk < kn ? M[(int64_t)c * nu + k0 + kk] : make_double2(0.0, 0.0);
      mr[kk * (nu + 1) + c] = b.x;
      mi[kk * (nu + 1) + c] = b.y;
      ms[kk * (nu + 1) + c] = b.x + b.y;
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < kOut; ++m) {
      const int o = tid + 256 * m;
      if (o >= outs) break;
      const int c = o % nu, rr = o / nu;
      if (c < k0) continue;   // M[k][c] = 0 for k > c
      for (int kk = 0; kk < kn; ++kk) {
        const int k = k0 + kk;
        s1[m] = fma(vr[k * kRMRows + rr], mr[kk * (nu + 1) + c], s1[m]);
        s2[m] = fma(vi[k * kRMRows + rr], mi[kk * (nu + 1) + c], s2[m]);
        s3[m] = fma(vs[k * kRMRows + rr], ms[kk * (nu + 1) + c], s3[m]);
      }
    }
  }
#pragma unroll
  for (int m = 0; m < kOut; ++m) {
    const int o = tid + 256 * m;
    if (o >= outs) break;
    const int c = o % nu, rr = o / nu;
    const int64_t r = r0 + rr;
    if (r < n) V[(int64_t)c * ldv + r] = make_double2(s1[m] - s2[m], s3[m] - s1[m] - s2[m]);
  }
}

// V <- V + V (M - I) for the near-identity factor M = I + Y (upper triangular), with the
// small product V Y in double-FP32 arithmetic on the FP32 pipe (this GPU's FP64 pipe runs at
// ~1/65 of its rate). Each FP64 value x is carried as hi + lo, hi = fl32(x),
// lo = fl32(x - hi); the product hi_v hi_y is formed exactly (its rounding error recovered by
// an FMA) and added to the running sum by an error-free two-sum; the error terms and the
// hi x lo cross products gather in an FP32 companion, whose own rounding leaves a relative
// error of ~1e-13 of the sum of the terms' magnitudes. Since ||Y|| <= ~||G - I|| (at most
// 5e-4 on this route, ~1e-6 after an FP32 first pass), that is ~1e-17 of |V| or less: below
// V's own FP64 rounding, which the final FP64 addition V + V Y then sets.
// Same blocking as right_multiply_kernel: kRMRows complete rows per block, staged first.
// gate: skip unless *gate != 0; skip_if: skip when *skip_if != 0.
constexpr int kDFK = 8;   // k chunk of M staged at a time
size_t right_multiply_df_smem(int nu) {
  return (size_t)(nu * kRMRows + kDFK * nu) * sizeof(float4);
}

// Error-free transformations, written with the _rn intrinsics so that the compiler neither
// contracts a product into a following addition nor reorders the sums.
__device__ __forceinline__ void two_sum(float& s, float b, float& err) {
  const float t = __fadd_rn(s, b);
  const float bb = __fsub_rn(t, s);
  err = __fadd_rn(err, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(b, bb)));
  s = t;
}
// s + lo += x y with the product's rounding error recovered exactly
__device__ __forceinline__ void df_mac(float& s, float& lo, float x, float y) {
  const float p = __fmul_rn(x, y);
  lo = __fadd_rn(lo, __fmaf_rn(x, y, -p));
  two_sum(s, p, lo);
}

// Y = M - I split once into FP32 (re hi, im hi, re lo, im lo) for every block of the
// multiply (the conversions run on the FP64 pipe).
__global__ void split_near_factor_kernel(const double2* __restrict__ M, int nu,
                                         float4* __restrict__ Ms, const int* gate,
                                         const int* skip_if) {
  if ((gate && *gate == 0) || (skip_if && *skip_if != 0)) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nu * nu) return;
  double2 b = M[t];
  if (t % nu == t / nu) b.x -= 1.0;   // exact: the diagonal is near 1
  const float br = (float)b.x, bi = (float)b.y;
  Ms[t] = make_float4(br, bi, (float)(b.x - br), (float)(b.y - bi));
}

__global__ void __launch_bounds__(256)
right_multiply_near_df_kernel(double2* V, int64_t ldv, int64_t n, int nu,
                              const float4* __restrict__ Ms, const int* gate, const int* skip_if) {
  if ((gate && *gate == 0) || (skip_if && *skip_if != 0)) return;
  extern __shared__ float4 df_smem[];
  float4* sV = df_smem;                 // [nu][kRMRows]: (re hi, im hi, re lo, im lo)
  float4* sM = sV + nu * kRMRows;       // [kDFK][nu]
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * kRMRows;
  for (int t = tid; t < kRMRows * nu; t += blockDim.x) {
    const int rr = t % kRMRows, c = t / kRMRows;
    const int64_t r = r0 + rr;
    const double2 v = (r < n) ? V[(int64_t)c * ldv + r] : make_double2(0.0, 0.0);
    const float hr = (float)v.x, hi = (float)v.y;
    sV[c * kRMRows + rr] = make_float4(hr, hi, (float)(v.x - hr), (float)(v.y - hi));
  }
  constexpr int kOut = kMaxNu * kRMRows / 256;
  const int outs = kRMRows * nu;
  float sr[kOut], srl[kOut], si[kOut], sil[kOut];
#pragma unroll
  for (int m = 0; m < kOut; ++m) sr[m] = srl[m] = si[m] = sil[m] = 0.f;
  for (int k0 = 0; k0 < nu; k0 += kDFK) {
    const int kn = min(kDFK, nu - k0);
    __syncthreads();
    for (int t = tid; t < kDFK * nu; t += blockDim.x) {
      const int kk = t / nu, c = t % nu;
      sM[kk * nu + c] = kk < kn ? Ms[(int64_t)c * nu + k0 + kk] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < kOut; ++m) {
      const int o = tid + 256 * m;
      if (o >= outs) break;
      const int c = o % nu, rr = o / nu;
      const int kend = min(kn, c - k0 + 1);   // M[k][c] = 0 for k > c
      for (int kk = 0; kk < kend; ++kk) {
        const float4 a = sV[(k0 + kk) * kRMRows + rr];
        const float4 b = sM[kk * nu + c];
        // real part: a.re b.re - a.im b.im, then the hi x lo cross terms
        df_mac(sr[m], srl[m], a.x, b.x);
        df_mac(sr[m], srl[m], -a.y, b.y);
        srl[m] = __fmaf_rn(a.x, b.z, srl[m]);
        srl[m] = __fmaf_rn(a.z, b.x, srl[m]);
        srl[m] = __fmaf_rn(-a.y, b.w, srl[m]);
        srl[m] = __fmaf_rn(-a.w, b.y, srl[m]);
        // imaginary part: a.re b.im + a.im b.re
        df_mac(si[m], sil[m], a.x, b.y);
        df_mac(si[m], sil[m], a.y, b.x);
        sil[m] = __fmaf_rn(a.x, b.w, sil[m]);
        sil[m] = __fmaf_rn(a.z, b.y, sil[m]);
        sil[m] = __fmaf_rn(a.y, b.z, sil[m]);
        sil[m] = __fmaf_rn(a.w, b.x, sil[m]);
      }
    }
  }
#pragma unroll
  for (int m = 0; m < kOut; ++m) {
    const int o = tid + 256 * m;
    if (o >= outs) break;
    const int c = o % nu, rr = o / nu;
    const int64_t r = r0 + rr;
    if (r >= n) continue;
    // V + V Y: the block's own rows, still unchanged in global memory
    const double2 v = V[(int64_t)c * ldv + r];
    V[(int64_t)c * ldv + r] = make_double2(v.x + ((double)sr[m] + (double)srl[m]),
                                           v.y + ((double)si[m] + (double)sil[m]));
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

namespace {

struct CqLayout {
  int tiles_u = 0;           // upper Gram tiles
  int64_t parts = 0, rows_per_part = 0;
  int near_blocks = 0;       // blocks of the near-identity element kernels (64 threads)
  int near_tiles = 0;        // 8 x 8 tiles of the near-identity products
  unsigned sum_blocks = 0;   // blocks of sum_parts_kernel (eight threads per element)
};

CqLayout cq_layout(bem_ctx* ctx, int64_t n, int nu) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  CqLayout L;
  const int T = (nu + kGT - 1) / kGT;
  L.tiles_u = T * (T + 1) / 2;
  L.parts = std::max<int64_t>(1, std::min<int64_t>((n + kGT - 1) / kGT,
                                                   (2 * (int64_t)sms + L.tiles_u - 1) / L.tiles_u));
  L.rows_per_part = (n + L.parts - 1) / L.parts;
  L.parts = (n + L.rows_per_part - 1) / L.rows_per_part;
  L.near_blocks = (int)(((int64_t)nu * nu + 63) / 64);
  L.near_tiles = ((nu + 7) / 8) * ((nu + 7) / 8);
  L.sum_blocks = (unsigned)((8 * (int64_t)nu * nu + 255) / 256);
  return L;
}

// Work space: nine nu x nu complex matrices (G, Z, R1, R2, P, Q, Y, P1, Q1), the Gram
// partials, then 256 deficiency flags, 8 pass flags and the |E|^2 block sums.
struct CqWork {
  double2 *G, *Z, *R1, *R2, *P, *Q, *Y, *P1, *Q1, *part;
  int* deficient;
  int* flags;
  float* epsp;
};

CqWork cq_work(void* work, int nu, const CqLayout& L) {
  CqWork w;
  double2* p = reinterpret_cast<double2*>(work);
  const size_t m = (size_t)nu * nu;
  w.G = p; w.Z = p + m; w.R1 = p + 2 * m; w.R2 = p + 3 * m; w.P = p + 4 * m; w.Q = p + 5 * m;
  w.Y = p + 6 * m; w.P1 = p + 7 * m; w.Q1 = p + 8 * m; w.part = p + 9 * m;
  w.deficient = reinterpret_cast<int*>(w.part + (size_t)L.parts * m);
  w.flags = w.deficient + 256;
  w.epsp = reinterpret_cast<float*>(w.flags + 8);
  return w;
}

// ||G - I||_F up to which the near-identity factor is used; its error is O(||G - I||^4)
// (at 8e-4 it still matches the Cholesky factor to rounding)
constexpr float kNearEps = 5e-4f;
// ||G - I||_F up to which the first step alone is exact to rounding
constexpr float kNearEpsSmall = 1e-5f;

bem_status set_smem(bem_ctx* ctx, const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return BEM_OK;
  return cuda_check(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)bytes),
                    "cholqr attribute");
}

// One FP64 pass V <- V R^{-1} whose Gram matrix is expected near the identity: the
// near-identity factor, or the classic Cholesky factorisation and triangular inverse when
// ||G - I||_F > kNearEps (flag *classic, set on the device). Everything is skipped unless
// *gate != 0 (gate null: always runs).
bem_status near_pass(bem_ctx* ctx, double* V_dev, int64_t ldv, int64_t n, int nu,
                     const CqLayout& L, const CqWork& w, const int* gate, int* classic,
                     cudaStream_t s) {
  int* done = classic + 2;   // classic flag and its "second step not needed" companion
  bem_status st = cuda_check(ctx, cudaMemsetAsync(classic, 0, 3 * sizeof(int), s), "cholqr flag");
  if (st != BEM_OK) return st;
  double2* V = reinterpret_cast<double2*>(V_dev);
  const unsigned nb = (unsigned)L.near_blocks;
  gram_partial_kernel<<<dim3((unsigned)L.tiles_u, (unsigned)L.parts), 256, 0, s>>>(
      V, ldv, n, nu, L.rows_per_part, w.part, gate);
  sum_parts_kernel<<<L.sum_blocks, 256, 0, s>>>(w.part, (int)L.parts, nu, w.G, gate);
  const unsigned nt = (unsigned)((nu + kNT - 1) / kNT);
  const dim3 tgrid(nt, nt);
  near_tile_kernel<0><<<tgrid, 64, 0, s>>>(w.G, nullptr, nullptr, nullptr, nu, w.P, w.Q, nullptr,
                                           w.epsp, gate, nullptr);
  near_y1_kernel<<<nb, 64, 0, s>>>(w.G, w.P, w.Q, w.epsp, (int)(nt * nt), nu, kNearEps,
                                   kNearEpsSmall, w.Y, w.Z, classic, done, gate);
  const size_t chol_smem = nu <= 64 ? (size_t)nu * nu * sizeof(double2) : 0;
  cholesky_kernel<<<1, 1024, chol_smem, s>>>(w.G, nu, ctx->d_status, nullptr, classic);
  triangular_inverse_kernel<<<nu, 128, 0, s>>>(w.G, nu, w.Z, classic);
  near_tile_kernel<1><<<tgrid, 64, 0, s>>>(w.G, w.Y, nullptr, nullptr, nu, w.P1, w.Q1, nullptr,
                                           nullptr, gate, done);
  near_tile_kernel<2><<<tgrid, 64, 0, s>>>(w.G, w.Y, w.P1, w.Q1, nu, nullptr, nullptr, w.Z,
                                           nullptr, gate, done);
  // V <- V Z: the classic inverse in FP64, the near-identity factor as V + V (Z - I)
  const unsigned rb = (unsigned)((n + kRMRows - 1) / kRMRows);
  right_multiply_kernel<<<rb, 256, right_multiply_smem(nu), s>>>(V, ldv, n, nu, w.Z, gate,
                                                                 nullptr, classic);
  float4* Zs = reinterpret_cast<float4*>(w.R2);   // R2 is free outside the classic passes
  split_near_factor_kernel<<<(unsigned)((nu * nu + 255) / 256), 256, 0, s>>>(w.Z, nu, Zs, gate,
                                                                            classic);
  right_multiply_near_df_kernel<<<rb, 256, right_multiply_df_smem(nu), s>>>(V, ldv, n, nu, Zs,
                                                                            gate, classic);
  ctx->launches += 11;
  return cuda_check(ctx, cudaGetLastError(), "cholqr kernels");
}

// Classic FP64 pass: Gram, Cholesky (optionally refreshing collapsed columns), inverse,
// V <- V R^{-1}; R kept in R_out.
bem_status classic_pass(bem_ctx* ctx, double* V_dev, int64_t ldv, int64_t n, int nu,
                        const CqLayout& L, const CqWork& w, double2* R_out, uint64_t refresh_seed,
                        cudaStream_t s) {
  double2* V = reinterpret_cast<double2*>(V_dev);
  gram_partial_kernel<<<dim3((unsigned)L.tiles_u, (unsigned)L.parts), 256, 0, s>>>(
      V, ldv, n, nu, L.rows_per_part, w.part, nullptr);
  sum_parts_kernel<<<L.sum_blocks, 256, 0, s>>>(w.part, (int)L.parts, nu, R_out, nullptr);
  const size_t chol_smem = nu <= 64 ? (size_t)nu * nu * sizeof(double2) : 0;
  cholesky_kernel<<<1, 1024, chol_smem, s>>>(R_out, nu, ctx->d_status,
                                             refresh_seed ? w.deficient : nullptr, nullptr);
  triangular_inverse_kernel<<<nu, 128, 0, s>>>(R_out, nu, w.Z, nullptr);
  right_multiply_kernel<<<(unsigned)((n + kRMRows - 1) / kRMRows), 256, right_multiply_smem(nu),
                          s>>>(V, ldv, n, nu, w.Z, nullptr, nullptr, nullptr);
  ctx->launches += 5;
  if (refresh_seed) {
    refresh_columns_kernel<<<(unsigned)((n * nu + 255) / 256), 256, 0, s>>>(V, ldv, n, nu,
                                                                           w.deficient,
                                                                           refresh_seed);
    ctx->launches++;
  }
  return cuda_check(ctx, cudaGetLastError(), "cholqr kernels");
}

}  // namespace

size_t cholqr2_work_bytes(bem_ctx* ctx, int64_t n, int nu) {
  const CqLayout L = cq_layout(ctx, n, nu);
  return (9 + (size_t)L.parts) * (size_t)nu * nu * sizeof(double2) +
         (256 + 8) * sizeof(int) + (size_t)L.near_tiles * sizeof(float);
}

// CholeskyQR2 of V (n x nu, ld ldv) with caller-provided work (cholqr2_work_bytes);
// asynchronous; a Gram matrix that is not positive definite is flagged in the context's
// status word.
//
// Without R: the first pass runs in FP32 (nu <= 128, no refresh): it only has to make V
// well conditioned. The FP64 second pass then sees G = I + E with small E and uses the
// near-identity factor. If V is too ill-conditioned for FP32 the first pass leaves V alone
// (device flag) and a third pass runs (its kernels return at once otherwise); the second
// pass then falls back to the classic factorisation by itself. With R: two classic passes
// and R = R2 R1.
bem_status cholqr2_impl(bem_ctx* ctx, double* V_dev, int64_t n, int64_t ldv, int nu,
                        double* R_dev, void* work, cudaStream_t s, uint64_t refresh_seed) {
  const CqLayout L = cq_layout(ctx, n, nu);
  const CqWork w = cq_work(work, nu, L);
  bem_status st = BEM_OK;
  const size_t chol_smem = nu <= 64 ? (size_t)nu * nu * sizeof(double2) : 0;
  if ((st = set_smem(ctx, (const void*)cholesky_kernel, chol_smem)) != BEM_OK) return st;
  if ((st = set_smem(ctx, (const void*)right_multiply_kernel, right_multiply_smem(nu))) != BEM_OK)
    return st;
  if ((st = set_smem(ctx, (const void*)right_multiply_near_df_kernel,
                     right_multiply_df_smem(nu))) != BEM_OK)
    return st;
  if (R_dev) {
    if ((st = classic_pass(ctx, V_dev, ldv, n, nu, L, w, w.R1, refresh_seed, s)) != BEM_OK) return st;
    if ((st = classic_pass(ctx, V_dev, ldv, n, nu, L, w, w.R2, 0, s)) != BEM_OK) return st;
    upper_product_kernel<<<1, 256, 0, s>>>(w.R2, w.R1, nu, reinterpret_cast<double2*>(R_dev));
    ctx->launches++;
    return cuda_check(ctx, cudaGetLastError(), "cholqr kernels");
  }
  const bool fp32_first = refresh_seed == 0 && nu <= 128;
  if (!fp32_first) {
    if ((st = classic_pass(ctx, V_dev, ldv, n, nu, L, w, w.R1, refresh_seed, s)) != BEM_OK) return st;
    return near_pass(ctx, V_dev, ldv, n, nu, L, w, nullptr, w.flags + 1, s);
  }
  int* fallback = w.flags;
  const size_t ci_smem = (size_t)nu * nu * sizeof(float2);
  if ((st = set_smem(ctx, (const void*)chol_inv32_kernel<4>, ci_smem)) != BEM_OK ||
      (st = set_smem(ctx, (const void*)chol_inv32_kernel<16>, ci_smem)) != BEM_OK)
    return st;
  st = cuda_check(ctx, cudaMemsetAsync(fallback, 0, sizeof(int), s), "cholqr flag");
  if (st != BEM_OK) return st;
  double2* V = reinterpret_cast<double2*>(V_dev);
  gram_partial32_kernel<<<dim3((unsigned)L.tiles_u, (unsigned)L.parts), 256, 0, s>>>(
      V, ldv, n, nu, L.rows_per_part, w.part);
  sum_parts_kernel<<<L.sum_blocks, 256, 0, s>>>(w.part, (int)L.parts, nu, w.G, nullptr);
  if (nu <= 64)
    chol_inv32_kernel<4><<<1, 1024, ci_smem, s>>>(w.G, nu, w.Z, fallback);
  else
    chol_inv32_kernel<16><<<1, 1024, ci_smem, s>>>(w.G, nu, w.Z, fallback);
  right_multiply_kernel<<<(unsigned)((n + kRMRows - 1) / kRMRows), 256, right_multiply_smem(nu),
                          s>>>(V, ldv, n, nu, w.Z, nullptr, fallback, nullptr);
  ctx->launches += 4;
  if ((st = cuda_check(ctx, cudaGetLastError(), "cholqr kernels")) != BEM_OK) return st;
  if ((st = near_pass(ctx, V_dev, ldv, n, nu, L, w, nullptr, w.flags + 1, s)) != BEM_OK) return st;
  return near_pass(ctx, V_dev, ldv, n, nu, L, w, fallback, w.flags + 4, s);
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
  if (ctx->async) return cuda_check(ctx, cudaGetLastError(), "bem_cholqr2");
  return take_status(ctx, s, "bem_cholqr2");
}
