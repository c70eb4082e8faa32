// Plain FP64 path of the fused assembly + projection (Section 3, Eq. RR_approx).
//
// apply_fp64_kernel: Y_j = A(z_j) V. One block owns a 32-row tile of A(z_j) for one node
// and one 64-column chunk of V; it walks the columns of A in panels of 16, evaluates the
// 32 x 16 panel of entries into shared memory (7-point rule off the diagonal, the
// precomputed self term on it) and multiplies it into the 32 x 64 accumulator at once,
// so A(z_j) is never stored.
// xhy_fp64_kernel: C_j = s_j X^H Y_j, one block per 32 x 32 output tile and batch entry,
// summing over rows in a fixed order (deterministic, no atomics).
#include <math.h>

#include "internal.h"

namespace bem {
namespace {

constexpr int kBM = 32;   // rows per block
constexpr int kBK = 16;   // columns of A per panel
constexpr int kVC = 64;   // columns of V per block
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads)
apply_fp64_kernel(Geometry g, const double* __restrict__ self, const double* __restrict__ z,
                  const double* __restrict__ V, int64_t ldv, int nu,
                  double* __restrict__ Y, OpCoef op) {
  __shared__ double2 sA[kBM][kBK];
  __shared__ double2 sV[kBK][kVC];
  __shared__ double sQ[4][7][kBK];     // x, y, z, weight of the panel's quadrature points
  __shared__ double sN[3][kBK];        // unit normals of the panel's triangles
  const bool general = !op_single(op);
  __shared__ double sC[3][kBM];        // centroids of the tile's rows

  const int64_t n = g.n;
  const int tid = threadIdx.x;
  const int64_t row0 = (int64_t)blockIdx.x * kBM;
  const int j = blockIdx.y;
  const int col0 = blockIdx.z * kVC;
  const double kr = z[2 * j], ki = z[2 * j + 1];

  if (tid < kBM) {
    const int64_t i = row0 + tid;
    for (int c = 0; c < 3; ++c) sC[c][tid] = (i < n) ? g.cx[c * n + i] : 0.0;
  }

  // GEMM mapping: row gr, columns gc0 + 8 m
  const int gr = tid / 8;
  const int gc0 = tid % 8;
  double2 acc[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) acc[m] = make_double2(0.0, 0.0);

  // evaluation mapping: column el, rows er0 + 16 m
  const int el = tid % kBK;
  const int er0 = tid / kBK;

  for (int64_t l0 = 0; l0 < n; l0 += kBK) {
    __syncthreads();   // previous panel fully consumed
    // panel geometry
    for (int t = tid; t < 7 * kBK; t += kThreads) {
      const int q = t / kBK, lc = t % kBK;
      const int64_t l = l0 + lc;
      const bool ok = l < n;
      sQ[0][q][lc] = ok ? g.qp[(0 * 7 + q) * n + l] : 0.0;
      sQ[1][q][lc] = ok ? g.qp[(1 * 7 + q) * n + l] : 0.0;
      sQ[2][q][lc] = ok ? g.qp[(2 * 7 + q) * n + l] : 0.0;
      sQ[3][q][lc] = ok ? g.qw[q * n + l] : 0.0;
    }
    if (general && tid < 3 * kBK) {
      const int c = tid / kBK, lc = tid % kBK;
      sN[c][lc] = (l0 + lc < n) ? g.nrm[c * n + l0 + lc] : 0.0;
    }
    // V panel (zero outside n x nu)
    for (int t = tid; t < kBK * kVC; t += kThreads) {
      const int k = t / kVC, c = t % kVC;
      const int64_t l = l0 + k;
      const int col = col0 + c;
      double2 v = make_double2(0.0, 0.0);
      if (l < n && col < nu) v = reinterpret_cast<const double2*>(V)[(int64_t)col * ldv + l];
      sV[k][c] = v;
    }
    __syncthreads();
    // evaluate the 32 x 16 panel of A(z_j)
    {
      const int64_t l = l0 + el;
#pragma unroll
      for (int m = 0; m < kBM / (kThreads / kBK); ++m) {
        const int rr = er0 + m * (kThreads / kBK);
        const int64_t i = row0 + rr;
        double2 a = make_double2(0.0, 0.0);
        if (i < n && l < n) {
          if (i == l) {
            a = reinterpret_cast<const double2*>(self)[(int64_t)j * n + l];
          } else {
            const double xi = sC[0][rr], yi = sC[1][rr], zi = sC[2][rr];
            if (general) {   // T = c_G G + c_H (1/2 I + K)
              for (int q = 0; q < 7; ++q)
                op_point64(a, op, sQ[3][q][el], sQ[0][q][el] - xi, sQ[1][q][el] - yi,
                           sQ[2][q][el] - zi, sN[0][el], sN[1][el], sN[2][el], kr, ki, false);
            } else
            for (int q = 0; q < 7; ++q) {
              const double dx = xi - sQ[0][q][el], dy = yi - sQ[1][q][el], dz = zi - sQ[2][q][el];
              const double r = sqrt(dx * dx + dy * dy + dz * dz);
              double s, c;
              sincos(kr * r, &s, &c);
              const double amp = sQ[3][q][el] * exp(-ki * r) / r;
              a.x += amp * c;
              a.y += amp * s;
            }
          }
        }
        sA[rr][el] = a;
      }
    }
    __syncthreads();
    // accumulate Y += A_panel V_panel
#pragma unroll 4
    for (int k = 0; k < kBK; ++k) {
      const double2 a = sA[gr][k];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const double2 v = sV[k][gc0 + 8 * m];
        acc[m].x = fma(a.x, v.x, fma(-a.y, v.y, acc[m].x));
        acc[m].y = fma(a.x, v.y, fma(a.y, v.x, acc[m].y));
      }
    }
  }
  const int64_t i = row0 + gr;
  if (i < n) {
    double2* Yj = reinterpret_cast<double2*>(Y) + (int64_t)j * n * nu;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int col = col0 + gc0 + 8 * m;
      if (col < nu) Yj[(int64_t)col * n + i] = acc[m];
    }
  }
}

constexpr int kT = 32;   // output tile of X^H Y

__global__ void __launch_bounds__(kThreads)
xhy_fp64_kernel(const double* __restrict__ X, int64_t ldx, int p, const double* __restrict__ Y,
                int64_t ldy, int64_t strideY, int q, int64_t n, const double* __restrict__ scale,
                double* __restrict__ C) {
  __shared__ double2 sX[kT][kT + 1];
  __shared__ double2 sY[kT][kT + 1];
  const int tiles_a = (p + kT - 1) / kT;
  const int ta = blockIdx.x % tiles_a, tb = blockIdx.x / tiles_a;
  const int jb = blockIdx.y;
  const int tid = threadIdx.x;
  const int oa = tid % kT;        // output row within the tile
  const int ob0 = tid / kT;       // output columns ob0 + 8 m
  const double2* Xc = reinterpret_cast<const double2*>(X);
  const double2* Yc = reinterpret_cast<const double2*>(Y) + (int64_t)jb * strideY;
  double2 acc[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) acc[m] = make_double2(0.0, 0.0);
  for (int64_t r0 = 0; r0 < n; r0 += kT) {
    __syncthreads();
    for (int t = tid; t < kT * kT; t += kThreads) {
      const int rr = t % kT, cc = t / kT;
      const int64_t r = r0 + rr;
      const int a = ta * kT + cc, b = tb * kT + cc;
      sX[rr][cc] = (r < n && a < p) ? Xc[(int64_t)a * ldx + r] : make_double2(0.0, 0.0);
      sY[rr][cc] = (r < n && b < q) ? Yc[(int64_t)b * ldy + r] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < kT; ++rr) {
      const double2 x = sX[rr][oa];   // conj(x) * y
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const double2 y = sY[rr][ob0 + 8 * m];
        acc[m].x = fma(x.x, y.x, fma(x.y, y.y, acc[m].x));
        acc[m].y = fma(x.x, y.y, fma(-x.y, y.x, acc[m].y));
      }
    }
  }
  double2 s = make_double2(1.0, 0.0);
  if (scale) s = reinterpret_cast<const double2*>(scale)[jb];
  const int a = ta * kT + oa;
  if (a < p) {
    double2* Cj = reinterpret_cast<double2*>(C) + (int64_t)jb * p * q;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int b = tb * kT + ob0 + 8 * m;
      if (b < q)
        Cj[(int64_t)b * p + a] = make_double2(s.x * acc[m].x - s.y * acc[m].y,
                                             s.x * acc[m].y + s.y * acc[m].x);
    }
  }
}

}  // namespace

cudaError_t launch_apply_fp64(bem_ctx* ctx, const double* V, int64_t ldv, int nu, double* Y,
                              cudaStream_t s) {
  const int64_t n = ctx->geo.n;
  dim3 grid((unsigned)((n + kBM - 1) / kBM), (unsigned)ctx->con.N, (unsigned)((nu + kVC - 1) / kVC));
  apply_fp64_kernel<<<grid, kThreads, 0, s>>>(ctx->geo, ctx->con.self, ctx->con.z, V, ldv, nu, Y,
                                              ctx->op);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t launch_xhy_fp64(bem_ctx* ctx, const double* X, int64_t ldx, int p, const double* Y,
                            int64_t ldy, int64_t strideY, int q, int64_t n, int nb,
                            const double* scale, double* C, cudaStream_t s) {
  const int tiles = ((p + kT - 1) / kT) * ((q + kT - 1) / kT);
  dim3 grid((unsigned)tiles, (unsigned)nb);
  xhy_fp64_kernel<<<grid, kThreads, 0, s>>>(X, ldx, p, Y, ldy, strideY, q, n, scale, C);
  ctx->launches++;
  return cudaGetLastError();
}

}  // namespace bem
