// Dense FP32 matrices of the operator and their LU factorisation.
//
// * assemble32_kernel: M = sum_k c_k A(kappa_k) as a dense n x n complex64 matrix
//   (column-major), one thread per entry, FP32 evaluation with MUFU ex2/sin/cos as in the
//   mixed projection, self terms from an FP32 table. With one wavenumber this is A(sigma),
//   the matrix the residual-inverse refinement factorises; with the contour nodes and
//   c_j = w_j / (z_j - s) it is the Schur complement S = sum_j B_j / (z_j - s) of the
//   inverse power step (Algorithm 1, Eq. linsyssim).
// * lu32: right-looking blocked LU with partial pivoting (panel width 32): panel
//   factorisation in one block, row interchanges, triangular solve for the block row,
//   complex GEMM update of the trailing matrix. lu32_solve applies it to a block of
//   right-hand sides. FP32 is enough here: both users only need an approximate inverse
//   (the refinement's fixed point is defined by FP64 residuals).
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "selfterm.cuh"

namespace bem {
namespace {

constexpr float kLog2eF = 1.4426950408889634f;
constexpr float kInv2PiF = 0.15915494309189535f;
constexpr float kTwoPiHiF = 6.28318548202514648f;
constexpr float kTwoPiLoF = -1.7484555314695172e-7f;

__device__ __forceinline__ float mufu_ex2(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float mufu_sin(float x) {
  float r;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float mufu_cos(float x) {
  float r;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

constexpr int kMaxK = 64;   // wavenumbers per assembly

struct KList {
  int nk;
  float kr[kMaxK], kmi[kMaxK];   // Re k, -Im k log2(e)
  float ki[kMaxK];               // Im k
  float cr[kMaxK], ci[kMaxK];    // coefficients
};

// One thread per entry (i, l), i fastest (coalesced column-major writes).
__global__ void __launch_bounds__(256)
assemble32_kernel(Geometry g, KList K, const float2* __restrict__ self32, float2* __restrict__ M,
                  OpCoef op) {
  const int64_t n = g.n;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const int64_t i = t % n, l = t / n;
  float sr = 0.f, si = 0.f;
  if (i == l) {
    for (int k = 0; k < K.nk; ++k) {
      const float2 v = self32[(int64_t)k * n + l];
      sr += K.cr[k] * v.x - K.ci[k] * v.y;
      si += K.cr[k] * v.y + K.ci[k] * v.x;
    }
  } else {
    const float xi = g.cx32[i], yi = g.cx32[n + i], zi = g.cx32[2 * n + i];
    const bool general = !op_single(op);
    float nx = 0.f, ny = 0.f, nz = 0.f;
    if (general) {
      nx = (float)g.nrm[l];
      ny = (float)g.nrm[n + l];
      nz = (float)g.nrm[2 * n + l];
    }
    float rr[7], am[7], sq[7];   // sq: (y - x) . n / r^2 (general operator)
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      const float dx = xi - g.qp32[q * n + l], dy = yi - g.qp32[(7 + q) * n + l],
                  dz = zi - g.qp32[(14 + q) * n + l];
      const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      const float rs = rsqrtf(r2);
      rr[q] = r2 * rs;
      am[q] = g.qw32[q * n + l] * rs;
      sq[q] = general ? -(dx * nx + dy * ny + dz * nz) * rs * rs : 0.f;
    }
    for (int k = 0; k < K.nk; ++k) {
      float er = 0.f, ei = 0.f;
#pragma unroll
      for (int q = 0; q < 7; ++q) {
        const float a = am[q] * mufu_ex2(K.kmi[k] * rr[q]);
        const float ph = K.kr[k] * rr[q];
        const float nrot = fmaf(ph, kInv2PiF, 12582912.0f) - 12582912.0f;
        const float red = fmaf(-nrot, kTwoPiLoF, fmaf(-nrot, kTwoPiHiF, ph));
        if (general) {   // T = c_G G + c_H (1/2 I + K): times F
          float fr, fi;
          op_factor(op, sq[q], ph, K.ki[k] * rr[q], fr, fi);
          const float cr = a * mufu_cos(red), ci = a * mufu_sin(red);
          er += cr * fr - ci * fi;
          ei += cr * fi + ci * fr;
        } else {
          er = fmaf(a, mufu_cos(red), er);
          ei = fmaf(a, mufu_sin(red), ei);
        }
      }
      sr += K.cr[k] * er - K.ci[k] * ei;
      si += K.cr[k] * ei + K.ci[k] * er;
    }
  }
  M[t] = make_float2(sr, si);
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cdivf(float2 a, float2 b) {
  const float d = b.x * b.x + b.y * b.y;
  return make_float2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

constexpr int kNB = 32;   // panel width

// Factor the panel A[k0:n, k0:k0+kb] in place (one block, 1024 threads).
__global__ void __launch_bounds__(1024)
lu_panel_kernel(float2* A, int64_t n, int64_t k0, int kb, int* ipiv, int* status) {
  __shared__ float bval[32];
  __shared__ int bidx[32];
  __shared__ int piv;
  __shared__ float2 prow[kNB];
  const int tid = threadIdx.x, lane = tid % 32, w = tid / 32;
  for (int c = 0; c < kb; ++c) {
    const int64_t col = k0 + c;
    float bv = -1.f;
    int64_t bi = col;
    for (int64_t r = col + tid; r < n; r += blockDim.x) {
      const float2 v = A[col * n + r];
      const float a = fabsf(v.x) + fabsf(v.y);
      if (a > bv) { bv = a; bi = r; }
    }
    int bii = (int)bi;
    for (int off = 16; off > 0; off >>= 1) {
      const float ov = __shfl_down_sync(0xffffffffu, bv, off);
      const int oi = __shfl_down_sync(0xffffffffu, bii, off);
      if (ov > bv || (ov == bv && oi < bii)) { bv = ov; bii = oi; }
    }
    if (lane == 0) { bval[w] = bv; bidx[w] = bii; }
    __syncthreads();
    if (tid == 0) {
      float b = -1.f;
      int bj = (int)col;
      for (int q = 0; q < (int)(blockDim.x / 32); ++q)
        if (bval[q] > b || (bval[q] == b && bidx[q] < bj)) { b = bval[q]; bj = bidx[q]; }
      piv = bj;
      ipiv[col] = bj;
      if (!(b > 0.f)) atomicOr(status, kStatusNotSPD);
    }
    __syncthreads();
    const int64_t pr = piv;
    // swap rows col and pr inside the panel
    if (pr != col && tid < kb) {
      const float2 a = A[(k0 + tid) * n + col], b = A[(k0 + tid) * n + pr];
      A[(k0 + tid) * n + col] = b;
      A[(k0 + tid) * n + pr] = a;
    }
    __syncthreads();
    if (tid < kb) prow[tid] = A[(k0 + tid) * n + col];
    __syncthreads();
    const float2 dinv = cdivf(make_float2(1.f, 0.f), prow[c]);
    // multipliers and the rank-1 update of the rest of the panel
    for (int64_t r = col + 1 + tid; r < n; r += blockDim.x) {
      const float2 m = cmulf(A[col * n + r], dinv);
      A[col * n + r] = m;
      for (int j = c + 1; j < kb; ++j) {
        const float2 u = prow[j];
        float2 v = A[(k0 + j) * n + r];
        v.x -= m.x * u.x - m.y * u.y;
        v.y -= m.x * u.y + m.y * u.x;
        A[(k0 + j) * n + r] = v;
      }
    }
    __syncthreads();
  }
}

// Apply the interchanges ipiv[k0 .. k0+kb) to the columns outside [k0, k0+kb) (one thread
// per column, in order).
__global__ void lu_swap_kernel(float2* A, int64_t n, int64_t ncols, int64_t k0, int kb,
                               const int* ipiv, int64_t skip_begin, int64_t skip_end) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= ncols || (j >= skip_begin && j < skip_end)) return;
  for (int c = 0; c < kb; ++c) {
    const int64_t r = k0 + c, p = ipiv[k0 + c];
    if (p != r) {
      const float2 a = A[j * n + r];
      A[j * n + r] = A[j * n + p];
      A[j * n + p] = a;
    }
  }
}

// Block row: U12 = L11^{-1} A12 (unit lower L11 = rows/cols k0..k0+kb of A), one thread
// per column j of B (B = A12 with leading dimension ldb, rows k0..k0+kb).
__global__ void lu_trsm_lower_kernel(const float2* __restrict__ L, int64_t ldl, int64_t k0, int kb,
                                     float2* B, int64_t ldb, int64_t ncols) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= ncols) return;
  float2 x[kNB];
  for (int r = 0; r < kb; ++r) x[r] = B[j * ldb + k0 + r];
  for (int r = 0; r < kb; ++r)
    for (int c = 0; c < r; ++c) {
      const float2 l = L[(k0 + c) * ldl + k0 + r];
      x[r].x -= l.x * x[c].x - l.y * x[c].y;
      x[r].y -= l.x * x[c].y + l.y * x[c].x;
    }
  for (int r = 0; r < kb; ++r) B[j * ldb + k0 + r] = x[r];
}

// Diagonal block of the backward substitution: x = U11^{-1} b (upper, non-unit), one thread
// per right-hand side.
__global__ void lu_trsm_upper_kernel(const float2* __restrict__ U, int64_t ldu, int64_t k0, int kb,
                                     float2* B, int64_t ldb, int64_t ncols) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= ncols) return;
  float2 x[kNB];
  for (int r = 0; r < kb; ++r) x[r] = B[j * ldb + k0 + r];
  for (int r = kb - 1; r >= 0; --r) {
    for (int c = r + 1; c < kb; ++c) {
      const float2 u = U[(k0 + c) * ldu + k0 + r];
      x[r].x -= u.x * x[c].x - u.y * x[c].y;
      x[r].y -= u.x * x[c].y + u.y * x[c].x;
    }
    x[r] = cdivf(x[r], U[(k0 + r) * ldu + k0 + r]);
  }
  for (int r = 0; r < kb; ++r) B[j * ldb + k0 + r] = x[r];
}

constexpr int kGB = 64;   // GEMM tile
// C[m x n] -= A[m x k] B[k x n] (complex FP32, column-major, k <= 32).
__global__ void __launch_bounds__(256)
cgemm_sub_kernel(int64_t m, int64_t n, int k, const float2* __restrict__ A, int64_t lda,
                 const float2* __restrict__ B, int64_t ldb, float2* C, int64_t ldc) {
  __shared__ float2 sA[kNB][kGB + 1];
  __shared__ float2 sB[kNB][kGB + 1];
  const int64_t i0 = (int64_t)blockIdx.x * kGB, j0 = (int64_t)blockIdx.y * kGB;
  const int tid = threadIdx.x;
  for (int t = tid; t < kNB * kGB; t += 256) {
    const int r = t % kGB, c = t / kGB;   // A: row i0 + r, column c
    sA[c][r] = (i0 + r < m && c < k) ? A[c * lda + i0 + r] : make_float2(0.f, 0.f);
    const int rb = t % kNB, cb = t / kNB;   // B: row rb, column j0 + cb
    sB[rb][cb] = (rb < k && j0 + cb < n) ? B[(j0 + cb) * ldb + rb] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int ti = tid % 16, tj = tid / 16;   // rows ti + 16 a, columns tj + 16 b
  float2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);
  for (int kk = 0; kk < k; ++kk) {
    float2 av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = sA[kk][ti + 16 * a];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = sB[kk][tj + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        acc[a][b].x = fmaf(av[a].x, bv[b].x, fmaf(-av[a].y, bv[b].y, acc[a][b].x));
        acc[a][b].y = fmaf(av[a].x, bv[b].y, fmaf(av[a].y, bv[b].x, acc[a][b].y));
      }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t i = i0 + ti + 16 * a;
    if (i >= m) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t j = j0 + tj + 16 * b;
      if (j < n) {
        float2 c = C[j * ldc + i];
        c.x -= acc[a][b].x;
        c.y -= acc[a][b].y;
        C[j * ldc + i] = c;
      }
    }
  }
}

}  // namespace

bem_status assemble32(bem_ctx* ctx, int nk, const double* kz_host, const double* coef_host,
                      float2* M, cudaStream_t s) {
  if (nk < 1 || nk > kMaxK) return fail(ctx, BEM_EINVAL, "assemble32: 1 <= nk <= 64");
  const int64_t n = ctx->geo.n;
  KList K;
  K.nk = nk;
  for (int k = 0; k < nk; ++k) {
    K.kr[k] = (float)kz_host[2 * k];
    K.kmi[k] = (float)(-kz_host[2 * k + 1]) * kLog2eF;
    K.ki[k] = (float)kz_host[2 * k + 1];
    K.cr[k] = (float)coef_host[2 * k];
    K.ci[k] = (float)coef_host[2 * k + 1];
  }
  // self terms of these wavenumbers (FP32 table in the small workspace)
  bem_status st = ensure_small(ctx, (size_t)nk * n * sizeof(float2) + 2 * nk * sizeof(double) + 256);
  if (st != BEM_OK) return st;
  double* zd = ctx->d_small;
  float* self32 = reinterpret_cast<float*>(ctx->d_small + 2 * nk + 32);
  st = cuda_check(ctx, cudaMemcpyAsync(zd, kz_host, 2 * nk * sizeof(double), cudaMemcpyHostToDevice, s),
                  "assemble32 copy");
  if (st != BEM_OK) return st;
  st = cuda_check(ctx, launch_self32(ctx, nk, zd, self32, s), "assemble32 self terms");
  if (st != BEM_OK) return st;
  assemble32_kernel<<<(unsigned)((n * n + 255) / 256), 256, 0, s>>>(
      ctx->geo, K, reinterpret_cast<const float2*>(self32), M, ctx->op);
  ctx->launches++;
  return cuda_check(ctx, cudaGetLastError(), "assemble32 kernel");
}

bem_status lu32(bem_ctx* ctx, float2* A, int64_t n, int* ipiv, cudaStream_t s) {
  for (int64_t k0 = 0; k0 < n; k0 += kNB) {
    const int kb = (int)std::min<int64_t>(kNB, n - k0);
    lu_panel_kernel<<<1, 1024, 0, s>>>(A, n, k0, kb, ipiv, ctx->d_status);
    lu_swap_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(A, n, n, k0, kb, ipiv, k0, k0 + kb);
    ctx->launches += 2;
    const int64_t rest = n - k0 - kb;
    if (rest > 0) {
      lu_trsm_lower_kernel<<<(unsigned)((rest + 127) / 128), 128, 0, s>>>(
          A, n, k0, kb, A + (k0 + kb) * n, n, rest);
      dim3 grid((unsigned)((rest + kGB - 1) / kGB), (unsigned)((rest + kGB - 1) / kGB));
      cgemm_sub_kernel<<<grid, 256, 0, s>>>(rest, rest, kb, A + k0 * n + k0 + kb, n,
                                             A + (k0 + kb) * n + k0, n,
                                             A + (k0 + kb) * n + k0 + kb, n);
      ctx->launches += 2;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(ctx, e, "lu32");
  }
  return BEM_OK;
}

bem_status lu32_solve(bem_ctx* ctx, const float2* LU, const int* ipiv, int64_t n, float2* B,
                      int64_t m, cudaStream_t s) {
  // row interchanges on the right-hand sides
  for (int64_t k0 = 0; k0 < n; k0 += kNB) {
    const int kb = (int)std::min<int64_t>(kNB, n - k0);
    lu_swap_kernel<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(B, n, m, k0, kb, ipiv, -1, -1);
    ctx->launches++;
  }
  // forward: unit lower, block by block
  for (int64_t k0 = 0; k0 < n; k0 += kNB) {
    const int kb = (int)std::min<int64_t>(kNB, n - k0);
    lu_trsm_lower_kernel<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(LU, n, k0, kb, B, n, m);
    const int64_t rest = n - k0 - kb;
    if (rest > 0) {
      dim3 grid((unsigned)((rest + kGB - 1) / kGB), (unsigned)((m + kGB - 1) / kGB));
      cgemm_sub_kernel<<<grid, 256, 0, s>>>(rest, m, kb, LU + k0 * n + k0 + kb, n, B + k0, n,
                                             B + k0 + kb, n);
    }
    ctx->launches += 2;
  }
  // backward: upper, last block first
  const int64_t nblk = (n + kNB - 1) / kNB;
  for (int64_t b = nblk - 1; b >= 0; --b) {
    const int64_t k0 = b * kNB;
    const int kb = (int)std::min<int64_t>(kNB, n - k0);
    lu_trsm_upper_kernel<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(LU, n, k0, kb, B, n, m);
    if (k0 > 0) {
      dim3 grid((unsigned)((k0 + kGB - 1) / kGB), (unsigned)((m + kGB - 1) / kGB));
      cgemm_sub_kernel<<<grid, 256, 0, s>>>(k0, m, kb, LU + k0 * n, n, B + k0, n, B, n);
    }
    ctx->launches += 2;
  }
  return cuda_check(ctx, cudaGetLastError(), "lu32_solve");
}

}  // namespace bem
