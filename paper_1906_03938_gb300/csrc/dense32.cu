// Dense FP32 matrices of the operator and their LU factorisation.
//
// * assemble32_kernel: M = sum_k c_k A(kappa_k) as a dense n x n complex64 matrix
//   (column-major), one thread per entry, FP32 evaluation with MUFU ex2/sin/cos as in the
//   mixed projection, self terms from an FP32 table. With one wavenumber this is A(sigma),
//   the matrix the residual-inverse refinement factorises; with the contour nodes and
//   c_j = w_j / (z_j - s) it is the Schur complement S = sum_j B_j / (z_j - s) of the
//   inverse power step (Algorithm 1, Eq. linsyssim).
// * lu32: right-looking blocked LU with partial pivoting in two levels. Panels of 256
//   columns are factorised 32 columns at a time: each column's pivot is searched by all
//   blocks (partial maxima, then one block picks the row, swaps it in and publishes it),
//   the multipliers and the rank-1 update of the 32-column sub-panel run over all rows;
//   the rest of the 256-column panel gets the sub-panel's interchanges, a triangular solve
//   and a CUDA-core complex GEMM (k = 32). Then the panel's interchanges go to the other
//   columns, U12 = L11^{-1} A12 is solved in 32-row blocks and the trailing matrix is
//   updated with k = 256 by cuBLAS (a plain complex FP32 GEMM, FP32 emulated on the
//   tensor cores where the library offers it). lu32_solve applies the factors to a block
//   of right-hand sides. FP32 is enough here: both users only need an approximate inverse
//   (the refinement's fixed point is defined by FP64 residuals).
#include <cublas_v2.h>
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <climits>
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

constexpr int kNB = 32;       // sub-panel width (and block size of the triangular solves)
constexpr int kPanel = 256;   // panel width of the trailing updates
constexpr int kPivBlock = 256;
constexpr int kPivParts = 1024;   // most blocks of a pivot search

// Blocks of a pivot search over rows [r0, n): one per 256 rows, at most kPivParts.
inline int piv_parts(int64_t rows) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(kPivParts, (rows + kPivBlock - 1) / kPivBlock));
}

__device__ __forceinline__ void piv_better(float& bv, int& bi, float v, int i) {
  if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
}

// block-wide arg-max (largest |re| + |im|, smallest row on ties) -> partials[blockIdx.x]
__device__ __forceinline__ void piv_block_reduce(float bv, int bi, float* pval, int* pidx) {
  __shared__ float sv[kPivBlock / 32];
  __shared__ int si[kPivBlock / 32];
  for (int off = 16; off > 0; off >>= 1) {
    const float ov = __shfl_down_sync(0xffffffffu, bv, off);
    const int oi = __shfl_down_sync(0xffffffffu, bi, off);
    piv_better(bv, bi, ov, oi);
  }
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (lane == 0) { sv[w] = bv; si[w] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = sv[0];
    int j = si[0];
    for (int q = 1; q < kPivBlock / 32; ++q) piv_better(b, j, sv[q], si[q]);
    pval[blockIdx.x] = b;
    pidx[blockIdx.x] = j;
  }
}

// partial maxima of column col over rows [col, n) (the first column of a sub-panel)
__global__ void __launch_bounds__(kPivBlock)
lu_colmax_kernel(const float2* __restrict__ A, int64_t n, int64_t col, float* pval, int* pidx) {
  float bv = -1.f;
  int bi = INT_MAX;
  for (int64_t r = col + blockIdx.x * (int64_t)kPivBlock + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * kPivBlock) {
    const float2 v = A[col * n + r];
    piv_better(bv, bi, fabsf(v.x) + fabsf(v.y), (int)r);
  }
  piv_block_reduce(bv, bi, pval, pidx);
}

// One block: the pivot row p of column col from the partial maxima; ipiv[col] = p; rows col
// and p exchanged in the sub-panel's columns [j0, jend).
__global__ void __launch_bounds__(32)
lu_pivot_kernel(float2* A, int64_t n, int64_t col, int64_t j0, int64_t jend,
                const float* __restrict__ pval, const int* __restrict__ pidx, int parts,
                int* ipiv, int* status) {
  float bv = -1.f;
  int bi = INT_MAX;
  for (int q = threadIdx.x; q < parts; q += 32) piv_better(bv, bi, pval[q], pidx[q]);
  for (int off = 16; off > 0; off >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, bv, off);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
    piv_better(bv, bi, ov, oi);
  }
  const int64_t p = (bi == INT_MAX) ? col : bi;
  if (threadIdx.x == 0) {
    ipiv[col] = (int)p;
    if (!(bv > 0.f)) atomicOr(status, kStatusNotSPD);   // exactly singular column
  }
  if (p != col)
    for (int64_t c = j0 + threadIdx.x; c < jend; c += 32) {
      const float2 a = A[c * n + col], b = A[c * n + p];
      A[c * n + col] = b;
      A[c * n + p] = a;
    }
}

// Rows r > col: multiplier l = A[r, col] / A[col, col] stored in place, columns (col, jend)
// updated by -l * A[col, c]; then the partial maxima of the updated column col + 1.
__global__ void __launch_bounds__(kPivBlock)
lu_colupdate_kernel(float2* A, int64_t n, int64_t col, int64_t jend, float* pval, int* pidx) {
  __shared__ float2 prow[kNB];
  const int w = (int)(jend - col);   // columns col .. jend-1 of the pivot row
  if (threadIdx.x < w) prow[threadIdx.x] = A[(col + threadIdx.x) * n + col];
  __syncthreads();
  const float2 dinv = cdivf(make_float2(1.f, 0.f), prow[0]);
  float bv = -1.f;
  int bi = INT_MAX;
  for (int64_t r = col + 1 + blockIdx.x * (int64_t)kPivBlock + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * kPivBlock) {
    const float2 m = cmulf(A[col * n + r], dinv);
    A[col * n + r] = m;
    for (int j = 1; j < w; ++j) {
      const float2 u = prow[j];
      float2 v = A[(col + j) * n + r];
      v.x -= m.x * u.x - m.y * u.y;
      v.y -= m.x * u.y + m.y * u.x;
      A[(col + j) * n + r] = v;
      if (j == 1) piv_better(bv, bi, fabsf(v.x) + fabsf(v.y), (int)r);
    }
  }
  if (w > 1) piv_block_reduce(bv, bi, pval, pidx);
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

// Real representation of the complex panel L (m x k, column-major, leading dimension ld):
// Ah (2m x 2k, leading dimension 2m) with rows (2i, 2i+1) = (Re, Im) of row i and columns
// [Re L | -Im L] over [Im L | Re L], so that Ah [Re B; Im B] gives the interleaved
// (Re, Im) rows of L B.
__global__ void lu_real_rep_kernel(const float2* __restrict__ L, int64_t ld, int64_t m, int k,
                                   float* __restrict__ Ah) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= m * k) return;
  const int64_t i = t % m;
  const int l = (int)(t / m);
  const float2 v = L[(int64_t)l * ld + i];
  const int64_t m2 = 2 * m;
  Ah[(int64_t)l * m2 + 2 * i] = v.x;
  Ah[(int64_t)l * m2 + 2 * i + 1] = v.y;
  Ah[(int64_t)(k + l) * m2 + 2 * i] = -v.y;
  Ah[(int64_t)(k + l) * m2 + 2 * i + 1] = v.x;
}

// Planar copy of the complex block U (k x nc, leading dimension ld): Bp (2k x nc, leading
// dimension 2k) = [Re U; Im U].
__global__ void lu_planar_kernel(const float2* __restrict__ U, int64_t ld, int k, int64_t nc,
                                 float* __restrict__ Bp) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)k * nc) return;
  const int l = (int)(t % k);
  const int64_t j = t / k;
  const float2 v = U[j * ld + l];
  Bp[j * 2 * k + l] = v.x;
  Bp[j * 2 * k + k + l] = v.y;
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

void release_cublas(bem_ctx* ctx) {
  if (ctx->cublas) cublasDestroy(static_cast<cublasHandle_t>(ctx->cublas));
  ctx->cublas = nullptr;
}

namespace {

// C[m x nc] -= A[m x k] B[k x nc] (complex FP32, column-major) by cuBLAS on stream s: the
// complex product as one real GEMM of the real representation of A (2m x 2k) with the
// planar [Re B; Im B] (2k x nc) into the interleaved rows of C (2m x nc, leading dimension
// 2 ldc), the same 8 flops per complex multiply-add, FP32 products emulated on the tensor
// cores by BF16x9 (FP32 accuracy); the plain FP32 GEMM where the library lacks the
// emulation. work: (2m + nc) 2k floats.
bem_status cublas_update(bem_ctx* ctx, int64_t m, int64_t nc, int k, const float2* A,
                         int64_t lda, const float2* B, int64_t ldb, float2* C, int64_t ldc,
                         float* work, cudaStream_t s) {
  if (!ctx->cublas) {
    cublasHandle_t h = nullptr;
    if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS)
      return fail(ctx, BEM_ECUDA, "lu32: cublasCreate failed");
    cublasSetEmulationStrategy(h, CUBLAS_EMULATION_STRATEGY_EAGER);
    ctx->cublas = h;
  }
  cublasHandle_t h = static_cast<cublasHandle_t>(ctx->cublas);
  if (cublasSetStream(h, s) != CUBLAS_STATUS_SUCCESS)
    return fail(ctx, BEM_ECUDA, "lu32: cublasSetStream failed");
  float* Ah = work;
  float* Bp = work + 4 * m * (int64_t)k;
  lu_real_rep_kernel<<<(unsigned)((m * k + 255) / 256), 256, 0, s>>>(A, lda, m, k, Ah);
  lu_planar_kernel<<<(unsigned)((k * nc + 255) / 256), 256, 0, s>>>(B, ldb, k, nc, Bp);
  ctx->launches += 2;
  const float alpha = -1.f, beta = 1.f;
  cublasStatus_t cs = cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_N, (int)(2 * m), (int)nc, 2 * k,
                                   &alpha, Ah, CUDA_R_32F, (int)(2 * m), Bp, CUDA_R_32F, 2 * k,
                                   &beta, reinterpret_cast<float*>(C), CUDA_R_32F,
                                   (int)(2 * ldc), CUBLAS_COMPUTE_32F_EMULATED_16BFX9,
                                   CUBLAS_GEMM_DEFAULT);
  if (cs == CUBLAS_STATUS_NOT_SUPPORTED || cs == CUBLAS_STATUS_INVALID_VALUE)
    cs = cublasSgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, (int)(2 * m), (int)nc, 2 * k, &alpha, Ah,
                     (int)(2 * m), Bp, 2 * k, &beta, reinterpret_cast<float*>(C), (int)(2 * ldc));
  if (cs != CUBLAS_STATUS_SUCCESS)
    return fail(ctx, BEM_ECUDA, "lu32: GEMM failed (cuBLAS status " + std::to_string((int)cs) + ")");
  return BEM_OK;
}

}  // namespace

bem_status lu32(bem_ctx* ctx, float2* A, int64_t n, int* ipiv, cudaStream_t s) {
  if (!ctx->d_piv_val) {
    if (cudaMalloc(&ctx->d_piv_val, kPivParts * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&ctx->d_piv_idx, kPivParts * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, BEM_ENOMEM, "lu32: pivot workspace allocation failed");
    }
  }
  float* pval = ctx->d_piv_val;
  int* pidx = ctx->d_piv_idx;
  // GEMM operands in real form: (2 n + n) 2 kPanel floats at most
  const size_t lu_work = (size_t)3 * n * 2 * kPanel * sizeof(float);
  if (lu_work > ctx->lu_work_bytes) {
    cudaFree(ctx->d_lu_work);
    ctx->d_lu_work = nullptr;
    ctx->lu_work_bytes = 0;
    if (cudaMalloc(&ctx->d_lu_work, lu_work) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, BEM_ENOMEM, "lu32: GEMM workspace allocation failed");
    }
    ctx->lu_work_bytes = lu_work;
  }
  for (int64_t K0 = 0; K0 < n; K0 += kPanel) {
    const int kb = (int)std::min<int64_t>(kPanel, n - K0);
    for (int64_t J0 = K0; J0 < K0 + kb; J0 += kNB) {
      const int jb = (int)std::min<int64_t>(kNB, K0 + kb - J0);
      const int64_t jend = J0 + jb;
      // the sub-panel A[J0:n, J0:jend), one column at a time
      int parts = piv_parts(n - J0);
      lu_colmax_kernel<<<parts, kPivBlock, 0, s>>>(A, n, J0, pval, pidx);
      ctx->launches++;
      for (int64_t col = J0; col < jend; ++col) {
        lu_pivot_kernel<<<1, 32, 0, s>>>(A, n, col, J0, jend, pval, pidx, parts, ipiv,
                                          ctx->d_status);
        const int next = piv_parts(n - col - 1);
        lu_colupdate_kernel<<<next, kPivBlock, 0, s>>>(A, n, col, jend, pval, pidx);
        parts = next;
        ctx->launches += 2;
      }
      // the rest of the panel: interchanges, block row, update (k = 32)
      if (kb > jb)
        lu_swap_kernel<<<(unsigned)((kb + 127) / 128), 128, 0, s>>>(A + K0 * n, n, kb, J0, jb, ipiv,
                                                                  J0 - K0, jend - K0);
      const int64_t rin = K0 + kb - jend;
      if (rin > 0) {
        lu_trsm_lower_kernel<<<(unsigned)((rin + 127) / 128), 128, 0, s>>>(A, n, J0, jb,
                                                                           A + jend * n, n, rin);
        const int64_t below = n - jend;
        if (below > 0) {
          dim3 grid((unsigned)((below + kGB - 1) / kGB), (unsigned)((rin + kGB - 1) / kGB));
          cgemm_sub_kernel<<<grid, 256, 0, s>>>(below, rin, jb, A + J0 * n + jend, n,
                                                 A + jend * n + J0, n, A + jend * n + jend, n);
        }
        ctx->launches += 2;
      }
      if (kb > jb) ctx->launches++;
    }
    // the panel's interchanges in every other column
    lu_swap_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(A, n, n, K0, kb, ipiv, K0, K0 + kb);
    ctx->launches++;
    const int64_t rest = n - K0 - kb;
    if (rest > 0) {
      // U12 = L11^{-1} A12, 32 rows at a time
      for (int64_t b0 = K0; b0 < K0 + kb; b0 += kNB) {
        const int bb = (int)std::min<int64_t>(kNB, K0 + kb - b0);
        lu_trsm_lower_kernel<<<(unsigned)((rest + 127) / 128), 128, 0, s>>>(
            A, n, b0, bb, A + (K0 + kb) * n, n, rest);
        ctx->launches++;
        const int64_t below = K0 + kb - (b0 + bb);
        if (below > 0) {
          dim3 grid((unsigned)((below + kGB - 1) / kGB), (unsigned)((rest + kGB - 1) / kGB));
          cgemm_sub_kernel<<<grid, 256, 0, s>>>(below, rest, bb, A + b0 * n + b0 + bb, n,
                                                 A + (K0 + kb) * n + b0, n,
                                                 A + (K0 + kb) * n + b0 + bb, n);
          ctx->launches++;
        }
      }
      // trailing matrix, k = kb
      const bem_status st = cublas_update(ctx, rest, rest, kb, A + K0 * n + K0 + kb, n,
                                          A + (K0 + kb) * n + K0, n, A + (K0 + kb) * n + K0 + kb,
                                          n, ctx->d_lu_work, s);
      if (st != BEM_OK) return st;
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
