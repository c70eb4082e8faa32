// Matrix-free solves with the Schur complement of Algorithm 1 (Eq. linsyssim):
//     S X = B,   S = sum_j c_j A(z_j)   (c_j = w_j / (z_j - s) in the inverse power steps),
// by restarted GMRES on every column of B at once. S is never formed: each Arnoldi step
// applies it to the current block of basis vectors (one vector per column) with the
// node-summed fused kernel (one evaluation of the n^2 N entries serves all columns). The
// Arnoldi vectors are FP32; each new vector is orthogonalised against its column's
// previous ones by classical Gram-Schmidt run twice (dot products accumulated in FP64),
// the small Hessenberg least-squares problems are solved on the host by Givens rotations
// (FP64), and convergence is tested on the true residual ||B - S X|| / ||B|| per column
// at every restart.
#include <math.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "internal.h"

namespace bem {
namespace {

using cplx = std::complex<double>;

unsigned nb(int64_t count, int t = 256) { return (unsigned)((count + t - 1) / t); }

constexpr int kDotThreads = 256;

// h[i][c] = V_i[:, c]^H W[:, c] for i < k (block (i, c)), FP32 products, FP64 sums.
__global__ void __launch_bounds__(kDotThreads)
block_dots_kernel(const float2* __restrict__ Vb, const float2* __restrict__ W, int64_t n,
                  int nu, double2* __restrict__ h) {
  const int i = blockIdx.x, c = blockIdx.y;
  const float2* v = Vb + ((int64_t)i * nu + c) * n;
  const float2* w = W + (int64_t)c * n;
  double re = 0.0, im = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += kDotThreads) {
    const float2 a = v[r], b = w[r];
    re += (double)(a.x * b.x + a.y * b.y);
    im += (double)(a.x * b.y - a.y * b.x);
  }
  __shared__ double sr[kDotThreads], si[kDotThreads];
  sr[threadIdx.x] = re;
  si[threadIdx.x] = im;
  __syncthreads();
  for (int s = kDotThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sr[threadIdx.x] += sr[threadIdx.x + s];
      si[threadIdx.x] += si[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) h[(int64_t)i * nu + c] = make_double2(sr[0], si[0]);
}

// W[:, c] -= sum_{i < k} V_i[:, c] h[i][c]
__global__ void block_update_kernel(const float2* __restrict__ Vb, float2* __restrict__ W,
                                    int64_t n, int nu, int k, const double2* __restrict__ h) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * nu) return;
  const int c = (int)(t / n);
  const int64_t r = t % n;
  float2 acc = W[t];
  for (int i = 0; i < k; ++i) {
    const float2 v = Vb[((int64_t)i * nu + c) * n + r];
    const double2 hh = h[(int64_t)i * nu + c];
    const float hr = (float)hh.x, hi = (float)hh.y;
    acc.x -= v.x * hr - v.y * hi;
    acc.y -= v.x * hi + v.y * hr;
  }
  W[t] = acc;
}

// nrm[c] = ||W[:, c]|| (FP64 sums)
__global__ void __launch_bounds__(kDotThreads)
col_norms_kernel(const float2* __restrict__ W, int64_t n, double* __restrict__ nrm) {
  const int c = blockIdx.x;
  const float2* w = W + (int64_t)c * n;
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += kDotThreads) {
    const float2 a = w[r];
    s += (double)(a.x * a.x + a.y * a.y);
  }
  __shared__ double ss[kDotThreads];
  ss[threadIdx.x] = s;
  __syncthreads();
  for (int k = kDotThreads / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) ss[threadIdx.x] += ss[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) nrm[c] = sqrt(ss[0]);
}

// Out[:, c] = W[:, c] * scale[c]
__global__ void col_scale_kernel(const float2* __restrict__ W, int64_t n, int nu,
                                 const double* __restrict__ scale, float2* __restrict__ Out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * nu) return;
  const float f = (float)scale[t / n];
  const float2 a = W[t];
  Out[t] = make_float2(a.x * f, a.y * f);
}

// X[:, c] += sum_{i < k} V_i[:, c] y[i][c]
__global__ void block_combine_kernel(const float2* __restrict__ Vb, int64_t n, int nu, int k,
                                     const double2* __restrict__ y, float2* __restrict__ X) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * nu) return;
  const int c = (int)(t / n);
  const int64_t r = t % n;
  float2 acc = X[t];
  for (int i = 0; i < k; ++i) {
    const float2 v = Vb[((int64_t)i * nu + c) * n + r];
    const double2 yy = y[(int64_t)i * nu + c];
    const float yr = (float)yy.x, yi = (float)yy.y;
    acc.x += v.x * yr - v.y * yi;
    acc.y += v.x * yi + v.y * yr;
  }
  X[t] = acc;
}

// R = B - R (R holds S X on entry)
__global__ void residual_kernel(const float2* __restrict__ B, float2* __restrict__ R,
                                int64_t count) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const float2 b = B[t], r = R[t];
  R[t] = make_float2(b.x - r.x, b.y - r.y);
}

}  // namespace

size_t gmres_sum_work_bytes(bem_ctx* ctx, int nu, int restart) {
  const int64_t n = ctx->geo.n;
  const size_t blk = (size_t)n * nu * sizeof(float2);
  const size_t small = (size_t)(restart + 1) * nu * sizeof(double2);
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  return up((size_t)(restart + 1) * blk) + 2 * up(blk) + up(small) + up((size_t)nu * sizeof(double)) +
         up(mixed_sum_work_bytes(ctx, nu, false));
}

bem_status gmres_sum32(bem_ctx* ctx, const double* coef_host, const float2* B, float2* X, int nu,
                       double tol, int max_iter, int restart, void* work, cudaStream_t s,
                       int* iters_out, double* relres_host) {
  const int64_t n = ctx->geo.n;
  const size_t blk = (size_t)n * nu * sizeof(float2);
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  unsigned char* w = reinterpret_cast<unsigned char*>(work);
  float2* Vb = reinterpret_cast<float2*>(w);
  w += up((size_t)(restart + 1) * blk);
  float2* W = reinterpret_cast<float2*>(w);
  w += up(blk);
  float2* R = reinterpret_cast<float2*>(w);
  w += up(blk);
  double2* h = reinterpret_cast<double2*>(w);
  w += up((size_t)(restart + 1) * nu * sizeof(double2));
  double* nrm = reinterpret_cast<double*>(w);
  w += up((size_t)nu * sizeof(double));
  void* sum_work = w;
  const int64_t cnt = n * nu;

  std::vector<double> bnorm(nu), rn(nu), hn(nu);
  std::vector<double2> hh((size_t)(restart + 1) * nu);
  bem_status st = BEM_OK;
  auto sync_copy = [&](void* dst, const void* src, size_t bytes) {
    st = cuda_check(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s), "gmres copy");
    if (st == BEM_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), "gmres sync");
    return st == BEM_OK;
  };
  // ||B||
  col_norms_kernel<<<nu, kDotThreads, 0, s>>>(B, n, nrm);
  ctx->launches++;
  if (!sync_copy(bnorm.data(), nrm, nu * sizeof(double))) return st;
  cudaMemsetAsync(X, 0, blk, s);
  int total = 0;
  bool done = false;
  while (!done) {
    // R = B - S X (the true residual), its norms, V_0 = R / ||R||
    if (total == 0) {
      cudaMemcpyAsync(R, B, blk, cudaMemcpyDeviceToDevice, s);
    } else {
      if ((st = mixed_sum_apply(ctx, X, n, 0, false, nu, coef_host, R, sum_work, s)) != BEM_OK)
        return st;
      residual_kernel<<<nb(cnt), 256, 0, s>>>(B, R, cnt);
      ctx->launches++;
    }
    col_norms_kernel<<<nu, kDotThreads, 0, s>>>(R, n, nrm);
    ctx->launches++;
    if (!sync_copy(rn.data(), nrm, nu * sizeof(double))) return st;
    bool all = true;
    for (int c = 0; c < nu; ++c) {
      const double rel = bnorm[c] > 0 ? rn[c] / bnorm[c] : 0.0;
      if (relres_host) relres_host[c] = rel;
      if (rel > tol) all = false;
    }
    if (all || total >= max_iter) break;
    std::vector<double> inv(nu);
    for (int c = 0; c < nu; ++c) inv[c] = rn[c] > 0 ? 1.0 / rn[c] : 0.0;
    cudaMemcpyAsync(nrm, inv.data(), nu * sizeof(double), cudaMemcpyHostToDevice, s);
    col_scale_kernel<<<nb(cnt), 256, 0, s>>>(R, n, nu, nrm, Vb);
    ctx->launches++;
    // Arnoldi with Givens rotations per column
    std::vector<cplx> H((size_t)(restart + 1) * restart * nu, 0.0);   // H[(i * restart + k) * nu + c]
    std::vector<cplx> g((size_t)(restart + 1) * nu, 0.0), cs((size_t)restart * nu), sn((size_t)restart * nu);
    for (int c = 0; c < nu; ++c) g[c] = rn[c];
    int k = 0;
    for (; k < restart && total < max_iter; ++k, ++total) {
      float2* Vk = Vb + (size_t)k * n * nu;
      if ((st = mixed_sum_apply(ctx, Vk, n, 0, false, nu, coef_host, W, sum_work, s)) != BEM_OK)
        return st;
      for (int pass = 0; pass < 2; ++pass) {
        block_dots_kernel<<<dim3(k + 1, nu), kDotThreads, 0, s>>>(Vb, W, n, nu, h);
        block_update_kernel<<<nb(cnt), 256, 0, s>>>(Vb, W, n, nu, k + 1, h);
        ctx->launches += 2;
        if (!sync_copy(hh.data(), h, (size_t)(k + 1) * nu * sizeof(double2))) return st;
        for (int i = 0; i <= k; ++i)
          for (int c = 0; c < nu; ++c)
            H[((size_t)i * restart + k) * nu + c] +=
                cplx(hh[(size_t)i * nu + c].x, hh[(size_t)i * nu + c].y);
      }
      col_norms_kernel<<<nu, kDotThreads, 0, s>>>(W, n, nrm);
      ctx->launches++;
      if (!sync_copy(hn.data(), nrm, nu * sizeof(double))) return st;
      std::vector<double> inv(nu);
      for (int c = 0; c < nu; ++c) inv[c] = hn[c] > 0 ? 1.0 / hn[c] : 0.0;
      cudaMemcpyAsync(nrm, inv.data(), nu * sizeof(double), cudaMemcpyHostToDevice, s);
      col_scale_kernel<<<nb(cnt), 256, 0, s>>>(W, n, nu, nrm, Vb + (size_t)(k + 1) * n * nu);
      ctx->launches++;
      double worst = 0.0;
      for (int c = 0; c < nu; ++c) {
        H[((size_t)(k + 1) * restart + k) * nu + c] = hn[c];
        // previous rotations, then a new one zeroing H[k+1][k]
        for (int i = 0; i < k; ++i) {
          cplx& a = H[((size_t)i * restart + k) * nu + c];
          cplx& b = H[((size_t)(i + 1) * restart + k) * nu + c];
          const cplx cc = cs[(size_t)i * nu + c], ss = sn[(size_t)i * nu + c];
          const cplx ta = std::conj(cc) * a + std::conj(ss) * b;
          const cplx tb = -ss * a + cc * b;
          a = ta;
          b = tb;
        }
        cplx& a = H[((size_t)k * restart + k) * nu + c];
        cplx& b = H[((size_t)(k + 1) * restart + k) * nu + c];
        const double den = std::sqrt(std::norm(a) + std::norm(b));
        cplx cc = 1.0, ss = 0.0;
        if (den > 0) {
          cc = a / den;
          ss = b / den;
        }
        cs[(size_t)k * nu + c] = cc;
        sn[(size_t)k * nu + c] = ss;
        a = den;
        b = 0.0;
        const cplx gk = g[(size_t)k * nu + c];
        g[(size_t)k * nu + c] = std::conj(cc) * gk;
        g[(size_t)(k + 1) * nu + c] = -ss * gk;
        const double rel = bnorm[c] > 0 ? std::abs(g[(size_t)(k + 1) * nu + c]) / bnorm[c] : 0.0;
        worst = std::max(worst, rel);
      }
      if (worst <= 0.5 * tol) {   // estimated residual well below tol: form X
        ++k;
        ++total;
        break;
      }
    }
    // y = R^{-1} g (back substitution per column), X += V y
    std::vector<double2> y((size_t)k * nu);
    for (int c = 0; c < nu; ++c) {
      std::vector<cplx> yc(k);
      for (int i = k - 1; i >= 0; --i) {
        cplx acc = g[(size_t)i * nu + c];
        for (int m = i + 1; m < k; ++m) acc -= H[((size_t)i * restart + m) * nu + c] * yc[m];
        const cplx d = H[((size_t)i * restart + i) * nu + c];
        yc[i] = std::abs(d) > 0 ? acc / d : 0.0;
      }
      for (int i = 0; i < k; ++i) y[(size_t)i * nu + c] = make_double2(yc[i].real(), yc[i].imag());
    }
    if (k > 0) {
      cudaMemcpyAsync(h, y.data(), (size_t)k * nu * sizeof(double2), cudaMemcpyHostToDevice, s);
      block_combine_kernel<<<nb(cnt), 256, 0, s>>>(Vb, n, nu, k, h, X);
      ctx->launches++;
    }
    if (k == 0) done = true;
  }
  if (iters_out) *iters_out = total;
  return cuda_check(ctx, cudaGetLastError(), "gmres");
}

}  // namespace bem
