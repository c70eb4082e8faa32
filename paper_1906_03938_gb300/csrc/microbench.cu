// Throughput microbenchmarks of the pipes that bound the hot path, and per-launch timing of
// the projection's main kernel. The results are the denominators of the roofline fractions
// the benchmark reports for the evaluation-bound kernels (FP64 FMA for the plain path,
// FP32 FMA and the MUFU transcendental unit for the mixed path).
#include <vector>

#include "f32x2.cuh"
#include "internal.h"

namespace bem {
namespace {

constexpr int kIters = 4096;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fma64_kernel(double* out, double seed) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = seed + threadIdx.x + k;
  const double m = 0.999999, c = 1e-7;
#pragma unroll 4
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == 12345.678) out[0] = s;   // keeps the loop alive, never true in practice
}

__global__ void __launch_bounds__(kThreads) fma32_kernel(float* out, float seed) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = seed + threadIdx.x + k;
  const float m = 0.9999f, c = 1e-4f;
#pragma unroll 4
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], m, c);
  }
  float s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == 12345.678f) out[0] = s;
}

// kind 0: ex2.approx, 1: sin.approx, 2: cos.approx, 3: rsqrt.approx (one MUFU op each)
template <int kKind>
__global__ void __launch_bounds__(kThreads) mufu_kernel(float* out, float seed) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1e-3f * (seed + threadIdx.x + k);
#pragma unroll 4
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float r;
      if (kKind == 0) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[k]));
      if (kKind == 1) asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[k]));
      if (kKind == 2) asm volatile("cos.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[k]));
      if (kKind == 3) asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[k]));
      a[k] = r;
    }
  }
  float s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == 12345.678f) out[0] = s;
}

// paired FP32 FMA (fma.rn.f32x2): 4 flops per instruction and thread
__global__ void __launch_bounds__(kThreads) fma32x2_kernel(float* out, float seed) {
  f2_t a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = f2(seed + threadIdx.x + k, seed - k);
  const f2_t m = f2dup(0.9999f), c = f2dup(1e-4f);
#pragma unroll 4
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma2(a[k], m, c);
  }
  float s = 0, x, y;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    f2split(a[k], x, y);
    s += x + y;
  }
  if (s == 12345.678f) out[0] = s;
}

// the fused kernel's polynomial e^{i phi} (sincos_poly2), two phases per call; the next
// phases depend on the results (one extra paired FMA per call)
__global__ void __launch_bounds__(kThreads) sincos_poly_kernel(float* out, float seed) {
  f2_t a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = f2(1e-3f * (seed + threadIdx.x + k), 0.5f + k);
  const f2_t m = f2dup(3.0f);
#pragma unroll 2
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      f2_t c, s, sg;
      sincos_poly2(a[k], c, s, sg);
      a[k] = fma2(c ^ sg, m, s);
    }
  }
  float s = 0, x, y;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    f2split(a[k], x, y);
    s += x + y;
  }
  if (s == 12345.678f) out[0] = s;
}

}  // namespace
}  // namespace bem

using namespace bem;

extern "C" bem_status bem_microbench(bem_ctx* ctx, int kind, double* ops_per_s) {
  if (!ctx || !ops_per_s || kind < 0 || kind > 7)
    return fail(ctx, BEM_EINVAL, "bem_microbench: bad argument");
  cudaSetDevice(ctx->device);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  bem_status st = ensure_small(ctx, 64);
  if (st != BEM_OK) return st;
  const int blocks = sms * 8;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, 0);
    switch (kind) {
      case 0: fma64_kernel<<<blocks, kThreads>>>(ctx->d_small, 1.0); break;
      case 1: fma32_kernel<<<blocks, kThreads>>>(reinterpret_cast<float*>(ctx->d_small), 1.0f); break;
      case 2: mufu_kernel<0><<<blocks, kThreads>>>(reinterpret_cast<float*>(ctx->d_small), 1.0f); break;
      case 3: mufu_kernel<1><<<blocks, kThreads>>>(reinterpret_cast<float*>(ctx->d_small), 1.0f); break;
      case 4: mufu_kernel<2><<<blocks, kThreads>>>(reinterpret_cast<float*>(ctx->d_small), 1.0f); break;
      case 5: mufu_kernel<3><<<blocks, kThreads>>>(reinterpret_cast<float*>(ctx->d_small), 1.0f); break;
      case 6: fma32x2_kernel<<<blocks, kThreads>>>(reinterpret_cast<float*>(ctx->d_small), 1.0f); break;
      default: sincos_poly_kernel<<<blocks, kThreads>>>(reinterpret_cast<float*>(ctx->d_small), 1.0f); break;
    }
    cudaEventRecord(e1, 0);
    ctx->launches++;
    st = cuda_check(ctx, cudaEventSynchronize(e1), "bem_microbench");
    if (st != BEM_OK) break;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != BEM_OK) return st;
  // flops for the FMA kinds (2 per FMA lane), operations for the MUFU kinds, phases for
  // the polynomial sine / cosine
  const double per = kind <= 1 ? 2.0 : (kind == 6 ? 4.0 : (kind == 7 ? 2.0 : 1.0));
  const double ops = (double)blocks * kThreads * kIters * 8 * per;
  *ops_per_s = ops / (best * 1e-3);
  return BEM_OK;
}

extern "C" bem_status bem_set_timing(bem_ctx* ctx, int enable) {
  if (!ctx) return BEM_EINVAL;
  cudaSetDevice(ctx->device);
  ctx->timing = enable != 0;
  if (ctx->timing && ctx->ev.empty()) {
    ctx->ev.resize(2 * kMaxTimed);
    for (auto& e : ctx->ev)
      if (cudaEventCreate(&e) != cudaSuccess) return fail(ctx, BEM_ECUDA, "bem_set_timing: event creation failed");
  }
  ctx->n_timed = 0;
  return BEM_OK;
}

extern "C" bem_status bem_kernel_times(bem_ctx* ctx, double* ms_out, int max_out, int* count) {
  if (!ctx || !count) return BEM_EINVAL;
  cudaSetDevice(ctx->device);
  const int n = ctx->n_timed < max_out ? ctx->n_timed : max_out;
  for (int t = 0; t < n; ++t) {
    bem_status st = cuda_check(ctx, cudaEventSynchronize(ctx->ev[2 * t + 1]), "bem_kernel_times");
    if (st != BEM_OK) return st;
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->ev[2 * t], ctx->ev[2 * t + 1]);
    if (ms_out) ms_out[t] = ms;
  }
  *count = n;
  ctx->n_timed = 0;
  return BEM_OK;
}
