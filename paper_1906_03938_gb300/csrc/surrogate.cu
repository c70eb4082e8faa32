// Surrogate network of the near-field correction: initialisation, inference, and training
// with the library's own forward and backward kernels (FP32) and Adam.
//
// The network (layout in surrogate.cuh) maps a near pair's canonical features to
// (A_near - A_7) / h. Training minimises the mean over samples of the squared error at the
// network's output, i.e. in units of out_scale / (d / h)^7 (relative to the size the
// correction has at that distance), summed over the two outputs. One block handles 64 samples: the forward pass keeps the three
// hidden layers in shared memory, the backward pass forms the block's gradient with sums
// over its samples in a fixed order; block gradients are then added in block order and
// Adam updates the trained parameters (deterministic). The standardisation of the features
// and the output scale are fitted from the training data (mean and standard deviation),
// not trained. Inference (the mixed projection, bem_surrogate_forward) uses a copy whose
// weights are rounded to BF16.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "surrogate.cuh"

namespace bem {
namespace {

constexpr int kGS = 64;          // samples per block of the gradient kernel
constexpr int kPad = kNetHid + 1;

__device__ __forceinline__ double uniform_u01(uint64_t seed, uint64_t idx) {
  uint64_t z = seed + (idx + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1.0p-53;
}

// Xavier-uniform weights, zero biases, identity standardisation and output scale.
__global__ void init_kernel(float* __restrict__ net, uint64_t seed) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kNetFloats) return;
  float v = 0.f;
  int fan_in = 0, fan_out = 0;
  if (t >= kOffW1 && t < kOffB1) { fan_in = kNetIn; fan_out = kNetHid; }
  else if (t >= kOffW2 && t < kOffB2) { fan_in = kNetHid; fan_out = kNetHid; }
  else if (t >= kOffW3 && t < kOffB3) { fan_in = kNetHid; fan_out = kNetHid; }
  else if (t >= kOffW4 && t < kOffB4) { fan_in = kNetHid; fan_out = kNetOut; }
  if (fan_in) {
    const float lim = sqrtf(6.f / (float)(fan_in + fan_out));
    v = (float)(2.0 * uniform_u01(seed, (uint64_t)t) - 1.0) * lim;
  } else if ((t >= kOffInScale && t < kOffInScale + kNetIn) ||
             (t >= kOffOutScale && t < kOffOutScale + kNetOut)) {
    v = 1.f;
  } else if (t >= kOffFeatLo && t < kOffFeatLo + kNetIn) {
    v = -INFINITY;   // no box until the scalings are fitted to training data
  } else if (t >= kOffFeatHi && t < kOffFeatHi + kNetIn) {
    v = INFINITY;
  }
  net[t] = v;
}

// Inference copy: weights and biases rounded to BF16, scalings kept.
__global__ void round_bf16_kernel(const float* __restrict__ net, float* __restrict__ inf) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kNetFloats) return;
  const float v = net[t];
  inf[t] = (t >= kOffTrainBegin && t < kOffTrainEnd) ? __bfloat162float(__float2bfloat16(v)) : v;
}

__global__ void forward_kernel(const float* __restrict__ net, const float* __restrict__ feat,
                               int64_t count, float* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  float f[kNetIn];
#pragma unroll
  for (int i = 0; i < kNetIn; ++i) f[i] = feat[t * kNetIn + i];
  const float2 o = surrogate_eval(net, f);
  out[2 * t] = o.x;
  out[2 * t + 1] = o.y;
}

// Mean and standard deviation of column c of the features (c < 11) or of the network's
// targets (c = 11, 12: target times (d / h)^7): one block per column, fixed-order FP64
// sums. Sets in_shift / in_scale (1 / std, or 1 for a constant column) and out_scale (std,
// or 1), and the features' range (the training box of the quadrature fallback).
__global__ void fit_scaling_kernel(const float* __restrict__ feat, const float* __restrict__ target,
                                   int64_t count, float* __restrict__ net) {
  __shared__ double s1[256], s2[256];
  __shared__ float slo[256], shi[256];
  const int c = blockIdx.x;
  double a = 0.0, b = 0.0;
  float lo = INFINITY, hi = -INFINITY;
  for (int64_t t = threadIdx.x; t < count; t += blockDim.x) {
    double v;
    if (c < kNetIn) {
      v = feat[t * kNetIn + c];
      lo = fminf(lo, (float)v);
      hi = fmaxf(hi, (float)v);
    } else {   // the network's own target: (A_near - A_7) / h times (d / h)^7
      float f[kNetIn];
      for (int q = 0; q < kNetIn; ++q) f[q] = feat[t * kNetIn + q];
      v = (double)target[t * kNetOut + (c - kNetIn)] * (double)surrogate_decay(f);
    }
    a += v;
    b += v * v;
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  slo[threadIdx.x] = lo;
  shi[threadIdx.x] = hi;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s1[threadIdx.x] += s1[threadIdx.x + w];
      s2[threadIdx.x] += s2[threadIdx.x + w];
      slo[threadIdx.x] = fminf(slo[threadIdx.x], slo[threadIdx.x + w]);
      shi[threadIdx.x] = fmaxf(shi[threadIdx.x], shi[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double mean = s1[0] / (double)count;
    const double var = fmax(s2[0] / (double)count - mean * mean, 0.0);
    const double sd = sqrt(var);
    if (c < kNetIn) {
      net[kOffInShift + c] = (float)mean;
      net[kOffInScale + c] = sd > 1e-6 ? (float)(1.0 / sd) : 1.f;
      net[kOffFeatLo + c] = slo[0];
      net[kOffFeatHi + c] = shi[0];
    } else {
      net[kOffOutScale + (c - kNetIn)] = sd > 0.0 ? (float)sd : 1.f;
    }
  }
}

size_t grad_smem_bytes() {
  return (size_t)(kGS * kNetIn + 3 * kGS * kPad + 2 * kGS * kPad + kGS * kNetOut +
                  kNetHid * kNetIn + 2 * kNetHid * kNetHid + kNetOut * kNetHid) *
         sizeof(float);
}

// Block gradient and loss of samples idx(b, s) = (a * (start + b * 64 + s) + c) mod count
// for s < 64 with start + b * 64 + s < end (an affine permutation of the data set; a is
// coprime to count and a * count stays below 2^63).
__global__ void __launch_bounds__(256)
grad_kernel(const float* __restrict__ net, const float* __restrict__ feat,
            const float* __restrict__ target, int64_t count, int64_t start, int64_t end,
            int64_t perm_a, int64_t perm_c, float inv_n, float* __restrict__ gpart,
            float* __restrict__ lpart) {
  extern __shared__ float sm[];
  float* xs = sm;                              // [64][11]
  float* h1 = xs + kGS * kNetIn;               // [64][65]
  float* h2 = h1 + kGS * kPad;
  float* h3 = h2 + kGS * kPad;
  float* dA = h3 + kGS * kPad;                 // [64][65]
  float* dB = dA + kGS * kPad;
  float* dz = dB + kGS * kPad;                 // [64][2]
  float* W1 = dz + kGS * kNetOut;              // [64][11]
  float* W2 = W1 + kNetHid * kNetIn;           // [64][64]
  float* W3 = W2 + kNetHid * kNetHid;
  float* W4 = W3 + kNetHid * kNetHid;          // [2][64]
  __shared__ float red[256];
  __shared__ float sdec[kGS];                  // (d / h)^7 of each sample
  const int tid = threadIdx.x;
  const int64_t first = start + (int64_t)blockIdx.x * kGS;
  const int64_t left = end - first;
  const int ns = left <= 0 ? 0 : (left < kGS ? (int)left : kGS);
  for (int t = tid; t < kNetHid * kNetIn; t += 256) W1[t] = net[kOffW1 + t];
  for (int t = tid; t < kNetHid * kNetHid; t += 256) {
    W2[t] = net[kOffW2 + t];
    W3[t] = net[kOffW3 + t];
  }
  for (int t = tid; t < kNetOut * kNetHid; t += 256) W4[t] = net[kOffW4 + t];
  for (int t = tid; t < kGS * kNetIn; t += 256) {
    const int s = t / kNetIn, i = t % kNetIn;
    float v = 0.f;
    if (s < ns) {
      const int64_t idx = (int64_t)(((uint64_t)perm_a * (uint64_t)(first + s) + (uint64_t)perm_c) %
                                    (uint64_t)count);
      v = (feat[idx * kNetIn + i] - net[kOffInShift + i]) * net[kOffInScale + i];
    }
    xs[t] = v;
  }
  if (tid < kGS) {
    float dec = 1.f;
    if (tid < ns) {
      const int64_t idx = (int64_t)(((uint64_t)perm_a * (uint64_t)(first + tid) + (uint64_t)perm_c) %
                                    (uint64_t)count);
      float f[kNetIn];
      for (int q = 0; q < kNetIn; ++q) f[q] = feat[idx * kNetIn + q];
      dec = surrogate_decay(f);
    }
    sdec[tid] = dec;
  }
  __syncthreads();
  const int s = tid % kGS, og = tid / kGS;   // lanes over samples, 4 groups of outputs
  // forward
  for (int o = og; o < kNetHid; o += 4) {
    float a = net[kOffB1 + o];
    for (int i = 0; i < kNetIn; ++i) a = fmaf(W1[o * kNetIn + i], xs[s * kNetIn + i], a);
    h1[s * kPad + o] = tanhf(a);
  }
  __syncthreads();
  for (int o = og; o < kNetHid; o += 4) {
    float a = net[kOffB2 + o];
    for (int i = 0; i < kNetHid; ++i) a = fmaf(W2[o * kNetHid + i], h1[s * kPad + i], a);
    h2[s * kPad + o] = tanhf(a);
  }
  __syncthreads();
  for (int o = og; o < kNetHid; o += 4) {
    float a = net[kOffB3 + o];
    for (int i = 0; i < kNetHid; ++i) a = fmaf(W3[o * kNetHid + i], h2[s * kPad + i], a);
    h3[s * kPad + o] = tanhf(a);
  }
  __syncthreads();
  float lsum = 0.f;
  if (og < kNetOut) {
    const int o = og;
    float a = net[kOffB4 + o];
    for (int i = 0; i < kNetHid; ++i) a = fmaf(W4[o * kNetHid + i], h3[s * kPad + i], a);
    float d = 0.f;
    if (s < ns) {
      const int64_t idx = (int64_t)(((uint64_t)perm_a * (uint64_t)(first + s) + (uint64_t)perm_c) %
                                    (uint64_t)count);
      // the error at the network's output, in units of out_scale / (d/h)^7:
      // (pred - t) (d/h)^7 / osc = z - t (d/h)^7 / osc
      const float osc = net[kOffOutScale + o];
      const float diff = a - target[idx * kNetOut + o] * sdec[s] / osc;
      lsum = diff * diff;
      d = 2.f * diff * inv_n;
    }
    dz[s * kNetOut + o] = d;
  }
  red[tid] = lsum;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  if (tid == 0) lpart[blockIdx.x] = red[0] * inv_n;
  float* g = gpart + (size_t)blockIdx.x * kNetFloats;
  // output layer
  for (int t = tid; t < kNetOut * kNetHid; t += 256) {
    const int o = t / kNetHid, i = t % kNetHid;
    float a = 0.f;
    for (int q = 0; q < kGS; ++q) a = fmaf(dz[q * kNetOut + o], h3[q * kPad + i], a);
    g[kOffW4 + t] = a;
  }
  if (tid < kNetOut) {
    float a = 0.f;
    for (int q = 0; q < kGS; ++q) a += dz[q * kNetOut + tid];
    g[kOffB4 + tid] = a;
  }
  // d3 = (W4^T dz) * (1 - h3^2)
  for (int i = og; i < kNetHid; i += 4) {
    float a = 0.f;
    for (int o = 0; o < kNetOut; ++o) a = fmaf(W4[o * kNetHid + i], dz[s * kNetOut + o], a);
    const float hv = h3[s * kPad + i];
    dA[s * kPad + i] = a * (1.f - hv * hv);
  }
  __syncthreads();
  // layer 3: gradient, then d2 = (W3^T d3) * (1 - h2^2)
  for (int t = tid; t < kNetHid * kNetHid; t += 256) {
    const int o = t / kNetHid, i = t % kNetHid;
    float a = 0.f;
    for (int q = 0; q < kGS; ++q) a = fmaf(dA[q * kPad + o], h2[q * kPad + i], a);
    g[kOffW3 + t] = a;
  }
  if (tid < kNetHid) {
    float a = 0.f;
    for (int q = 0; q < kGS; ++q) a += dA[q * kPad + tid];
    g[kOffB3 + tid] = a;
  }
  for (int i = og; i < kNetHid; i += 4) {
    float a = 0.f;
    for (int o = 0; o < kNetHid; ++o) a = fmaf(W3[o * kNetHid + i], dA[s * kPad + o], a);
    const float hv = h2[s * kPad + i];
    dB[s * kPad + i] = a * (1.f - hv * hv);
  }
  __syncthreads();
  // layer 2: gradient, then d1 = (W2^T d2) * (1 - h1^2) (into dA, free again)
  for (int t = tid; t < kNetHid * kNetHid; t += 256) {
    const int o = t / kNetHid, i = t % kNetHid;
    float a = 0.f;
    for (int q = 0; q < kGS; ++q) a = fmaf(dB[q * kPad + o], h1[q * kPad + i], a);
    g[kOffW2 + t] = a;
  }
  if (tid < kNetHid) {
    float a = 0.f;
    for (int q = 0; q < kGS; ++q) a += dB[q * kPad + tid];
    g[kOffB2 + tid] = a;
  }
  __syncthreads();
  for (int i = og; i < kNetHid; i += 4) {
    float a = 0.f;
    for (int o = 0; o < kNetHid; ++o) a = fmaf(W2[o * kNetHid + i], dB[s * kPad + o], a);
    const float hv = h1[s * kPad + i];
    dA[s * kPad + i] = a * (1.f - hv * hv);
  }
  __syncthreads();
  // layer 1
  for (int t = tid; t < kNetHid * kNetIn; t += 256) {
    const int o = t / kNetIn, i = t % kNetIn;
    float a = 0.f;
    for (int q = 0; q < kGS; ++q) a = fmaf(dA[q * kPad + o], xs[q * kNetIn + i], a);
    g[kOffW1 + t] = a;
  }
  if (tid < kNetHid) {
    float a = 0.f;
    for (int q = 0; q < kGS; ++q) a += dA[q * kPad + tid];
    g[kOffB1 + tid] = a;
  }
  // the standardisation and the output scale are not trained
  if (tid < kOffTrainBegin) g[tid] = 0.f;
  if (tid < kNetFloats - kOffTrainEnd) g[kOffTrainEnd + tid] = 0.f;
}

// grad = sum of the block gradients in block order; loss likewise (into loss[0]).
__global__ void reduce_grad_kernel(const float* __restrict__ gpart, const float* __restrict__ lpart,
                                   int nb, float* __restrict__ grad, float* __restrict__ loss) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < kNetFloats) {
    float a = 0.f;
    for (int b = 0; b < nb; ++b) a += gpart[(size_t)b * kNetFloats + t];
    grad[t] = a;
  }
  if (t == 0) {
    float a = 0.f;
    for (int b = 0; b < nb; ++b) a += lpart[b];
    loss[0] += a;
  }
}

// Adam (Kingma & Ba) on the trained parameters.
__global__ void adam_kernel(float* __restrict__ net, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ grad, float lr, float bc1, float bc2) {
  const int t = kOffTrainBegin + blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kOffTrainEnd) return;
  const float g = grad[t];
  const float mt = 0.9f * m[t] + 0.1f * g;
  const float vt = 0.999f * v[t] + 0.001f * g * g;
  m[t] = mt;
  v[t] = vt;
  net[t] -= lr * (mt / bc1) / (sqrtf(vt / bc2) + 1e-8f);
}

// Device buffers of the network: master weights, inference copy, Adam moments, gradient.
struct NetBufs {
  float *master, *inf, *m, *v, *grad, *loss;
};

NetBufs net_bufs(bem_ctx* ctx) {
  NetBufs b;
  b.master = ctx->d_net;
  b.inf = ctx->d_net + kNetFloats;
  b.m = ctx->d_net + 2 * kNetFloats;
  b.v = ctx->d_net + 3 * kNetFloats;
  b.grad = ctx->d_net + 4 * kNetFloats;
  b.loss = ctx->d_net + 5 * kNetFloats;
  return b;
}

bem_status ensure_net(bem_ctx* ctx) {
  if (ctx->d_net) return BEM_OK;
  ctx->net_floats = 5 * kNetFloats + 64;
  if (cudaMalloc(&ctx->d_net, ctx->net_floats * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    ctx->d_net = nullptr;
    return fail(ctx, BEM_ENOMEM, "surrogate: device allocation failed");
  }
  return BEM_OK;
}

bem_status refresh_inference(bem_ctx* ctx, cudaStream_t s) {
  const NetBufs b = net_bufs(ctx);
  round_bf16_kernel<<<(kNetFloats + 255) / 256, 256, 0, s>>>(b.master, b.inf);
  ctx->launches++;
  ctx->net_ready = true;
  return cuda_check(ctx, cudaGetLastError(), "surrogate kernels");
}

int64_t gcd64(int64_t a, int64_t b) {
  while (b) {
    const int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

// grad/loss of samples [start, end) of the permutation (a, c) into the buffers
bem_status batch_grad(bem_ctx* ctx, const float* feat, const float* target, int64_t count,
                      int64_t start, int64_t end, int64_t pa, int64_t pc, float* gpart, float* lpart,
                      cudaStream_t s) {
  const NetBufs b = net_bufs(ctx);
  const int nb = (int)((end - start + kGS - 1) / kGS);
  const size_t smem = grad_smem_bytes();
  bem_status st = cuda_check(ctx, cudaFuncSetAttribute(grad_kernel,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)smem),
                             "surrogate attribute");
  if (st != BEM_OK) return st;
  grad_kernel<<<nb, 256, smem, s>>>(b.master, feat, target, count, start, end, pa, pc,
                                    1.f / (float)(end - start), gpart, lpart);
  reduce_grad_kernel<<<(kNetFloats + 255) / 256, 256, 0, s>>>(gpart, lpart, nb, b.grad, b.loss);
  ctx->launches += 2;
  return cuda_check(ctx, cudaGetLastError(), "surrogate kernels");
}

}  // namespace
}  // namespace bem

using namespace bem;

extern "C" {

int bem_surrogate_size(void) { return kNetFloats; }

bem_status bem_surrogate_init(bem_ctx* ctx, uint64_t seed, void* stream) {
  if (!ctx) return BEM_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  bem_status st = ensure_net(ctx);
  if (st != BEM_OK) return st;
  const NetBufs b = net_bufs(ctx);
  init_kernel<<<(kNetFloats + 255) / 256, 256, 0, s>>>(b.master, seed);
  ctx->launches++;
  st = cuda_check(ctx, cudaMemsetAsync(b.m, 0, 2 * kNetFloats * sizeof(float), s), "surrogate init");
  if (st != BEM_OK) return st;
  return refresh_inference(ctx, s);
}

bem_status bem_surrogate_set(bem_ctx* ctx, const float* params_host, int64_t count, void* stream) {
  if (!ctx) return BEM_EINVAL;
  if (!params_host || count != kNetFloats)
    return fail(ctx, BEM_EINVAL, "bem_surrogate_set: need bem_surrogate_size() floats");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  bem_status st = ensure_net(ctx);
  if (st != BEM_OK) return st;
  const NetBufs b = net_bufs(ctx);
  st = cuda_check(ctx, cudaMemcpyAsync(b.master, params_host, kNetFloats * sizeof(float),
                                       cudaMemcpyHostToDevice, s), "bem_surrogate_set copy");
  if (st == BEM_OK)
    st = cuda_check(ctx, cudaMemsetAsync(b.m, 0, 2 * kNetFloats * sizeof(float), s), "surrogate set");
  if (st == BEM_OK) st = refresh_inference(ctx, s);
  if (st == BEM_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), "bem_surrogate_set");
  return st;
}

bem_status bem_surrogate_get(bem_ctx* ctx, int which, float* params_host, int64_t count,
                             void* stream) {
  if (!ctx) return BEM_EINVAL;
  if (!params_host || count != kNetFloats || (which != 0 && which != 1))
    return fail(ctx, BEM_EINVAL, "bem_surrogate_get: need bem_surrogate_size() floats, which 0/1");
  if (!ctx->net_ready) return fail(ctx, BEM_ESTATE, "bem_surrogate_get: no network");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const NetBufs b = net_bufs(ctx);
  bem_status st = cuda_check(ctx, cudaMemcpyAsync(params_host, which ? b.inf : b.master,
                                                  kNetFloats * sizeof(float),
                                                  cudaMemcpyDeviceToHost, s),
                             "bem_surrogate_get copy");
  if (st == BEM_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), "bem_surrogate_get");
  return st;
}

bem_status bem_surrogate_forward(bem_ctx* ctx, const float* feat_dev, int64_t count,
                                 float* out_dev, void* stream) {
  if (!ctx) return BEM_EINVAL;
  if (!feat_dev || !out_dev || count < 1)
    return fail(ctx, BEM_EINVAL, "bem_surrogate_forward: need features, output, count >= 1");
  if (!ctx->net_ready) return fail(ctx, BEM_ESTATE, "bem_surrogate_forward: no network");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  forward_kernel<<<(unsigned)((count + 127) / 128), 128, 0, s>>>(net_bufs(ctx).inf, feat_dev, count,
                                                                 out_dev);
  ctx->launches++;
  return cuda_check(ctx, cudaGetLastError(), "surrogate kernels");
}

bem_status bem_surrogate_grad(bem_ctx* ctx, const float* feat_dev, const float* target_dev,
                              int64_t count, float* grad_dev, double* loss_host, void* stream) {
  if (!ctx) return BEM_EINVAL;
  if (!feat_dev || !target_dev || count < 1 || !grad_dev)
    return fail(ctx, BEM_EINVAL, "bem_surrogate_grad: need features, targets, gradient, count");
  if (!ctx->net_ready) return fail(ctx, BEM_ESTATE, "bem_surrogate_grad: no network");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = (int)((count + kGS - 1) / kGS);
  bem_status st = ensure_scratch(ctx, ((size_t)nb * kNetFloats + nb) * sizeof(float));
  if (st != BEM_OK) return st;
  float* gpart = reinterpret_cast<float*>(ctx->d_scratch);
  float* lpart = gpart + (size_t)nb * kNetFloats;
  const NetBufs b = net_bufs(ctx);
  st = cuda_check(ctx, cudaMemsetAsync(b.loss, 0, sizeof(float), s), "surrogate grad");
  if (st == BEM_OK) st = batch_grad(ctx, feat_dev, target_dev, count, 0, count, 1, 0, gpart, lpart, s);
  if (st == BEM_OK)
    st = cuda_check(ctx, cudaMemcpyAsync(grad_dev, b.grad, kNetFloats * sizeof(float),
                                         cudaMemcpyDeviceToDevice, s), "surrogate grad");
  float l = 0.f;
  if (st == BEM_OK)
    st = cuda_check(ctx, cudaMemcpyAsync(&l, b.loss, sizeof(float), cudaMemcpyDeviceToHost, s),
                    "surrogate grad");
  if (st == BEM_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), "surrogate grad");
  if (st == BEM_OK && loss_host) *loss_host = l;
  return st;
}

bem_status bem_surrogate_train(bem_ctx* ctx, const float* feat_dev, const float* target_dev,
                               int64_t count, int epochs, int batch, double lr, int fit_scaling,
                               uint64_t seed, double* loss_host, void* stream) {
  if (!ctx) return BEM_EINVAL;
  if (!feat_dev || !target_dev || count < 1 || epochs < 1 || batch < 1 || !(lr > 0.0))
    return fail(ctx, BEM_EINVAL, "bem_surrogate_train: bad arguments");
  if (!ctx->net_ready) return fail(ctx, BEM_ESTATE, "bem_surrogate_train: no network (init first)");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t B = std::min<int64_t>(count, batch);
  const int nb = (int)((B + kGS - 1) / kGS);
  bem_status st = ensure_scratch(ctx, ((size_t)nb * kNetFloats + nb) * sizeof(float));
  if (st != BEM_OK) return st;
  float* gpart = reinterpret_cast<float*>(ctx->d_scratch);
  float* lpart = gpart + (size_t)nb * kNetFloats;
  const NetBufs b = net_bufs(ctx);
  if (fit_scaling) {
    fit_scaling_kernel<<<kNetIn + kNetOut, 256, 0, s>>>(feat_dev, target_dev, count, b.master);
    ctx->launches++;
  }
  static const int64_t primes[] = {1000003, 999983, 1000033, 999979, 1000037, 999961, 1000039};
  const int64_t steps = (count + B - 1) / B;
  int64_t t_adam = 0;
  std::vector<float> losses(epochs);
  for (int e = 0; e < epochs && st == BEM_OK; ++e) {
    // affine permutation of the data set for this epoch
    int64_t pa = 1;
    for (int q = 0; q < 7; ++q) {
      const int64_t cand = primes[(q + e) % 7] % count;
      if (cand > 0 && gcd64(cand, count) == 1) {
        pa = cand;
        break;
      }
    }
    const int64_t pc = (int64_t)((seed * 0x9E3779B97F4A7C15ull + (uint64_t)e * 0xBF58476D1CE4E5B9ull) %
                                 (uint64_t)count);
    st = cuda_check(ctx, cudaMemsetAsync(b.loss, 0, sizeof(float), s), "surrogate train");
    for (int64_t k = 0; k < steps && st == BEM_OK; ++k) {
      const int64_t start = k * B, end = std::min(count, start + B);
      st = batch_grad(ctx, feat_dev, target_dev, count, start, end, pa, pc, gpart, lpart, s);
      if (st != BEM_OK) break;
      ++t_adam;
      const float bc1 = 1.f - powf(0.9f, (float)t_adam), bc2 = 1.f - powf(0.999f, (float)t_adam);
      // learning rate decayed geometrically from lr to lr / 100 over the run
      const float lr_t = (float)(lr * pow(0.01, (double)(t_adam - 1) / (double)(epochs * steps)));
      adam_kernel<<<(kOffTrainEnd - kOffTrainBegin + 255) / 256, 256, 0, s>>>(
          b.master, b.m, b.v, b.grad, lr_t, bc1, bc2);
      ctx->launches++;
    }
    if (st == BEM_OK)
      st = cuda_check(ctx, cudaMemcpyAsync(&losses[e], b.loss, sizeof(float), cudaMemcpyDeviceToHost, s),
                      "surrogate train");
    if (st == BEM_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), "surrogate train");
    if (loss_host) loss_host[e] = losses[e] / (double)steps;
  }
  if (st == BEM_OK) st = refresh_inference(ctx, s);
  if (st == BEM_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), "surrogate train");
  return st;
}

}  // extern "C"
