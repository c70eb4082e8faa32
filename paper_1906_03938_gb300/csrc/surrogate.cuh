// Surrogate network of the near-field correction: layout and per-thread evaluation.
//
// A multilayer perceptron 11 -> 64 -> 64 -> 64 -> 2 with tanh activations maps the canonical
// features of a near pair (its triangle's vertices in a frame attached to the collocation
// point, divided by the panel diameter h, then Re(k h) and Im(k h)) to the correction
// (A_near - A_7) / h of that pair. Parameters, one float array:
//   in_shift[11], in_scale[11]   features are standardised as (f - shift) * scale
//   W1[64][11], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[2][64], b4[2]
//   out_scale[2]                 the output is out_scale * (W4 h3 + b4) / (d / h)^7
//   feat_lo[11], feat_hi[11]     the training data's box: a pair whose features leave it
//                                (widened by 2 % of its width) takes the plain 8 x 8 rule
//                                (the inference kernel in near.cu checks it)
// d / h is the distance from the collocation point to the triangle's centroid in units of
// h, read off the features: the 7-point rule's error on a smooth integrand falls like
// (h / d)^7 (measured slope -7.5 over near pairs), so the network itself only has to
// represent a correction of nearly uniform size across all near pairs.
// The weights used for inference are rounded to BF16 (stored as floats); sums are FP32.
#pragma once

namespace bem {

constexpr int kNetIn = 11;
constexpr int kNetHid = 64;
constexpr int kNetOut = 2;
constexpr int kOffInShift = 0;
constexpr int kOffInScale = kOffInShift + kNetIn;
constexpr int kOffW1 = kOffInScale + kNetIn;
constexpr int kOffB1 = kOffW1 + kNetHid * kNetIn;
constexpr int kOffW2 = kOffB1 + kNetHid;
constexpr int kOffB2 = kOffW2 + kNetHid * kNetHid;
constexpr int kOffW3 = kOffB2 + kNetHid;
constexpr int kOffB3 = kOffW3 + kNetHid * kNetHid;
constexpr int kOffW4 = kOffB3 + kNetHid;
constexpr int kOffB4 = kOffW4 + kNetOut * kNetHid;
constexpr int kOffOutScale = kOffB4 + kNetOut;
constexpr int kOffFeatLo = kOffOutScale + kNetOut;
constexpr int kOffFeatHi = kOffFeatLo + kNetIn;
constexpr int kNetFloats = kOffFeatHi + kNetIn;
// first and one-past-last index of the trained parameters (the scalings are fitted from
// the data, not trained)
constexpr int kOffTrainBegin = kOffW1;
constexpr int kOffTrainEnd = kOffOutScale;

// (d / h)^7 from the raw features (the centroid of the three vertices in the pair's frame).
__device__ __forceinline__ float surrogate_decay(const float feat[kNetIn]) {
  const float cx = (feat[0] + feat[3] + feat[6]) * (1.f / 3.f);
  const float cy = (feat[1] + feat[4] + feat[7]) * (1.f / 3.f);
  const float cz = (feat[2] + feat[5] + feat[8]) * (1.f / 3.f);
  const float d2 = cx * cx + cy * cy + cz * cz;
  return d2 * d2 * d2 * sqrtf(d2);
}

// One evaluation per thread; every lane of a warp reads the same weight at the same time
// (broadcast loads through the read-only cache).
__device__ __forceinline__ float2 surrogate_eval(const float* __restrict__ net,
                                                 const float feat[kNetIn]) {
  float x[kNetIn];
#pragma unroll
  for (int i = 0; i < kNetIn; ++i)
    x[i] = (feat[i] - __ldg(net + kOffInShift + i)) * __ldg(net + kOffInScale + i);
  float h[kNetHid], g[kNetHid];
#pragma unroll
  for (int o = 0; o < kNetHid; ++o) {
    float a = __ldg(net + kOffB1 + o);
#pragma unroll
    for (int i = 0; i < kNetIn; ++i) a = fmaf(__ldg(net + kOffW1 + o * kNetIn + i), x[i], a);
    h[o] = tanhf(a);
  }
#pragma unroll 4
  for (int o = 0; o < kNetHid; ++o) {
    float a = __ldg(net + kOffB2 + o);
#pragma unroll
    for (int i = 0; i < kNetHid; ++i) a = fmaf(__ldg(net + kOffW2 + o * kNetHid + i), h[i], a);
    g[o] = tanhf(a);
  }
#pragma unroll 4
  for (int o = 0; o < kNetHid; ++o) {
    float a = __ldg(net + kOffB3 + o);
#pragma unroll
    for (int i = 0; i < kNetHid; ++i) a = fmaf(__ldg(net + kOffW3 + o * kNetHid + i), g[i], a);
    h[o] = tanhf(a);
  }
  const float inv_s = 1.f / surrogate_decay(feat);
  float out[kNetOut];
#pragma unroll
  for (int o = 0; o < kNetOut; ++o) {
    float a = __ldg(net + kOffB4 + o);
#pragma unroll
    for (int i = 0; i < kNetHid; ++i) a = fmaf(__ldg(net + kOffW4 + o * kNetHid + i), h[i], a);
    out[o] = a * __ldg(net + kOffOutScale + o) * inv_s;
  }
  return make_float2(out[0], out[1]);
}

}  // namespace bem
