// Residuals A(lambda) x and A'(lambda) x in double-FP32 ("float-float") arithmetic, for the
// iterations of the eigenpair refinement (the accuracy of an eigenpair is
// ||T(lambda) u|| / ||u||, Section 4). This GPU's FP64 pipe runs at about 1/65 of its FP32
// pipe, and the FP64 residual spends ~77 FP64 instructions per quadrature point on sqrt,
// exp, sincos and a division; here every point is evaluated with pairs of FP32 numbers
// (hi + lo, ~48 significant bits; Dekker's and Knuth's error-free sums and products, with
// FMA for the exact product error), so that each entry carries a relative error of about
// 1e-13, far below the 1e-8 residuals the refinement drives to and certifies. The final
// residuals reported by the refinement are still computed by the FP64 kernel.
//
// Per quadrature point (single layer, Eq. GreenFun): d = x_i - y_lq and r^2 in pairs; r and
// 1/r from the MUFU rsqrt seed and one Newton correction in pairs; the phase Re(k) r reduced
// by pi/32 in three parts (Cody and Waite) with the table of cos, sin(j pi/32) (Tang's
// table-driven method) and short Taylor series of the remainder; e^{-Im(k) r} reduced in
// base 2 by 1/32 with the table of 2^(j/32) and a Taylor series. Both A and its
// k-derivative A' (kernel i e^{ikr}/(4 pi)) come from the same evaluation.
#include <math.h>

#include "ff_tables.cuh"
#include "internal.h"

namespace bem {
namespace {

struct FF {
  float h, l;
};

// Knuth's two-sum and the fast two-sum (|a| >= |b|); Dekker's product error by FMA. The
// _rn intrinsics are never contracted into FMAs by the compiler.
__device__ __forceinline__ FF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ FF fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const FF s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ FF ff_neg(FF a) { return {-a.h, -a.l}; }
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ FF ff_mulf(FF a, float b) {
  const float p = __fmul_rn(a.h, b);
  float e = fmaf(a.h, b, -p);
  e = fmaf(a.l, b, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ FF ff_from(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ double ff_to(FF a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ FF ff_sqr(FF a) {   // a^2 (the lo^2 term is below the pair's rounding)
  const float p = __fmul_rn(a.h, a.h);
  float e = fmaf(a.h, a.h, -p);
  e = fmaf(2.f * a.h, a.l, e);
  return fast_two_sum(p, e);
}

// 1/6 as an FP32 pair
constexpr float kSixthHi = 0.166666672f;
constexpr float kSixthLo = -4.96705388e-09f;

struct Tables {
  float trig[64][4];   // cos hi, cos lo, sin hi, sin lo of j pi / 32
  float exp2[32][2];   // 2^(j / 32) hi, lo
};

// (cos phi, sin phi), phi >= 0 (below 2^11 pi / 32 = 201): phi = j pi/32 + delta,
// |delta| <= pi/64, cos/sin(j pi/32) from the table, cos/sin(delta) by Taylor series (the
// leading terms in pairs, the tails in FP32, each tail below 1e-14 in absolute error).
__device__ __forceinline__ void ff_cossin(FF phi, const Tables& T, FF& co, FF& si) {
  using namespace ff;
  const float t = __fmul_rn(phi.h, kInvPi32);
  const float tb = __fadd_rn(t, 12582912.f);
  const float jf = __fsub_rn(tb, 12582912.f);
  const int j = __float_as_int(tb) & 63;
  // delta = phi - jf (P1 + P2 + P3): jf P1 is exact and phi.h - jf P1 exact (Sterbenz)
  const float a = fmaf(-jf, kP1, phi.h);
  const FF p2 = {__fmul_rn(jf, kP2), fmaf(jf, kP2, -__fmul_rn(jf, kP2))};
  const FF s = two_sum(a, -p2.h);
  const FF d = fast_two_sum(s.h, __fadd_rn(s.l, __fsub_rn(phi.l, __fadd_rn(p2.l, jf * kP3))));
  // cos and sin of the remainder
  const FF d2 = ff_sqr(d);                 // delta^2
  const float u = d2.h;
  // sin d = d - d^3/6 + d^5/120 - d^7/5040: d^3/6 in pairs, the rest in FP32
  const FF d3 = ff_mul(d2, d);
  const FF s3 = ff_mul(d3, FF{-kSixthHi, -kSixthLo});
  const float stail = d.h * u * u * (1.f / 120.f - u * (1.f / 5040.f));
  FF sd = ff_add(d, s3);
  sd = fast_two_sum(sd.h, __fadd_rn(sd.l, stail));
  // cos d = 1 - d^2/2 + d^4/24 - d^6/720: the first two terms in pairs
  const FF c2 = two_sum(1.f, -0.5f * d2.h);
  const float ctail = u * u * (1.f / 24.f - u * (1.f / 720.f));
  const FF cd = fast_two_sum(c2.h, __fadd_rn(c2.l, __fadd_rn(-0.5f * d2.l, ctail)));
  const FF cj = {T.trig[j][0], T.trig[j][1]}, sj = {T.trig[j][2], T.trig[j][3]};
  co = ff_add(ff_mul(cj, cd), ff_neg(ff_mul(sj, sd)));
  si = ff_add(ff_mul(sj, cd), ff_mul(cj, sd));
}

// e^x for |x| below ~80: x log2(e) = k + j/32 + f, |f| <= 1/64; 2^(j/32) from the table,
// e^{f ln 2} by Taylor series (1 + g + g^2/2 in pairs, g^3/6 .. g^5/120 in FP32), then the
// exact scaling by 2^k.
__device__ __forceinline__ FF ff_exp(FF x, const Tables& T) {
  using namespace ff;
  const FF t = ff_mul(x, FF{kLog2eHi, kLog2eLo});
  const float tb = __fadd_rn(__fmul_rn(t.h, 32.f), 12582912.f);
  const float mf = __fsub_rn(tb, 12582912.f);   // m = rint(32 t)
  const int m = __float_as_int(tb) - 0x4B400000;
  const int k = m >> 5, jj = m & 31;
  const FF f = fast_two_sum(__fsub_rn(t.h, mf * (1.f / 32.f)), t.l);   // exact first part
  const FF g = ff_mul(f, FF{kLn2Hi, kLn2Lo});
  const FF g2 = ff_sqr(g);
  const float tail = g2.h * g.h * (1.f / 6.f + g.h * (1.f / 24.f + g.h * (1.f / 120.f)));
  FF e = two_sum(1.f, g.h);
  e = fast_two_sum(e.h, __fadd_rn(e.l, __fadd_rn(g.l, __fadd_rn(0.5f * g2.l, tail))));
  e = ff_add(e, FF{0.5f * g2.h, 0.f});
  e = ff_mul(e, FF{T.exp2[jj][0], T.exp2[jj][1]});
  const float sc = __int_as_float((k + 127) << 23);
  return {e.h * sc, e.l * sc};
}

constexpr int kRows = 128;
constexpr int kChunk = 64;

// R_c = A(lambda_c) x_c (off-diagonal part plus the self term prefilled in R), and with
// kDeriv also Rd_c = A'(lambda_c) x_c; one thread per row, columns staged in shared memory.
template <bool kDeriv>
__global__ void __launch_bounds__(kRows)
residual_ff_kernel(Geometry g, const double* __restrict__ lam, const double* __restrict__ X,
                   int64_t ldx, double* __restrict__ R, double* __restrict__ Rd) {
  __shared__ Tables T;
  __shared__ float sP[7][3][2][kChunk];   // quadrature points, pairs
  __shared__ float sW[7][2][kChunk];      // weights / 4 pi, pairs
  __shared__ float sX[4][kChunk];         // x_l: re hi, re lo, im hi, im lo
  const int64_t n = g.n;
  const int c = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * kRows + threadIdx.x;
  for (int t = threadIdx.x; t < 64 * 4; t += kRows) (&T.trig[0][0])[t] = (&ff::kTrigTable[0][0])[t];
  for (int t = threadIdx.x; t < 32 * 2; t += kRows) (&T.exp2[0][0])[t] = (&ff::kExp2Table[0][0])[t];
  const FF kr = ff_from(lam[2 * c]), kin = ff_neg(ff_from(lam[2 * c + 1]));   // -Im k
  const double2* x = reinterpret_cast<const double2*>(X) + (int64_t)c * ldx;
  FF xi[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  if (i < n)
    for (int d = 0; d < 3; ++d) xi[d] = ff_from(g.cx[d * n + i]);
  FF ar = {0.f, 0.f}, ai = ar, dr = ar, di = ar;   // row sums of A x and A' x
  for (int64_t l0 = 0; l0 < n; l0 += kChunk) {
    __syncthreads();
    for (int t = threadIdx.x; t < 7 * kChunk; t += kRows) {
      const int q = t / kChunk, lc = t % kChunk;
      const int64_t l = l0 + lc;
      const bool ok = l < n;
      for (int d = 0; d < 3; ++d) {
        const FF v = ff_from(ok ? g.qp[(7 * d + q) * n + l] : 0.0);
        sP[q][d][0][lc] = v.h;
        sP[q][d][1][lc] = v.l;
      }
      const FF w = ff_from(ok ? g.qw[q * n + l] : 0.0);
      sW[q][0][lc] = w.h;
      sW[q][1][lc] = w.l;
    }
    for (int t = threadIdx.x; t < kChunk; t += kRows) {
      const int64_t l = l0 + t;
      const double2 v = l < n ? x[l] : make_double2(0.0, 0.0);
      const FF re = ff_from(v.x), im = ff_from(v.y);
      sX[0][t] = re.h; sX[1][t] = re.l; sX[2][t] = im.h; sX[3][t] = im.l;
    }
    __syncthreads();
    if (i >= n) continue;
    const int lim = (int)((n - l0) < kChunk ? (n - l0) : kChunk);
    for (int lc = 0; lc < lim; ++lc) {
      if (l0 + lc == i) continue;   // the self term is in R already
      FF er = {0.f, 0.f}, ei = er, edr = er, edi = er;   // the entry of A (and of A')
#pragma unroll 1
      for (int q = 0; q < 7; ++q) {
        FF d2[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const FF s = two_sum(xi[d].h, -sP[q][d][0][lc]);
          const FF dd = fast_two_sum(s.h, __fadd_rn(s.l, __fsub_rn(xi[d].l, sP[q][d][1][lc])));
          d2[d] = ff_sqr(dd);
        }
        const FF r2 = ff_add(ff_add(d2[0], d2[1]), d2[2]);
        // r = sqrt(r2) and 1/r: MUFU seed, one Newton correction each in pairs
        float y0;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(r2.h));
        const float s0 = __fmul_rn(r2.h, y0);
        const float res = __fadd_rn(fmaf(-s0, s0, r2.h), r2.l);
        const FF r = fast_two_sum(s0, __fmul_rn(__fmul_rn(res, y0), 0.5f));
        const float p = __fmul_rn(r.h, y0);
        const float qerr = fmaf(r.h, y0, -p) + r.l * y0;
        const float dlt = __fsub_rn(__fsub_rn(1.f, p), qerr);
        const FF rinv = fast_two_sum(y0, __fmul_rn(y0, dlt));
        FF co, si;
        ff_cossin(ff_mul(kr, r), T, co, si);
        const FF ex = ff_exp(ff_mul(kin, r), T);
        const FF amp = ff_mul(FF{sW[q][0][lc], sW[q][1][lc]}, ex);   // W e^{-Im k r}
        const FF aA = ff_mul(amp, rinv);
        er = ff_add(er, ff_mul(aA, co));
        ei = ff_add(ei, ff_mul(aA, si));
        if (kDeriv) {   // i W e^{i k r}: (-sin, cos)
          edr = ff_add(edr, ff_neg(ff_mul(amp, si)));
          edi = ff_add(edi, ff_mul(amp, co));
        }
      }
      const FF xr = {sX[0][lc], sX[1][lc]}, xim = {sX[2][lc], sX[3][lc]};
      ar = ff_add(ar, ff_add(ff_mul(er, xr), ff_neg(ff_mul(ei, xim))));
      ai = ff_add(ai, ff_add(ff_mul(er, xim), ff_mul(ei, xr)));
      if (kDeriv) {
        dr = ff_add(dr, ff_add(ff_mul(edr, xr), ff_neg(ff_mul(edi, xim))));
        di = ff_add(di, ff_add(ff_mul(edr, xim), ff_mul(edi, xr)));
      }
    }
  }
  if (i < n) {
    const double2 xv = x[i];
    double2* Rc = reinterpret_cast<double2*>(R) + (int64_t)c * n;
    const double2 sd = Rc[i];   // A_ii(lambda_c), written by the self-term kernel
    Rc[i] = make_double2(ff_to(ar) + (sd.x * xv.x - sd.y * xv.y),
                         ff_to(ai) + (sd.x * xv.y + sd.y * xv.x));
    if (kDeriv) {
      double2* Rdc = reinterpret_cast<double2*>(Rd) + (int64_t)c * n;
      const double2 sdd = Rdc[i];
      Rdc[i] = make_double2(ff_to(dr) + (sdd.x * xv.x - sdd.y * xv.y),
                            ff_to(di) + (sdd.x * xv.y + sdd.y * xv.x));
    }
  }
}

}  // namespace

cudaError_t launch_apply_ff(bem_ctx* ctx, int m, const double* lam_dev, const double* X,
                            int64_t ldx, double* R, double* Rd, cudaStream_t s) {
  if (!op_single(ctx->op)) {   // the general operator keeps the FP64 kernels
    cudaError_t e = launch_apply_percol64(ctx, m, lam_dev, X, ldx, R, false, s);
    if (e == cudaSuccess && Rd) e = launch_apply_percol64(ctx, m, lam_dev, X, ldx, Rd, true, s);
    return e;
  }
  const int64_t n = ctx->geo.n;
  cudaError_t e = launch_self_at(ctx, m, lam_dev, R, false, s);
  if (e == cudaSuccess && Rd) e = launch_self_at(ctx, m, lam_dev, Rd, true, s);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((n + kRows - 1) / kRows), (unsigned)m);
  if (Rd)
    residual_ff_kernel<true><<<grid, kRows, 0, s>>>(ctx->geo, lam_dev, X, ldx, R, Rd);
  else
    residual_ff_kernel<false><<<grid, kRows, 0, s>>>(ctx->geo, lam_dev, X, ldx, R, nullptr);
  ctx->launches++;
  if (near_active(ctx)) {
    e = launch_near_percol64(ctx, m, lam_dev, X, ldx, R, false, s);
    if (e == cudaSuccess && Rd) e = launch_near_percol64(ctx, m, lam_dev, X, ldx, Rd, true, s);
    return e;
  }
  return cudaGetLastError();
}

}  // namespace bem
