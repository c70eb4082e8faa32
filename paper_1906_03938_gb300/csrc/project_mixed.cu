// Mixed-precision fused assembly + projection (Section 3, Eq. RR_approx) on GB300.
//
// mixed_apply_kernel computes Y_j = A(z_j) V without storing A(z_j):
//  * a work unit is one 128-row tile of A, a group of G <= 4 contour nodes and a range of
//    16-column K-blocks (the column range is split when that balances the grid);
//  * 16 evaluation warps compute each 128 x 16 block of entries in FP32 for the G nodes
//    (7-point rule: one rsqrt per quadrature point shared by the nodes, then ex2, sin and
//    cos on the MUFU unit per node; the self term from the FP32 table on the diagonal),
//    with coordinates taken relative to the tile's first centroid, and write them as four
//    BF16 planes (Re/Im x hi/lo) into shared memory in the tensor core's canonical K-major
//    layout;
//  * one producer warp copies the matching K-block of the prepared BF16 basis planes
//    (four planes [Vr|Vi], [Vr_lo|Vi_lo], [-Vi|Vr], [-Vi_lo|Vr_lo]) with a bulk TMA copy
//    and stages the block's column geometry (FP64 -> tile-relative FP32) and self terms;
//  * one MMA warp issues, per node, six tcgen05 BF16 MMAs (M = 128, N = 2 C, K = 16)
//    that add Ar_hi[Vr|Vi] + Ar_hi[Vr_lo|Vi_lo] + Ar_lo[Vr|Vi] + Ai_hi[-Vi|Vr]
//    + Ai_hi[-Vi_lo|Vr_lo] + Ai_lo[-Vi|Vr] into an FP32 accumulator [Yr | Yi] in TMEM
//    (the split-precision "BF16x3" complex product);
//  * two shared-memory stages overlap evaluation, copies and MMAs (mbarriers; every wait
//    is bounded and a timeout aborts the block cleanly with an error status);
//  * the evaluation warps finally read the accumulators from TMEM and store the FP32
//    partial Y of the unit.
// mixed_pair_kernel is the same evaluation and contraction for units of one node (bases of
// more than 128 columns) whose nodes come in twin pairs: a cluster of two CTAs per twin
// pair, each evaluating half of every block for both nodes (see its own description).
// mixed_vhy_tc_kernel (BF16x3 on the tensor core, reading the same basis planes, one CTA
// per node, row part and quadrant of column chunks), then mixed_vhy_reduce_kernel,
// form Bhat_j = w_j V^H (sum over column splits of Y_j) with a fixed summation order.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "f32x2.cuh"
#include "internal.h"
#include "sm100.cuh"

namespace bem {
namespace {

using namespace sm100;

constexpr int kBM = 128;            // rows per tile (MMA M)
constexpr int kBK = 16;             // columns per K-block (MMA K)
constexpr int kStages = 2;
constexpr int kEvalWarps = 16;
constexpr int kEvalThreads = 32 * kEvalWarps;
constexpr int kThreads = 32 * (2 + kEvalWarps);
constexpr int kMaxG = 4;
constexpr int kPlaneBytes = kBM * kBK * 2;   // one BF16 plane of a 128 x 16 block: 4 KB
constexpr uint32_t kHalfPlane = kBM * (kBK / 2) * 2;   // its 8-column half: 2 KB
constexpr uint32_t kWaitLimit = kStageWaitDefault;   // polls (64 ns sleeps) before giving up
constexpr float kLog2e = 1.4426950408889634f;
// Quadrature points (of 7) per entry whose sine and cosine the fused kernel evaluates by
// the FMA-pipe polynomials rather than on the MUFU unit, by unit shape: units of several
// nodes (shared rsqrt, twin nodes sharing sine and cosine) and units of one node.
constexpr int kPolyPointsMulti = 1;
constexpr int kPolyPointsSingle = 1;
constexpr int kPolyPointsMax = 4;

struct MixedParams {
  int64_t n;          // unknowns
  int N;              // nodes
  int nu;             // basis columns
  int nup;            // nu rounded up to a multiple of 8
  int C;              // basis columns per MMA chunk (N of the MMA = 2 C)
  int nchunks;        // nup / C
  int G;              // nodes per unit
  int nG;             // node groups
  int nK;             // K-blocks
  int S;              // column splits
  int n_pad;          // rows rounded up to 128
  const double* cx;   // FP64 centroids, SoA
  const double* qp;   // FP64 quadrature points, q-major SoA
  const double* qw;   // FP64 weights / 4 pi
  const float2* self32;   // FP32 complex self terms, node-major
  const float* pack32;    // packed FP32 hi/lo panel geometry (64 floats per panel)
  const double* z;    // FP64 complex nodes
  const int* order;   // node schedule: slot -> node (| kTwinBit on the first of a twin pair)
  // node-summed mode (sum != 0): Y = sum_j c_j A(z_j) X_j into one accumulator per unit;
  // the FP32 partials of unit (row tile, node group gg, split) go to slice gg S + split
  int sum;
  const float2* coef;       // c_j (sum mode)
  int64_t b_node_stride;    // bytes between the nodes' basis planes (0: one X for all)
  int gchunk;               // node groups per unit (sum mode): a unit runs its K-blocks for
  int ngc;                  // each of its groups in turn; ngc = ceil(nG / gchunk) chunks
  OpCoef op;                // T = c_G G + c_H (1/2 I + K) (the kOp instantiations)
  const __nv_bfloat16* Bp;   // prepared basis planes, tile-native
  float* Yp;          // FP32 partial products [S][N][2 nup][n_pad]
  int* status;
  uint32_t wait_limit;   // polls of each pipeline-stage wait (the drains keep kWaitLimit)
};

struct SmemLayout {
  uint32_t a_off, b_off, graw_off, row_off, col_off, self_off, bar_off, misc_off, total;
  uint32_t a_stage_bytes, b_stage_bytes;
};
constexpr uint32_t kGeoBlockBytes = kBK * 64 * 4;   // packed geometry of one K-block

// bnodes: basis plane sets per stage (G in the node-summed mode with one X per node, else 1)
__host__ __device__ inline SmemLayout smem_layout(int G, int nup, int bnodes = 1) {
  SmemLayout L;
  L.a_stage_bytes = (uint32_t)G * 4 * kPlaneBytes;
  L.b_stage_bytes = (uint32_t)bnodes * 256 * nup;   // 4 planes x 2 nup rows x 16 k x 2 B each
  L.a_off = 0;
  L.b_off = L.a_off + kStages * L.a_stage_bytes;
  L.graw_off = L.b_off + kStages * L.b_stage_bytes;    // per stage: packed geometry copy
  L.row_off = L.graw_off + kStages * kGeoBlockBytes;
  L.col_off = L.row_off + kBM * 4 * 4;           // 128 rows x (x, y, z, valid)
  L.self_off = L.col_off + kStages * kBK * 7 * 16;   // per stage 16 x 7 float4 (x, y, z, w)
  L.bar_off = L.self_off + kStages * kBK * kMaxG * 8;  // per stage 16 x G complex self terms
  L.misc_off = L.bar_off + 12 * 8;               // 11 mbarriers (+1 pad)
  L.total = L.misc_off + 16;                     // tmem slot, abort flag
  return L;
}

__device__ __forceinline__ float ex2f(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sinf_mufu(float x) {
  float r;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float cosf_mufu(float x) {
  float r;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrtf_mufu(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// General operator: (sr, si) += a (cs + i sn) F, F = c_G + c_H s (i k r - 1) for the two
// columns at once; s = (y - x).n / r^2, ph = Re(k) r, kir = Im(k) r, m1 = (-1, -1).
__device__ __forceinline__ void op_acc2(f2_t& sr, f2_t& si, f2_t a, f2_t cs, f2_t sn, f2_t s,
                                       f2_t ph, f2_t kir, f2_t cgr2, f2_t cgi2, f2_t chr2,
                                       f2_t chi2, f2_t nchi2, f2_t m1) {
  const f2_t A = mul2(fma2(s, kir, s), m1);   // -s (1 + Im(k) r)
  const f2_t B = mul2(s, ph);                 //  s Re(k) r
  const f2_t fr = fma2(chr2, A, fma2(nchi2, B, cgr2));
  const f2_t fi = fma2(chr2, B, fma2(chi2, A, cgi2));
  const f2_t cr = mul2(a, cs), ci = mul2(a, sn);
  sr = fma2(cr, fr, fma2(mul2(ci, m1), fi, sr));
  si = fma2(cr, fi, fma2(ci, fr, si));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo_elem, float hi_elem) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo_elem, hi_elem);   // .x -> low 16 bits
  return *reinterpret_cast<uint32_t*>(&h);
}

// Two entries (row i, columns l0, l0 + 1) of one node: the self term on the diagonal, zero
// in the padding, then the hi/lo BF16 split into the four planes (Re hi, Re lo, Im hi, Im lo)
// at ag; self points at the staged self term of column l0 (that of l0 + 1 is kMaxG later).
__device__ __forceinline__ void put_entries(f2_t sr2, f2_t si2, const float2* self, int64_t i,
                                            int64_t l0, int64_t n, unsigned char* ag,
                                            bool scaled = false, float2 cf = float2(),
                                            uint32_t plane_bytes = kPlaneBytes) {
  float re[2], im[2];
  f2split(sr2, re[0], re[1]);
  f2split(si2, im[0], im[1]);
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    if (i == l0 + d) {   // diagonal: the self term
      const float2 sv = self[d * kMaxG];
      re[d] = sv.x;
      im[d] = sv.y;
    }
    if (scaled) {        // node-summed mode: c_j A_il(z_j)
      const float r = re[d] * cf.x - im[d] * cf.y;
      im[d] = re[d] * cf.y + im[d] * cf.x;
      re[d] = r;
    }
    if (i >= n || l0 + d >= n) {   // padding rows / columns of the tile
      re[d] = 0.f;
      im[d] = 0.f;
    }
  }
  const uint32_t hr = pack_bf16(re[0], re[1]);
  const uint32_t hi = pack_bf16(im[0], im[1]);
  const uint32_t lr = pack_bf16(re[0] - __uint_as_float(hr << 16),
                                re[1] - __uint_as_float(hr & 0xFFFF0000u));
  const uint32_t li = pack_bf16(im[0] - __uint_as_float(hi << 16),
                                im[1] - __uint_as_float(hi & 0xFFFF0000u));
  *reinterpret_cast<uint32_t*>(ag + 0 * plane_bytes) = hr;
  *reinterpret_cast<uint32_t*>(ag + 1 * plane_bytes) = lr;
  *reinterpret_cast<uint32_t*>(ag + 2 * plane_bytes) = hi;
  *reinterpret_cast<uint32_t*>(ag + 3 * plane_bytes) = li;
}

// Two entries of one node in one column l: rows i0 and i1 = i0 + 64 in the FFMA2 lanes (the
// self term on the diagonal, zero in the padding), split into BF16 hi/lo and stored as
// 16-bit values into the four planes of a column half (kHalfPlane apart) at ag (row i0)
// and ag + 1024 (row i1: eight 8-row groups of 128 bytes further); self points at the
// staged self term of column l.
__device__ __forceinline__ void put_rows(f2_t sr2, f2_t si2, const float2* self, int64_t i0,
                                         int64_t i1, int64_t l, int64_t n, unsigned char* ag) {
  float re[2], im[2];
  f2split(sr2, re[0], re[1]);
  f2split(si2, im[0], im[1]);
  const int64_t ii[2] = {i0, i1};
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    if (ii[d] == l) {   // diagonal: the self term
      const float2 sv = *self;
      re[d] = sv.x;
      im[d] = sv.y;
    }
    if (ii[d] >= n || l >= n) {   // padding rows / columns of the tile
      re[d] = 0.f;
      im[d] = 0.f;
    }
  }
  const uint32_t hr = pack_bf16(re[0], re[1]);
  const uint32_t hi = pack_bf16(im[0], im[1]);
  const uint32_t lr = pack_bf16(re[0] - __uint_as_float(hr << 16),
                                re[1] - __uint_as_float(hr & 0xFFFF0000u));
  const uint32_t li = pack_bf16(im[0] - __uint_as_float(hi << 16),
                                im[1] - __uint_as_float(hi & 0xFFFF0000u));
  const uint32_t v[4] = {hr, lr, hi, li};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    *reinterpret_cast<uint16_t*>(ag + q * kHalfPlane) = (uint16_t)(v[q] & 0xFFFFu);
    *reinterpret_cast<uint16_t*>(ag + 1024 + q * kHalfPlane) = (uint16_t)(v[q] >> 16);
  }
}

// bounded wait that also watches the block's abort flag
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity,
                                              volatile int* abort_flag, int* status,
                                              uint32_t limit = kWaitLimit) {
  for (uint32_t it = 0; it < limit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (it > 64) __nanosleep(64);
  }
  atomicOr(status, kStatusTimeout);
  *abort_flag = 1;
  return false;
}

// One work unit (row tile, node group, column split) of problem p; the body of the single
// and the grouped launch.
// tmem_given: TMEM columns already allocated by a persistent caller (its base address), or
// kNoTmem to allocate (and release) them here.
constexpr uint32_t kNoTmem = 0xffffffffu;
// kSum: the node-summed mode (p.sum is set accordingly by the host); kOp: the general
// operator c_G G + c_H (1/2 I + K) (else the single layer, c_G = 1, c_H = 0)
// kNP: quadrature points (the first kNP of 7) whose sine and cosine come from the FMA-pipe
// polynomials (sincos_poly2) instead of the MUFU unit, which balances the two pipes.
template <bool kSum, bool kOp = false, int kNP = 0>
__device__ __forceinline__ void mixed_apply_unit(const MixedParams& p, const int u,
                                                 const uint32_t tmem_given) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int bnodes = (kSum && p.b_node_stride) ? p.G : 1;
  const SmemLayout L = smem_layout(p.G, p.nup, bnodes);
  unsigned char* sA = smem + L.a_off;
  unsigned char* sB = smem + L.b_off;
  float4* sRow = reinterpret_cast<float4*>(smem + L.row_off);
  const float* sGraw = reinterpret_cast<const float*>(smem + L.graw_off);  // [stage][16][64]
  float4* sColAll = reinterpret_cast<float4*>(smem + L.col_off);    // [stage][16][7]
  float2* sSelfAll = reinterpret_cast<float2*>(smem + L.self_off);  // [stage][16][kMaxG]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
  uint64_t* afull = bars;        // [2] evaluation warps -> MMA
  uint64_t* bfull = bars + 2;    // [2] bulk copy -> MMA
  uint64_t* empty = bars + 4;    // [2] MMA done with the stage
  uint64_t* accfull = bars + 6;  // accumulators final
  uint64_t* gfull = bars + 7;    // [2] column geometry / self terms staged -> evaluation
  uint64_t* gready = bars + 9;   // [2] packed geometry bulk copy landed -> producer
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.misc_off);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.misc_off + 4);

  const int warp = threadIdx.x / 32;
  const int lane = threadIdx.x % 32;

  // unit -> (row tile, node group(s), column split); the node-summed mode takes a chunk of
  // gchunk node groups and runs the unit's K-blocks for each in turn (iteration
  // it = group offset * nkb + K-block offset), all into one accumulator
  const int split = u % p.S;
  const int t = u / p.S;
  const int ngc = kSum ? p.ngc : p.nG;
  const int gc = t % ngc;
  const int rt = t / ngc;
  const int g_begin = kSum ? gc * p.gchunk : gc;
  const int ngr = kSum ? min(p.gchunk, p.nG - g_begin) : 1;
  const int64_t row0 = (int64_t)rt * kBM;
  const int kb0 = (int)((int64_t)p.nK * split / p.S);
  const int kb1 = (int)((int64_t)p.nK * (split + 1) / p.S);
  const int nkb = kb1 - kb0;
  const int nit = ngr * nkb;
  const int gg = g_begin;                 // the node group (projection)
  const int j0 = gg * p.G;
  const int Gv = min(p.G, p.N - j0);
  const uint32_t acc_cols = 2u * p.nup;                 // TMEM columns per node
  const uint32_t accs = kSum ? 1u : (uint32_t)p.G;   // accumulators (nodes, or their sum)
  uint32_t tmem_cols = 32;
  while (tmem_cols < accs * acc_cols) tmem_cols <<= 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&afull[s], kEvalThreads);
      mbar_init(&bfull[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&gfull[s], 32);
      mbar_init(&gready[s], 1);
    }
    mbar_init(accfull, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1 && tmem_given == kNoTmem) {
    tmem_alloc(tmem_slot, tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_given == kNoTmem ? *tmem_slot : tmem_given;

  if (warp == 0) {
    // ---------------- producer: basis planes (bulk copy), column geometry, self terms ----
    // origin of this tile's relative coordinates: its first centroid
    const int64_t i_org = row0 < p.n ? row0 : p.n - 1;
    const double ox = p.cx[i_org], oy = p.cx[p.n + i_org], oz = p.cx[2 * p.n + i_org];
    const float oxh = (float)ox, oyh = (float)oy, ozh = (float)oz;
    const float oxl = (float)(ox - oxh), oyl = (float)(oy - oyh), ozl = (float)(oz - ozh);
    for (int r = lane; r < kBM; r += 32) {
      const int64_t i = row0 + r;
      float4 v = make_float4(2.0f, 2.0f, 2.0f, 0.f);   // padding rows: zeroed after evaluation
      if (i < p.n)
        v = make_float4((float)(p.cx[i] - ox), (float)(p.cx[p.n + i] - oy),
                        (float)(p.cx[2 * p.n + i] - oz), 1.f);
      sRow[r] = v;
    }
    // per iteration, with fewer than kMaxG nodes per unit (a short evaluation per K-block):
    // the column geometry as soon as the evaluation warps are done with the stage (afull of
    // the previous round), the basis planes once the MMAs are (empty); with kMaxG nodes both
    // once the MMAs are done (the evaluation is long enough to hide the copies)
    const bool early = p.G < kMaxG;
    int issued_g = 0, issued_b = 0;
    for (int it = 0; it < nit; ++it) {
      const int s = it % kStages;
      const uint32_t par = (it / kStages) & 1;
      const int kb = kb0 + (kSum ? it % nkb : it);
      const int j0i = kSum ? (g_begin + it / nkb) * p.G : j0;
      const int Gvi = kSum ? min(p.G, p.N - j0i) : Gv;
      int ok = 1;
      if (lane == 0)
        ok = early ? wait_or_abort(&afull[s], par ^ 1, abort_flag, p.status, p.wait_limit)
                   : wait_or_abort(&empty[s], par ^ 1, abort_flag, p.status, p.wait_limit);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      auto issue_b = [&]() {
        if (lane == 0) {
          const uint32_t bset = 256u * p.nup;   // one node's (or the shared) planes
          // one X per node (node-summed mode): the planes of each node of the unit, at its
          // own offset, also when the unit holds a single node
          const bool per_node = kSum && p.b_node_stride != 0;
          const int nb = per_node ? Gvi : 1;
          mbar_arrive_expect_tx(&bfull[s], (uint32_t)nb * bset);
          for (int g = 0; g < nb; ++g) {
            const size_t node_off =
                per_node ? (size_t)(p.order[j0i + g] & kNodeMask) * (size_t)p.b_node_stride : 0;
            bulk_g2s(sB + s * L.b_stage_bytes + g * bset,
                     reinterpret_cast<const unsigned char*>(p.Bp) + node_off + (size_t)kb * bset,
                     bset, &bfull[s]);
          }
        }
        ++issued_b;
      };
      if (!early) issue_b();   // the stage is free of the MMAs already
      if (lane == 0) {
        mbar_arrive_expect_tx(&gready[s], kGeoBlockBytes);
        bulk_g2s(smem + L.graw_off + s * kGeoBlockBytes, p.pack32 + (size_t)kb * kBK * 64,
                 kGeoBlockBytes, &gready[s]);
      }
      ++issued_g;
      // tile-relative FP32 coordinates from the hi/lo pairs: (y_hi - o_hi) + (y_lo - o_lo)
      if (!wait_or_abort(&gready[s], par, abort_flag, p.status, p.wait_limit)) break;
      const float* graw = sGraw + s * (kBK * 64);
      float4* sCol = sColAll + s * (kBK * 7);
      for (int x = lane; x < kBK * 7; x += 32) {
        const int k = x / 7, q = x % 7;
        const float4 hi = *reinterpret_cast<const float4*>(graw + k * 64 + 4 * q);
        const float4 lo = *reinterpret_cast<const float4*>(graw + k * 64 + 28 + 4 * q);
        sCol[x] = make_float4((hi.x - oxh) + (lo.x - oxl), (hi.y - oyh) + (lo.y - oyl),
                              (hi.z - ozh) + (lo.z - ozl), hi.w);
      }
      float2* sSelf = sSelfAll + s * (kBK * kMaxG);
      for (int x = lane; x < kBK * kMaxG; x += 32) {
        const int k = x / kMaxG, g = x % kMaxG;
        const int64_t l = (int64_t)kb * kBK + k;
        float2 v = make_float2(0.f, 0.f);
        if (l < p.n && g < Gvi && l >= row0 && l < row0 + kBM)
          v = p.self32[(int64_t)(p.order[j0i + g] & kNodeMask) * p.n + l];
        sSelf[x] = v;
      }
      mbar_arrive(&gfull[s]);   // release: the staged values are visible to the waiters
      if (early) {
        if (lane == 0) ok = wait_or_abort(&empty[s], par ^ 1, abort_flag, p.status, p.wait_limit);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        issue_b();
      }
    }
    if (lane == 0 && *abort_flag) {
      // let copies in flight land before the block exits (bounded)
      for (int it = max(0, issued_b - kStages); it < issued_b; ++it)
        mbar_wait(&bfull[it % kStages], (it / kStages) & 1, kWaitLimit);
      for (int it = max(0, issued_g - kStages); it < issued_g; ++it)
        mbar_wait(&gready[it % kStages], (it / kStages) & 1, kWaitLimit);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kBM, 2 * p.C);
      // (A plane, B plane) pairs of the split-precision complex product
      const int pa[6] = {0, 0, 1, 2, 2, 3};   // Ar_hi, Ar_hi, Ar_lo, Ai_hi, Ai_hi, Ai_lo
      const int pb[6] = {0, 1, 0, 2, 3, 2};   // [Vr|Vi], [Vr_lo|Vi_lo], [-Vi|Vr], [-Vi_lo|Vr_lo]
      const uint32_t bplane = 2u * p.C * kBK * 2;   // bytes of one basis plane per chunk
      for (int it = 0; it < nit; ++it) {
        const int s = it % kStages;
        const uint32_t par = (it / kStages) & 1;
        if (!wait_or_abort(&afull[s], par, abort_flag, p.status, p.wait_limit)) break;
        if (!wait_or_abort(&bfull[s], par, abort_flag, p.status, p.wait_limit)) break;
        tc_fence_after();
        const uint32_t a_base = smem_u32(sA + s * L.a_stage_bytes);
        const uint32_t b_base = smem_u32(sB + s * L.b_stage_bytes);
        const int Gvi = kSum ? min(p.G, p.N - (g_begin + it / nkb) * p.G) : Gv;
        for (int g = 0; g < Gvi; ++g) {
          const uint32_t bg = b_base + (bnodes > 1 ? g * 256u * p.nup : 0u);
          for (int c = 0; c < p.nchunks; ++c) {
            const uint32_t d = tmem_base + (kSum ? 0u : g * acc_cols) + c * 2 * p.C;
            const bool fresh = it == 0 && (!kSum || g == 0);
#pragma unroll
            for (int q = 0; q < 6; ++q) {
              const uint64_t ad = smem_desc(a_base + (g * 4 + pa[q]) * kPlaneBytes, 128, 256);
              const uint64_t bd = smem_desc(bg + (c * 4 + pb[q]) * bplane, 128, 256);
              mma_bf16(d, ad, bd, idesc, (fresh && q == 0) ? 0u : 1u);
            }
          }
        }
        mma_commit(&empty[s]);
      }
      mma_commit(accfull);
    }
  } else {
    // ---------------- evaluation warps ----------------
    const int e = warp - 2;               // 0..15: row group of the 128 x 16 block
    // node constants
    float kr[kMaxG], kmi[kMaxG];
    float kim[kOp ? kMaxG : 1];   // Im z_j (general operator)
    float2 cf[kSum ? kMaxG : 1];
    bool twin[kMaxG / 2];
    constexpr bool scaled = kSum;
    int Gvc = Gv;   // nodes of the current group
    auto load_nodes = [&](int j0x, int Gvx) {
#pragma unroll
      for (int g = 0; g < kMaxG; ++g) {
        const int code = p.order[j0x + (g < Gvx ? g : 0)];
        const int j = code & kNodeMask;
        if (kSum) cf[kSum ? g : 0] = p.coef[j];
        kr[g] = (float)p.z[2 * j];
        kmi[g] = (float)(-p.z[2 * j + 1]) * kLog2e;
        if (kOp) kim[kOp ? g : 0] = (float)p.z[2 * j + 1];
        // a twin pair sits at slots 2 P, 2 P + 1 of the schedule: inside this group when
        // the group starts at an even slot
        if (g % 2 == 0)
          twin[g / 2] = (code & kTwinBit) && (j0x % 2 == 0) && g + 1 < Gvx && kr[g] ==
                        (float)p.z[2 * (p.order[j0x + g + 1] & kNodeMask)];
      }
    };
    load_nodes(j0, Gv);
    // operator constants (kOp): F = c_G + c_H s (i k r - 1) per point, s = (y - x).n / r^2
    const f2_t m1 = f2(-1.f, -1.f);
    const f2_t cgr2 = f2((float)p.op.cgr, (float)p.op.cgr), cgi2 = f2((float)p.op.cgi, (float)p.op.cgi);
    const f2_t chr2 = f2((float)p.op.chr, (float)p.op.chr), chi2 = f2((float)p.op.chi, (float)p.op.chi);
    const f2_t nchi2 = f2(-(float)p.op.chi, -(float)p.op.chi);
    // this thread's entries: row 8 e + r8, columns 8 kg + 2 kp + {0, 1} for kg = 0, 1
    const int r8 = lane / 4, kp = lane % 4;
    const int row = 8 * e + r8;
    const int64_t i = row0 + row;

    for (int it = 0; it < nit; ++it) {
      const int s = it % kStages;
      const uint32_t par = (it / kStages) & 1;
      const int kb = kb0 + (kSum ? it % nkb : it);
      if (kSum && it > 0 && it % nkb == 0) {   // next node group of the chunk
        const int j0x = (g_begin + it / nkb) * p.G;
        Gvc = min(p.G, p.N - j0x);
        load_nodes(j0x, Gvc);
      }
      // the column geometry, and the stage's A planes free of the MMAs of its last round
      // (one lane per warp observes the MMAs' completion; the warp synchronises on it)
      int free_ok = 1;
      if (p.G < kMaxG && lane == 0)
        free_ok = wait_or_abort(&empty[s], par ^ 1, abort_flag, p.status, p.wait_limit);
      free_ok = __shfl_sync(0xffffffffu, free_ok, 0);
      const bool ready = wait_or_abort(&gfull[s], par, abort_flag, p.status, p.wait_limit) && free_ok;
      const float4* sCol = sColAll + s * (kBK * 7);
      const float2* sSelf = sSelfAll + s * (kBK * kMaxG);
      unsigned char* a_stage = sA + s * L.a_stage_bytes;
      const float4 xr = sRow[row];
#pragma unroll 1
      for (int kg = 0; kg < (ready ? 2 : 0); ++kg) {
        const int k0 = 8 * kg + 2 * kp;
        const int64_t l0 = (int64_t)kb * kBK + k0;
        // distances and weights of the 7 points of both columns, as pairs (column k0, k0 + 1)
        f2_t rr2[7], am2[7];
        f2_t s2[kOp ? 7 : 1];   // (y - x) . n / r^2 of both columns (general operator)
        {
          const float4* c0 = sCol + k0 * 7;
          const float4* c1 = c0 + 7;
          const f2_t xx = f2(xr.x, xr.x), xy = f2(xr.y, xr.y), xz = f2(xr.z, xr.z);
          // the columns' normals, negated (d = x - y here), from the staged packed geometry
          f2_t nnx = f2(0.f, 0.f), nny = nnx, nnz = nnx;
          if (kOp) {
            const float* gk = sGraw + s * (kBK * 64) + k0 * 64;
            nnx = f2(-gk[56], -gk[64 + 56]);
            nny = f2(-gk[57], -gk[64 + 57]);
            nnz = f2(-gk[58], -gk[64 + 58]);
          }
#pragma unroll
          for (int q = 0; q < 7; ++q) {
            const float4 y0 = c0[q], y1 = c1[q];
            const f2_t dx = sub2(xx, f2(y0.x, y1.x)), dy = sub2(xy, f2(y0.y, y1.y)),
                       dz = sub2(xz, f2(y0.z, y1.z));
            const f2_t r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
            float r20, r21;
            f2split(r2, r20, r21);
            const f2_t rs = f2(rsqrtf_mufu(r20), rsqrtf_mufu(r21));
            rr2[q] = mul2(r2, rs);
            am2[q] = mul2(f2(y0.w, y1.w), rs);
            if (kOp)
              s2[kOp ? q : 0] = mul2(fma2(dx, nnx, fma2(dy, nny, mul2(dz, nnz))), mul2(rs, rs));
          }
        }
        const uint32_t off = e * 256 + kg * 128 + r8 * 16 + kp * 4;
        const float2* selfk = sSelf + k0 * kMaxG;
#pragma unroll
        for (int g = 0; g < kMaxG; g += 2) {
          if (g >= Gvc) break;
          if (twin[g / 2]) {
            // twin nodes: one sine and one cosine of the shared phase for both
            f2_t sa = f2(0.f, 0.f), ia = f2(0.f, 0.f), sb = f2(0.f, 0.f), ib = f2(0.f, 0.f);
            const f2_t kma = f2(kmi[g], kmi[g]), kmb = f2(kmi[g + 1], kmi[g + 1]);
            const f2_t kr2 = f2(kr[g], kr[g]);
#pragma unroll
            for (int q = 0; q < 7; ++q) {
              float e0, e1, e2, e3;
              f2split(mul2(kma, rr2[q]), e0, e1);
              f2split(mul2(kmb, rr2[q]), e2, e3);
              f2_t aa = mul2(am2[q], f2(ex2f(e0), ex2f(e1)));
              f2_t ab = mul2(am2[q], f2(ex2f(e2), ex2f(e3)));
              const f2_t ph2 = mul2(kr2, rr2[q]);
              f2_t cs, sn;
              if (q < kNP) {   // FMA pipe: e^{i ph} = (-1)^n e^{i pi f}, the sign into aa, ab
                f2_t sg;
                sincos_poly2(ph2, cs, sn, sg);
                aa ^= sg;
                ab ^= sg;
              } else {
                float p0, p1;
                f2split(ph2, p0, p1);
                cs = f2(cosf_mufu(p0), cosf_mufu(p1));
                sn = f2(sinf_mufu(p0), sinf_mufu(p1));
              }
              if constexpr (kOp) {
                op_acc2(sa, ia, aa, cs, sn, s2[q], ph2,
                        mul2(f2(kim[g], kim[g]), rr2[q]), cgr2, cgi2, chr2, chi2, nchi2, m1);
                op_acc2(sb, ib, ab, cs, sn, s2[q], ph2,
                        mul2(f2(kim[g + 1], kim[g + 1]), rr2[q]), cgr2, cgi2, chr2, chi2, nchi2,
                        m1);
              } else {
                sa = fma2(aa, cs, sa);
                ia = fma2(aa, sn, ia);
                sb = fma2(ab, cs, sb);
                ib = fma2(ab, sn, ib);
              }
            }
            put_entries(sa, ia, selfk + g, i, l0, p.n, a_stage + g * 4 * kPlaneBytes + off,
                        scaled, cf[kSum ? g : 0]);
            put_entries(sb, ib, selfk + g + 1, i, l0, p.n,
                        a_stage + (g + 1) * 4 * kPlaneBytes + off, scaled, cf[kSum ? g + 1 : 0]);
          } else {
#pragma unroll
            for (int h = g; h < g + 2; ++h) {
              if (h >= Gvc) break;
              f2_t sr2 = f2(0.f, 0.f), si2 = f2(0.f, 0.f);
              const f2_t kmi2 = f2(kmi[h], kmi[h]), kr2 = f2(kr[h], kr[h]);
#pragma unroll
              for (int q = 0; q < 7; ++q) {
                float e0, e1;
                f2split(mul2(kmi2, rr2[q]), e0, e1);
                f2_t a = mul2(am2[q], f2(ex2f(e0), ex2f(e1)));
                const f2_t ph2 = mul2(kr2, rr2[q]);
                f2_t cs, sn;
                if (q < kNP) {   // FMA pipe: e^{i ph} = (-1)^n e^{i pi f}, the sign into a
                  f2_t sg;
                  sincos_poly2(ph2, cs, sn, sg);
                  a ^= sg;
                } else {
                  // the MUFU sine and cosine reduce their argument in revolutions
                  // themselves; that reduction's error (half an FP32 ulp of ph / 2 pi) is
                  // of the order of the rounding of ph itself, so no explicit reduction
                  // precedes them
                  float p0, p1;
                  f2split(ph2, p0, p1);
                  cs = f2(cosf_mufu(p0), cosf_mufu(p1));
                  sn = f2(sinf_mufu(p0), sinf_mufu(p1));
                }
                if constexpr (kOp) {
                  op_acc2(sr2, si2, a, cs, sn, s2[q], ph2, mul2(f2(kim[h], kim[h]), rr2[q]), cgr2,
                          cgi2, chr2, chi2, nchi2, m1);
                } else {
                  sr2 = fma2(a, cs, sr2);
                  si2 = fma2(a, sn, si2);
                }
              }
              put_entries(sr2, si2, selfk + h, i, l0, p.n, a_stage + h * 4 * kPlaneBytes + off,
                          scaled, cf[kSum ? h : 0]);
            }
          }
        }
      }
      fence_proxy_async_smem();
      mbar_arrive(&afull[s]);
      if (!ready) break;
    }

    // ---------------- epilogue: TMEM -> FP32 partial Y ----------------
    const bool ok = !*abort_flag && wait_or_abort(accfull, 0, abort_flag, p.status, p.wait_limit);
    if (__all_sync(0xffffffffu, ok)) {   // tcgen05.ld is warp-collective
      tc_fence_after();
      const int quarter = warp % 4;              // TMEM lanes this warp may read
      const int part = (warp - 2) / 4;           // four warps per quarter split the columns
      const int erow = quarter * 32 + lane;
      const int64_t ei = row0 + erow;
      const uint32_t cols_total = (kSum ? 1u : (uint32_t)Gv) * acc_cols;
      for (uint32_t c0 = part * 16; c0 < cols_total; c0 += 64) {
        float v[16];
        tmem_ld16(tmem_base + ((uint32_t)(quarter * 32) << 16) + c0, v);
        const int g = c0 / acc_cols;
        const int col = c0 % acc_cols;
        // projection: slice split, node j; node-summed: slice gg S + split
        const size_t slot = kSum ? (size_t)gc * p.S + split
                                  : (size_t)split * p.N + (p.order[j0 + g] & kNodeMask);
        float* dst = p.Yp + (slot * acc_cols + col) * p.n_pad + ei;
#pragma unroll
        for (int k = 0; k < 16; ++k) dst[(size_t)k * p.n_pad] = v[k];
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    // the accumulators may only be released once every MMA has completed (bounded wait:
    // immediate on the normal path, where the epilogue has already seen it)
    if (lane == 0) mbar_wait(accfull, 0, kWaitLimit);
    __syncwarp();
    tc_fence_after();
    if (tmem_given == kNoTmem) tmem_dealloc(tmem_base, tmem_cols);
  }
}

template <bool kOp, int kNP>
__global__ void __launch_bounds__(kThreads, 1) mixed_apply_kernel(MixedParams p) {
  mixed_apply_unit<false, kOp, kNP>(p, blockIdx.x, kNoTmem);
}

// ---------------------------------------------------------------------------------------
// Twin pairs across a cluster of two CTAs, for units of one node (bases of more than 128
// columns, whose [Yr | Yi] accumulator fills the 512 TMEM columns of an SM).
// CTA r of the cluster holds the accumulator of node r of a twin pair (two nodes with the
// same FP32 real part, so the same phase Re(z) r at every quadrature point). Per 128 x 16
// K-block each CTA evaluates columns 8 r .. 8 r + 7 for BOTH nodes: one rsqrt, one sine and
// one cosine per quadrature point serve two nodes, against one node per point in the
// unpaired unit. It writes node r's entries into its own A stage and the other node's into
// an export buffer, which one bulk copy moves into the peer's A stage (distributed shared
// memory, completing on the peer's xin mbarrier). A node's A stage is laid out as two
// contiguous 8 KB column halves, each with the four planes (Re hi, Re lo, Im hi, Im lo) of
// 128 rows x 8 columns, so that a half is one copy. Each MMA warp's commit arrives on the
// stage-free barriers of both CTAs (multicast): a stage, its export buffer and the copy's
// target are rewritten only once both CTAs' MMAs are done with them. Pairs whose first
// slot carries no twin flag run unpaired, each CTA evaluating its own node (the second
// idles when N is odd). Every wait is bounded; the CTAs leave the cluster together, after
// any copy still addressed to them has landed.
// Pipeline: three A stages (the evaluated blocks, their export buffers, column geometry)
// and two basis stages (64 KB each at 256 columns), with the basis copies in a warp of
// their own: the evaluation runs up to two K-blocks ahead of the MMAs, which hides the
// exchange between the partners and the MMAs' own duration behind it (with two stages
// the evaluation warps waited for a free stage a sixth of the time).
constexpr uint32_t kHalfBytes = 4 * kHalfPlane;        // the four planes of a half: 8 KB
constexpr int kPA = 3;                                 // A stages
constexpr int kPB = 2;                                 // basis stages
constexpr int kPairWarps = 3 + kEvalWarps;   // geometry producer, MMA, basis producer, evaluation
constexpr int kPairThreads = 32 * kPairWarps;

struct PairLayout {
  uint32_t a_off, x_off, b_off, graw_off, row_off, col_off, self_off, bar_off, misc_off, total;
  uint32_t b_stage_bytes;
};
__host__ __device__ inline PairLayout pair_layout(int nup) {
  PairLayout L;
  L.b_stage_bytes = 256u * nup;
  L.a_off = 0;
  L.x_off = L.a_off + kPA * 2 * kHalfBytes;
  L.b_off = L.x_off + kPA * kHalfBytes;
  L.graw_off = L.b_off + kPB * L.b_stage_bytes;
  L.row_off = L.graw_off + kPA * kGeoBlockBytes;
  L.col_off = L.row_off + kBM * 4 * 4;
  L.self_off = L.col_off + kPA * kBK * 7 * 16;
  L.bar_off = L.self_off + kPA * kBK * kMaxG * 8;
  L.misc_off = L.bar_off + 24 * 8;   // 20 mbarriers (+4 pad)
  L.total = L.misc_off + 16;         // tmem slot, abort flag, halves sent by the peer
  return L;
}

template <bool kOp, int kNP>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kPairThreads, 1)
    mixed_pair_kernel(MixedParams p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const PairLayout L = pair_layout(p.nup);
  unsigned char* sA = smem + L.a_off;
  unsigned char* sX = smem + L.x_off;
  unsigned char* sB = smem + L.b_off;
  float4* sRow = reinterpret_cast<float4*>(smem + L.row_off);
  const float* sGraw = reinterpret_cast<const float*>(smem + L.graw_off);
  float4* sColAll = reinterpret_cast<float4*>(smem + L.col_off);
  float2* sSelfAll = reinterpret_cast<float2*>(smem + L.self_off);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
  uint64_t* afull = bars;         // [kPA] this CTA's evaluation warps -> MMA
  uint64_t* empty = bars + 3;     // [kPA] the MMAs (both CTAs' when paired) done with the A stage
  uint64_t* gfull = bars + 6;     // [kPA] column geometry / self terms staged -> evaluation
  uint64_t* gready = bars + 9;    // [kPA] packed geometry bulk copy landed -> producer
  uint64_t* xin = bars + 12;      // [kPA] the peer's half of the A stage landed -> MMA
  uint64_t* bfull = bars + 15;    // [kPB] basis bulk copy -> MMA
  uint64_t* bempty = bars + 17;   // [kPB] this CTA's MMAs done with the basis stage
  uint64_t* accfull = bars + 19;  // accumulator final
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.misc_off);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.misc_off + 4);
  volatile uint32_t* peer_sent = reinterpret_cast<volatile uint32_t*>(smem + L.misc_off + 8);

  const int warp = threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  const uint32_t rank = cluster_ctarank();
  const uint32_t peer = rank ^ 1u;

  // cluster -> (row tile, pair of schedule slots, column split)
  const int npairs = (p.N + 1) / 2;
  const int cl = blockIdx.x / 2;
  const int split = cl % p.S;
  const int t = cl / p.S;
  const int pr = t % npairs;
  const int rt = t / npairs;
  const int slot0 = 2 * pr;
  const bool paired = (p.order[slot0] & kTwinBit) != 0 && slot0 + 1 < p.N;
  const int myslot = slot0 + (int)rank;
  const bool has_node = myslot < p.N;
  const int64_t row0 = (int64_t)rt * kBM;
  const int kb0 = (int)((int64_t)p.nK * split / p.S);
  const int kb1 = (int)((int64_t)p.nK * (split + 1) / p.S);
  const int nit = kb1 - kb0;
  const int ev0 = paired ? slot0 : myslot;   // evaluated nodes: the pair, or this CTA's own
  const int nev = paired ? 2 : 1;
  const uint32_t acc_cols = 2u * p.nup;
  uint32_t tmem_cols = 32;
  while (tmem_cols < acc_cols) tmem_cols <<= 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kPA; ++s) {
      mbar_init(&afull[s], kEvalThreads);
      mbar_init(&empty[s], paired ? 2 : 1);
      mbar_init(&gfull[s], 32);
      mbar_init(&gready[s], 1);
      mbar_init(&xin[s], 1);
    }
    for (int s = 0; s < kPB; ++s) {
      mbar_init(&bfull[s], 1);
      mbar_init(&bempty[s], 1);
    }
    mbar_init(accfull, 1);
    // the first round of each stage expects the peer's half before the peer can send it
    if (paired)
      for (int s = 0; s < kPA && s < nit; ++s) mbar_arrive_expect_tx(&xin[s], kHalfBytes);
    *abort_flag = 0;
    *peer_sent = 0;
    fence_mbar_init();
  }
  if (warp == 1 && has_node) {
    tmem_alloc(tmem_slot, tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();   // both CTAs' barriers exist before any copy or arrival reaches them
  tc_fence_after();
  if (!has_node) {      // the idle second CTA of an unpaired last slot (N odd)
    cluster_sync_all();
    cluster_sync_all();
    return;
  }
  const uint32_t tmem_base = *tmem_slot;
  int consumed = 0, sent = 0;   // (MMA thread) peer halves consumed, halves sent

  if (warp == 0) {
    // ---------------- geometry producer: column geometry and self terms per A stage ------
    const int64_t i_org = row0 < p.n ? row0 : p.n - 1;
    const double ox = p.cx[i_org], oy = p.cx[p.n + i_org], oz = p.cx[2 * p.n + i_org];
    const float oxh = (float)ox, oyh = (float)oy, ozh = (float)oz;
    const float oxl = (float)(ox - oxh), oyl = (float)(oy - oyh), ozl = (float)(oz - ozh);
    for (int r = lane; r < kBM; r += 32) {
      const int64_t i = row0 + r;
      float4 v = make_float4(2.0f, 2.0f, 2.0f, 0.f);
      if (i < p.n)
        v = make_float4((float)(p.cx[i] - ox), (float)(p.cx[p.n + i] - oy),
                        (float)(p.cx[2 * p.n + i] - oz), 1.f);
      sRow[r] = v;
    }
    int issued_g = 0;
    for (int it = 0; it < nit; ++it) {
      const int s = it % kPA;
      const uint32_t par = (it / kPA) & 1;
      const int kb = kb0 + it;
      // the geometry once the evaluation warps are done with the stage
      int ok = 1;
      if (lane == 0) ok = wait_or_abort(&afull[s], par ^ 1, abort_flag, p.status, p.wait_limit);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      if (lane == 0) {
        mbar_arrive_expect_tx(&gready[s], kGeoBlockBytes);
        bulk_g2s(smem + L.graw_off + s * kGeoBlockBytes, p.pack32 + (size_t)kb * kBK * 64,
                 kGeoBlockBytes, &gready[s]);
      }
      ++issued_g;
      if (!wait_or_abort(&gready[s], par, abort_flag, p.status, p.wait_limit)) break;
      const float* graw = sGraw + s * (kBK * 64);
      float4* sCol = sColAll + s * (kBK * 7);
      for (int x = lane; x < kBK * 7; x += 32) {
        const int k = x / 7, q = x % 7;
        const float4 hi = *reinterpret_cast<const float4*>(graw + k * 64 + 4 * q);
        const float4 lo = *reinterpret_cast<const float4*>(graw + k * 64 + 28 + 4 * q);
        sCol[x] = make_float4((hi.x - oxh) + (lo.x - oxl), (hi.y - oyh) + (lo.y - oyl),
                              (hi.z - ozh) + (lo.z - ozl), hi.w);
      }
      float2* sSelf = sSelfAll + s * (kBK * kMaxG);
      for (int x = lane; x < kBK * kMaxG; x += 32) {
        const int k = x / kMaxG, g = x % kMaxG;
        const int64_t l = (int64_t)kb * kBK + k;
        float2 v = make_float2(0.f, 0.f);
        if (l < p.n && g < nev && l >= row0 && l < row0 + kBM)
          v = p.self32[(int64_t)(p.order[ev0 + g] & kNodeMask) * p.n + l];
        sSelf[x] = v;
      }
      mbar_arrive(&gfull[s]);
    }
    if (lane == 0 && *abort_flag)   // let geometry copies in flight land (bounded)
      for (int it = max(0, issued_g - kPA); it < issued_g; ++it)
        mbar_wait(&gready[it % kPA], (it / kPA) & 1, kWaitLimit);
  } else if (warp == 2) {
    // ---------------- basis producer: one K-block of the basis planes per basis stage ----
    if (lane == 0) {
      const uint32_t bset = 256u * p.nup;
      int issued_b = 0;
      for (int it = 0; it < nit; ++it) {
        const int s = it % kPB;
        const uint32_t par = (it / kPB) & 1;
        if (!wait_or_abort(&bempty[s], par ^ 1, abort_flag, p.status, p.wait_limit)) break;
        mbar_arrive_expect_tx(&bfull[s], bset);
        bulk_g2s(sB + s * L.b_stage_bytes,
                 reinterpret_cast<const unsigned char*>(p.Bp) + (size_t)(kb0 + it) * bset, bset,
                 &bfull[s]);
        ++issued_b;
      }
      if (*abort_flag)   // let basis copies in flight land (bounded)
        for (int it = max(0, issued_b - kPB); it < issued_b; ++it)
          mbar_wait(&bfull[it % kPB], (it / kPB) & 1, kWaitLimit);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (and sender of the evaluated half to the peer) ----------
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kBM, 2 * p.C);
      const int pa[6] = {0, 0, 1, 2, 2, 3};
      const int pb[6] = {0, 1, 0, 2, 3, 2};
      const uint32_t bplane = 2u * p.C * kBK * 2;
      for (int it = 0; it < nit; ++it) {
        const int s = it % kPA;
        const uint32_t par = (it / kPA) & 1;
        const int sb = it % kPB;
        const uint32_t parb = (it / kPB) & 1;
        if (!wait_or_abort(&afull[s], par, abort_flag, p.status, p.wait_limit)) break;
        if (*abort_flag) break;
        if (paired) {
          // this CTA's half of the other node's block -> the same half of the peer's stage
          bulk_s2peer(mapa_shared(smem_u32(sA + s * 2 * kHalfBytes + rank * kHalfBytes), peer),
                      sX + s * kHalfBytes, kHalfBytes, mapa_shared(smem_u32(&xin[s]), peer));
          ++sent;
          if (!wait_or_abort(&xin[s], par, abort_flag, p.status, p.wait_limit)) break;
          ++consumed;
          // the stage's next round expects its half before these MMAs release the peer
          if (it + kPA < nit) mbar_arrive_expect_tx(&xin[s], kHalfBytes);
        }
        if (!wait_or_abort(&bfull[sb], parb, abort_flag, p.status, p.wait_limit)) break;
        tc_fence_after();
        const uint32_t a_base = smem_u32(sA + s * 2 * kHalfBytes);
        const uint32_t b_base = smem_u32(sB + sb * L.b_stage_bytes);
        for (int c = 0; c < p.nchunks; ++c) {
          const uint32_t d = tmem_base + c * 2 * p.C;
#pragma unroll
          for (int q = 0; q < 6; ++q) {
            // column halves kHalfBytes apart along K, 8-row groups 128 bytes apart
            const uint64_t ad = smem_desc(a_base + pa[q] * kHalfPlane, kHalfBytes, 128);
            const uint64_t bd = smem_desc(b_base + (c * 4 + pb[q]) * bplane, 128, 256);
            mma_bf16(d, ad, bd, idesc, (it == 0 && q == 0) ? 0u : 1u);
          }
        }
        if (paired) mma_commit_mc(&empty[s], (uint16_t)0x3);
        else mma_commit(&empty[s]);
        mma_commit(&bempty[sb]);
      }
      mma_commit(accfull);
      // the number of halves sent, read by the peer after the first end-of-unit sync
      if (paired) st_peer_u32(mapa_shared(smem_u32((const void*)peer_sent), peer), (uint32_t)sent);
    }
  } else {
    // ---------------- evaluation warps ----------------
    const int e = warp - 3;
    float kr[2], kmi[2], kim[2];
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const int j = p.order[ev0 + (g < nev ? g : 0)] & kNodeMask;
      kr[g] = (float)p.z[2 * j];
      kmi[g] = (float)(-p.z[2 * j + 1]) * kLog2e;
      kim[g] = (float)p.z[2 * j + 1];
    }
    const f2_t m1 = f2(-1.f, -1.f);
    const f2_t cgr2 = f2((float)p.op.cgr, (float)p.op.cgr), cgi2 = f2((float)p.op.cgi, (float)p.op.cgi);
    const f2_t chr2 = f2((float)p.op.chr, (float)p.op.chr), chi2 = f2((float)p.op.chi, (float)p.op.chi);
    const f2_t nchi2 = f2(-(float)p.op.chi, -(float)p.op.chi);
    // this thread's entries: rows r and r + 64 of one column (r = 4 e + lane / 8, column
    // 8 kg + lane % 8), paired in the FFMA2 lanes. A warp reads eight columns' geometry per
    // load (one 128-byte wavefront per quarter-warp, no bank conflicts) and writes 16-bit
    // entries of four rows x eight columns (64 contiguous bytes per store); against a pair
    // of columns of one row this halves the column-geometry loads, the bulk of the shared-
    // memory traffic besides the tensor core's operand reads.
    const int cq8 = lane % 8;
    const int rr = 4 * e + lane / 8;                       // 0 .. 63
    const int64_t i0 = row0 + rr, i1 = i0 + 64;
    const uint32_t off = (uint32_t)(rr / 8) * 128 + (rr % 8) * 16 + cq8 * 2;   // row r; r + 64 at + 1024
    // paired: the column half kg = rank for both nodes; unpaired: both halves, own node
    const int kg_lo = paired ? (int)rank : 0;
    const int kg_hi = paired ? (int)rank + 1 : 2;
    float4 xa = make_float4(0.f, 0.f, 0.f, 0.f), xb = xa;

    for (int it = 0; it < nit; ++it) {
      const int s = it % kPA;
      const uint32_t par = (it / kPA) & 1;
      const int kb = kb0 + it;
      int free_ok = 1;
      if (lane == 0) free_ok = wait_or_abort(&empty[s], par ^ 1, abort_flag, p.status, p.wait_limit);
      free_ok = __shfl_sync(0xffffffffu, free_ok, 0);
      const bool ready = wait_or_abort(&gfull[s], par, abort_flag, p.status, p.wait_limit) && free_ok;
      const float4* sCol = sColAll + s * (kBK * 7);
      const float2* sSelf = sSelfAll + s * (kBK * kMaxG);
      unsigned char* a_stage = sA + s * 2 * kHalfBytes;
      unsigned char* x_stage = sX + s * kHalfBytes;
      if (it == 0) {   // the rows, staged by the producer before its first release
        xa = sRow[rr];
        xb = sRow[rr + 64];
      }
#pragma unroll 1
      for (int kg = kg_lo; kg < (ready ? kg_hi : kg_lo); ++kg) {
        const int k = 8 * kg + cq8;
        const int64_t l = (int64_t)kb * kBK + k;
        f2_t rr2[7], am2[7];
        f2_t s2[kOp ? 7 : 1];
        {
          const float4* cq = sCol + k * 7;
          const f2_t xx = f2(xa.x, xb.x), xy = f2(xa.y, xb.y), xz = f2(xa.z, xb.z);
          f2_t nnx = f2(0.f, 0.f), nny = nnx, nnz = nnx;
          if (kOp) {   // the column's normal, negated (d = x - y here)
            const float* gk = sGraw + s * (kBK * 64) + k * 64;
            nnx = f2(-gk[56], -gk[56]);
            nny = f2(-gk[57], -gk[57]);
            nnz = f2(-gk[58], -gk[58]);
          }
#pragma unroll
          for (int q = 0; q < 7; ++q) {
            const float4 y = cq[q];
            const f2_t dx = sub2(xx, f2(y.x, y.x)), dy = sub2(xy, f2(y.y, y.y)),
                       dz = sub2(xz, f2(y.z, y.z));
            const f2_t r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
            float r20, r21;
            f2split(r2, r20, r21);
            const f2_t rs = f2(rsqrtf_mufu(r20), rsqrtf_mufu(r21));
            rr2[q] = mul2(r2, rs);
            am2[q] = mul2(f2(y.w, y.w), rs);
            if (kOp)
              s2[kOp ? q : 0] = mul2(fma2(dx, nnx, fma2(dy, nny, mul2(dz, nnz))), mul2(rs, rs));
          }
        }
        const float2* selfk = sSelf + k * kMaxG;
        if (paired) {
          f2_t sa = f2(0.f, 0.f), ia = f2(0.f, 0.f), sb = f2(0.f, 0.f), ib = f2(0.f, 0.f);
          const f2_t kma = f2(kmi[0], kmi[0]), kmb = f2(kmi[1], kmi[1]);
          const f2_t kr2 = f2(kr[0], kr[0]);
#pragma unroll
          for (int q = 0; q < 7; ++q) {
            float e0, e1, e2, e3;
            f2split(mul2(kma, rr2[q]), e0, e1);
            f2split(mul2(kmb, rr2[q]), e2, e3);
            f2_t aa = mul2(am2[q], f2(ex2f(e0), ex2f(e1)));
            f2_t ab = mul2(am2[q], f2(ex2f(e2), ex2f(e3)));
            const f2_t ph2 = mul2(kr2, rr2[q]);
            f2_t cs, sn;
            if (q < kNP) {
              f2_t sg;
              sincos_poly2(ph2, cs, sn, sg);
              aa ^= sg;
              ab ^= sg;
            } else {
              float p0, p1;
              f2split(ph2, p0, p1);
              cs = f2(cosf_mufu(p0), cosf_mufu(p1));
              sn = f2(sinf_mufu(p0), sinf_mufu(p1));
            }
            if constexpr (kOp) {
              op_acc2(sa, ia, aa, cs, sn, s2[q], ph2, mul2(f2(kim[0], kim[0]), rr2[q]), cgr2,
                      cgi2, chr2, chi2, nchi2, m1);
              op_acc2(sb, ib, ab, cs, sn, s2[q], ph2, mul2(f2(kim[1], kim[1]), rr2[q]), cgr2,
                      cgi2, chr2, chi2, nchi2, m1);
            } else {
              sa = fma2(aa, cs, sa);
              ia = fma2(aa, sn, ia);
              sb = fma2(ab, cs, sb);
              ib = fma2(ab, sn, ib);
            }
          }
          // node `rank` into this CTA's stage, the other into the export buffer
          unsigned char* own = a_stage + kg * kHalfBytes + off;
          unsigned char* other = x_stage + off;
          put_rows(sa, ia, selfk, i0, i1, l, p.n, rank == 0 ? own : other);
          put_rows(sb, ib, selfk + 1, i0, i1, l, p.n, rank == 0 ? other : own);
        } else {
          f2_t sr2 = f2(0.f, 0.f), si2 = f2(0.f, 0.f);
          const f2_t kmi2 = f2(kmi[0], kmi[0]), kr2 = f2(kr[0], kr[0]);
#pragma unroll
          for (int q = 0; q < 7; ++q) {
            float e0, e1;
            f2split(mul2(kmi2, rr2[q]), e0, e1);
            f2_t a = mul2(am2[q], f2(ex2f(e0), ex2f(e1)));
            const f2_t ph2 = mul2(kr2, rr2[q]);
            f2_t cs, sn;
            if (q < kNP) {
              f2_t sg;
              sincos_poly2(ph2, cs, sn, sg);
              a ^= sg;
            } else {
              float p0, p1;
              f2split(ph2, p0, p1);
              cs = f2(cosf_mufu(p0), cosf_mufu(p1));
              sn = f2(sinf_mufu(p0), sinf_mufu(p1));
            }
            if constexpr (kOp) {
              op_acc2(sr2, si2, a, cs, sn, s2[q], ph2, mul2(f2(kim[0], kim[0]), rr2[q]), cgr2,
                      cgi2, chr2, chi2, nchi2, m1);
            } else {
              sr2 = fma2(a, cs, sr2);
              si2 = fma2(a, sn, si2);
            }
          }
          put_rows(sr2, si2, selfk, i0, i1, l, p.n, a_stage + kg * kHalfBytes + off);
        }
      }
      fence_proxy_async_smem();
      mbar_arrive(&afull[s]);
      if (!ready) break;
    }

    // ---------------- epilogue: TMEM -> FP32 partial Y of this CTA's node ----------------
    const bool ok = !*abort_flag && wait_or_abort(accfull, 0, abort_flag, p.status, p.wait_limit);
    if (__all_sync(0xffffffffu, ok)) {
      tc_fence_after();
      const int quarter = warp % 4;   // TMEM lanes this warp may read
      const int part = (warp - 3) / 4;
      const int erow = quarter * 32 + lane;
      const int64_t ei = row0 + erow;
      const size_t slot = (size_t)split * p.N + (p.order[myslot] & kNodeMask);
      for (uint32_t c0 = part * 16; c0 < acc_cols; c0 += 64) {
        float v[16];
        tmem_ld16(tmem_base + ((uint32_t)(quarter * 32) << 16) + c0, v);
        float* dst = p.Yp + (slot * acc_cols + c0) * p.n_pad + ei;
#pragma unroll
        for (int k = 0; k < 16; ++k) dst[(size_t)k * p.n_pad] = v[k];
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  // this CTA's MMAs, and with them their arrivals on the peer's barriers, complete (bounded)
  if (warp == 1 && lane == 0) mbar_wait(accfull, 0, kWaitLimit);
  cluster_sync_all();   // neither CTA issues anything more; peer_sent is visible
  if (warp == 1) {
    if (lane == 0 && paired) {
      // halves the peer sent that an aborted loop did not consume: let them land (bounded)
      const int sentp = min((int)*peer_sent, nit);
      for (int it = consumed; it < sentp; ++it)
        mbar_wait(&xin[it % kPA], (it / kPA) & 1, kWaitLimit);
    }
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem_base, tmem_cols);
  }
  cluster_sync_all();   // no copy into either CTA is still in flight
}

// Node-summed form: Y = sum_j c_j A(z_j) X_j (the right-hand side of an inverse power
// step, X_j per node) or (sum_j c_j A(z_j)) X (one X: the Schur complement S applied).
template <bool kOp>
__global__ void __launch_bounds__(kThreads, 1) mixed_sum_kernel(MixedParams p) {
  mixed_apply_unit<true, kOp, kPolyPointsMulti>(p, blockIdx.x, kNoTmem);
}

// Persistent grouped kernel over several problems: one CTA per SM takes work units from a
// global counter (dynamic scheduling); unit b belongs to problem k, the last k with
// unit_start[k] <= b (problems are ordered by decreasing work, so the largest are handed
// out first and the small ones fill the tail). The CTA allocates the TMEM columns of the
// widest problem once and keeps them for all its units.
__global__ void __launch_bounds__(kThreads, 1)
mixed_apply_grouped_kernel(const MixedParams* __restrict__ plist, const int* __restrict__ unit_start,
                           int nprob, int total, int* next_unit, uint32_t tmem_cols) {
  __shared__ uint32_t s_tmem;
  __shared__ int s_unit;
  const int warp = threadIdx.x / 32;
  if (warp == 1) {
    tmem_alloc(&s_tmem, tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = s_tmem;
  for (;;) {
    if (threadIdx.x == 0) s_unit = atomicAdd(next_unit, 1);
    __syncthreads();
    const int b = s_unit;
    __syncthreads();   // every thread has read s_unit before it is replaced
    if (b >= total) break;
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (unit_start[mid] <= b) lo = mid; else hi = mid - 1;
    }
    const MixedParams p = plist[lo];
    mixed_apply_unit<false, false, kPolyPointsMulti>(p, b - unit_start[lo], tmem_base);
    __syncthreads();   // the unit's barriers, shared memory and accumulators are free again
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem_base, tmem_cols);
}

// Basis planes in the tile-native layout the kernel copies per K-block: for K-block kb,
// chunk c, plane pl, the 2C x 16 block in core matrices (row group ng, k group kg) of
// 8 rows x 8 bf16, row stride 16 B, at ng * 256 + kg * 128 bytes.
__global__ void prep_basis_planes_kernel(const double* __restrict__ V, int64_t ldv, int64_t n,
                                         int nu, int nup, int C, int nK,
                                         __nv_bfloat16* __restrict__ Bp, float2* __restrict__ V32,
                                         int* status) {
  // one thread per source element (panel l, column col); the split is formed in FP32
  // (hi + lo carries 16 significant bits, far above FP32's own rounding). A non-finite
  // basis entry is recorded in the status word (the projection is then invalid).
  const int64_t rows = (int64_t)nK * kBK;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= rows * nup) return;
  const int64_t l = t % rows;
  const int col = (int)(t / rows);
  float vr = 0.f, vi = 0.f;
  if (l < n && col < nu) {
    const double2 v = reinterpret_cast<const double2*>(V)[(int64_t)col * ldv + l];
    if (!isfinite(v.x) || !isfinite(v.y)) atomicOr(status, kStatusNonFinite);
    vr = (float)v.x;
    vi = (float)v.y;
    V32[(int64_t)col * n + l] = make_float2(vr, vi);
  }
  const __nv_bfloat16 vr_hi = __float2bfloat16(vr), vi_hi = __float2bfloat16(vi);
  const __nv_bfloat16 vr_lo = __float2bfloat16(vr - __bfloat162float(vr_hi));
  const __nv_bfloat16 vi_lo = __float2bfloat16(vi - __bfloat162float(vi_hi));
  const __nv_bfloat16 vals[4][2] = {{vr_hi, vi_hi},               // [Vr | Vi]
                                    {vr_lo, vi_lo},               // [Vr_lo | Vi_lo]
                                    {__hneg(vi_hi), vr_hi},       // [-Vi | Vr]
                                    {__hneg(vi_lo), vr_lo}};      // [-Vi_lo | Vr_lo]
  // position in the tile-native layout: (kb, chunk, plane, 8-row group, k half, row, k)
  const int kb = (int)(l / kBK), kin = (int)(l % kBK);
  const int kg = kin / 8, k8 = kin % 8;
  const int c = col / C, rc = col % C;
  const int nchunks = nup / C, ngroups = 2 * C / 8;
#pragma unroll
  for (int pl = 0; pl < 4; ++pl)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int rowN = h * C + rc;
      const int64_t idx =
          (((((int64_t)kb * nchunks + c) * 4 + pl) * ngroups + rowN / 8) * 2 + kg) * 64 +
          (rowN % 8) * 8 + k8;
      Bp[idx] = vals[pl][h];
    }
}

// Partial products P_r,j = V^H Y_j on the tensor core: a CTA takes node j, the rows of
// part r (32 rows per stage) and one quadrant (ca, cb) of P_j: the basis columns of chunk ca
// against the Y columns of chunk cb (C columns each; one quadrant when nup <= 128).
//  * the A operand is the prepared basis planes [Vr | Vi] (hi and lo) of the main kernel,
//    split into two M = 128 halves (Vr rows in half 0, Vi rows in half 1, zero rows above C)
//    so that each output's real and imaginary combinations meet in one TMEM lane;
//  * 8 converter warps sum the FP32 partials Y of the column splits, split them into BF16
//    hi/lo and store them as the B operand (N = 2 C = [Yr | Yi], K = rows, canonical
//    K-major layout);
//  * one MMA thread issues per 16-row K-block and half: A_hi B_hi + A_hi B_lo + A_lo B_hi
//    into D_h (128 x 2 C, FP32, TMEM);
//  * epilogue, lane a: Re = D0[a][b] + D1[a][C + b], Im = D0[a][C + b] - D1[a][b]
//    (conj(V)^T Y = Vr^T Yr + Vi^T Yi + i (Vr^T Yi - Vi^T Yr)), written as FP64 partials.
// Every wait is bounded; a timeout aborts the block cleanly with an error status.
constexpr int kVStages = 2;
constexpr int kVKB = 2;                       // 16-row K-blocks per stage
constexpr int kVRows = 16 * kVKB;             // rows per stage
constexpr int64_t kVMaxRows = 4096;           // rows per CTA (row part) at most
constexpr int kVConvWarps = 8;
constexpr int kVConvThreads = 32 * kVConvWarps;
constexpr int kVThreads = 32 * (2 + kVConvWarps);
constexpr uint32_t kVHalfBytes = 128 * 32;    // one 128-row x 16-k BF16 operand block

struct VhyLayout {
  uint32_t a_stage, b_stage, b_off, bar_off, misc_off, total, tmem_cols;
};
__host__ __device__ inline VhyLayout vhy_layout(int C) {
  VhyLayout L;
  L.a_stage = kVKB * 2 * 2 * kVHalfBytes;          // [kb][plane hi/lo][half]
  L.b_stage = kVKB * 2 * (uint32_t)(2 * C) * 32;   // [kb][plane hi/lo] N = 2 C rows x 32 B
  L.b_off = kVStages * L.a_stage;
  L.bar_off = L.b_off + kVStages * L.b_stage;
  L.misc_off = L.bar_off + 8 * 8;                  // 7 mbarriers (+1 pad)
  L.total = L.misc_off + 16;
  const uint32_t need = 4u * C + (C % 16 ? 8u : 0u);   // two halves x 2 C columns (+ overread)
  L.tmem_cols = 32;
  while (L.tmem_cols < need) L.tmem_cols <<= 1;
  return L;
}

// TPT: column/row-group tasks per converter thread and stage (8 C / 256 rounded up to 1, 2, 4).
template <int TPT>
__global__ void __launch_bounds__(kVThreads, 2)
mixed_vhy_tc_kernel(const __nv_bfloat16* __restrict__ Bp, const float* __restrict__ Yp,
                    int64_t n, int n_pad, int nu, int C, int nchunks, int N, int nK, int slices,
                    int64_t rows_per_part, double* __restrict__ part, int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const VhyLayout L = vhy_layout(C);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
  uint64_t* afull = bars;        // [2] basis planes landed
  uint64_t* bfull = bars + 2;    // [2] converted Y stored
  uint64_t* empty = bars + 4;    // [2] MMAs done with the stage
  uint64_t* accfull = bars + 6;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.misc_off);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.misc_off + 4);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int j = blockIdx.x;
  const int64_t r_begin = (int64_t)blockIdx.y * rows_per_part;
  const int64_t r_end = min(n, r_begin + rows_per_part);
  const int nst = (int)((r_end - r_begin + kVRows - 1) / kVRows);
  const int twoC = 2 * C;
  const uint32_t plane_bytes = (uint32_t)twoC * 32;   // one prepared plane of a chunk and K-block
  const uint32_t half_bytes = (uint32_t)C * 32;       // its Vr or Vi rows
  const int ca = (int)blockIdx.z / nchunks;           // basis chunk (rows of P_j)
  const int cb = (int)blockIdx.z % nchunks;           // Y chunk (columns of P_j)
  const int acc_cols = nchunks * twoC;                // FP32 partial columns per node

  // zero the A blocks once: rows C..127 of each half stay zero (the copies fill rows < C)
  for (uint32_t x = threadIdx.x; x < kVStages * L.a_stage / 16; x += blockDim.x)
    reinterpret_cast<uint4*>(smem)[x] = make_uint4(0u, 0u, 0u, 0u);
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    for (int st = 0; st < kVStages; ++st) {
      mbar_init(&afull[st], 1);
      mbar_init(&bfull[st], kVConvThreads);
      mbar_init(&empty[st], 1);
    }
    mbar_init(accfull, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, L.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ---------------- basis planes: bulk copies ----------------
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < nst; ++it) {
        const int st = it % kVStages;
        const uint32_t par = (it / kVStages) & 1;
        if (!wait_or_abort(&empty[st], par ^ 1, abort_flag, status)) break;
        const int kbg0 = (int)((r_begin + (int64_t)it * kVRows) / 16);
        const int nkb = min(kVKB, nK - kbg0);
        mbar_arrive_expect_tx(&afull[st], (uint32_t)nkb * 4u * half_bytes);
        unsigned char* a_st = smem + st * L.a_stage;
        for (int kb = 0; kb < nkb; ++kb) {
          // K-block sets of nchunks x 4 planes; chunk ca's [Vr|Vi] hi and lo planes
          const unsigned char* src = reinterpret_cast<const unsigned char*>(Bp) +
                                     (size_t)(kbg0 + kb) * (4u * plane_bytes * nchunks) +
                                     (size_t)ca * 4u * plane_bytes;
          for (int pl = 0; pl < 2; ++pl)
            for (int h = 0; h < 2; ++h)
              bulk_g2s(a_st + ((kb * 2 + pl) * 2 + h) * kVHalfBytes,
                       src + pl * plane_bytes + h * half_bytes, half_bytes, &afull[st]);
        }
        ++issued;
      }
      if (*abort_flag)
        for (int it = max(0, issued - kVStages); it < issued; ++it)
          mbar_wait(&afull[it % kVStages], (it / kVStages) & 1, kWaitLimit);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, (uint32_t)twoC);
      bool first = true;
      for (int it = 0; it < nst; ++it) {
        const int st = it % kVStages;
        const uint32_t par = (it / kVStages) & 1;
        if (!wait_or_abort(&afull[st], par, abort_flag, status)) break;
        if (!wait_or_abort(&bfull[st], par, abort_flag, status)) break;
        tc_fence_after();
        const int kbg0 = (int)((r_begin + (int64_t)it * kVRows) / 16);
        const int nkb = min(kVKB, nK - kbg0);
        const uint32_t a_st = smem_u32(smem + st * L.a_stage);
        const uint32_t b_st = smem_u32(smem + L.b_off + st * L.b_stage);
        for (int kb = 0; kb < nkb; ++kb) {
          const uint64_t bh = smem_desc(b_st + (kb * 2 + 0) * plane_bytes, 128, 256);
          const uint64_t bl = smem_desc(b_st + (kb * 2 + 1) * plane_bytes, 128, 256);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const uint32_t d = tmem_base + h * twoC;
            const uint64_t ah = smem_desc(a_st + ((kb * 2 + 0) * 2 + h) * kVHalfBytes, 128, 256);
            const uint64_t al = smem_desc(a_st + ((kb * 2 + 1) * 2 + h) * kVHalfBytes, 128, 256);
            mma_bf16(d, ah, bh, idesc, first ? 0u : 1u);
            mma_bf16(d, ah, bl, idesc, 1u);
            mma_bf16(d, al, bh, idesc, 1u);
          }
          first = false;
        }
        mma_commit(&empty[st]);
      }
      mma_commit(accfull);
    }
  } else {
    // ---------------- converters: Y (sum of the splits) -> BF16 hi/lo B operand ----------
    const int ct = threadIdx.x - 64;
    const int tasks = 4 * twoC;   // (column n, 8-row group g) pairs of a stage
    constexpr int GS = 4 / TPT;   // column splits loaded together: 8 x 16 B in flight
    for (int it = 0; it < nst; ++it) {
      const int st = it % kVStages;
      const uint32_t par = (it / kVStages) & 1;
      const bool ok = wait_or_abort(&empty[st], par ^ 1, abort_flag, status);
      const int64_t r0 = r_begin + (int64_t)it * kVRows;
      unsigned char* b_st = smem + L.b_off + st * L.b_stage;
      float y[TPT][8];
#pragma unroll
      for (int q = 0; q < TPT; ++q)
#pragma unroll
        for (int k = 0; k < 8; ++k) y[q][k] = 0.f;
      // Y of this thread's tasks, summed over the column splits in order; lanes take
      // consecutive columns, rows r0 + 8 g .. + 7 (< n_pad: stages end by round_up(n, 32))
      for (int s0 = 0; ok && s0 < slices; s0 += GS) {
        float4 u[GS][TPT][2];
#pragma unroll
        for (int g2 = 0; g2 < GS; ++g2)
#pragma unroll
          for (int q = 0; q < TPT; ++q) {
            const int t = ct + q * kVConvThreads;
            u[g2][q][0] = u[g2][q][1] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (s0 + g2 < slices && t < tasks) {
              const int nn = t % twoC, g = t / twoC;
              const float* src =
                  Yp + (((size_t)(s0 + g2) * N + j) * (size_t)acc_cols + (size_t)cb * twoC + nn) *
                           (size_t)n_pad + r0 + 8 * g;
              u[g2][q][0] = *reinterpret_cast<const float4*>(src);
              u[g2][q][1] = *reinterpret_cast<const float4*>(src + 4);
            }
          }
#pragma unroll
        for (int g2 = 0; g2 < GS; ++g2)
#pragma unroll
          for (int q = 0; q < TPT; ++q) {
            y[q][0] += u[g2][q][0].x; y[q][1] += u[g2][q][0].y;
            y[q][2] += u[g2][q][0].z; y[q][3] += u[g2][q][0].w;
            y[q][4] += u[g2][q][1].x; y[q][5] += u[g2][q][1].y;
            y[q][6] += u[g2][q][1].z; y[q][7] += u[g2][q][1].w;
          }
      }
#pragma unroll
      for (int q = 0; q < TPT; ++q) {
        const int t = ct + q * kVConvThreads;
        if (!ok || t >= tasks) continue;
        const int nn = t % twoC, g = t / twoC;
        if (r0 + 8 * g >= r_end) {
#pragma unroll
          for (int k = 0; k < 8; ++k) y[q][k] = 0.f;
        }
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          hi[k] = pack_bf16(y[q][2 * k], y[q][2 * k + 1]);
          lo[k] = pack_bf16(y[q][2 * k] - __uint_as_float(hi[k] << 16),
                            y[q][2 * k + 1] - __uint_as_float(hi[k] & 0xFFFF0000u));
        }
        const int kb = g / 2, kh = g % 2;
        const uint32_t off = (uint32_t)(nn / 8) * 256 + kh * 128 + (nn % 8) * 16;
        *reinterpret_cast<uint4*>(b_st + (kb * 2 + 0) * plane_bytes + off) =
            make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(b_st + (kb * 2 + 1) * plane_bytes + off) =
            make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
      fence_proxy_async_smem();
      mbar_arrive(&bfull[st]);
      if (!ok) break;
    }
    // ---------------- epilogue: TMEM -> FP64 partial ----------------
    const bool ok = !*abort_flag && wait_or_abort(accfull, 0, abort_flag, status);
    const int quarter = warp % 4;
    const int a = ca * C + quarter * 32 + lane;   // row of P_j
    if (__all_sync(0xffffffffu, ok) && quarter * 32 < C) {
      tc_fence_after();
      const int side = (warp - 2) / 4;   // two warps per lane quarter split the columns
      const uint32_t lane_addr = tmem_base + ((uint32_t)(quarter * 32) << 16);
      double2* P = reinterpret_cast<double2*>(part) + ((int64_t)blockIdx.y * N + j) * nu * nu;
      for (int b0 = 16 * side; b0 < C; b0 += 32) {
        float d0r[16], d0i[16], d1r[16], d1i[16];
        tmem_ld16(lane_addr + b0, d0r);                // Vr^T Yr
        tmem_ld16(lane_addr + C + b0, d0i);            // Vr^T Yi
        tmem_ld16(lane_addr + twoC + b0, d1r);         // Vi^T Yr
        tmem_ld16(lane_addr + twoC + C + b0, d1i);     // Vi^T Yi
        if (a < nu) {
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int b = cb * C + b0 + k;   // column of P_j
            if (b < nu)
              P[(int64_t)b * nu + a] = make_double2((double)d0r[k] + (double)d1i[k],
                                                    (double)d0i[k] - (double)d1r[k]);
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    if (lane == 0) mbar_wait(accfull, 0, kWaitLimit);
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem_base, L.tmem_cols);
  }
}

// Bhat_j = w_j sum_r P_r,j (parts added in order: deterministic).
__global__ void mixed_vhy_reduce_kernel(const double* __restrict__ part, int parts, int N, int nu,
                                        const double* __restrict__ w, double* __restrict__ Bhat) {
  const int64_t per = (int64_t)nu * nu;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= per * N) return;
  const int j = (int)(t / per);
  const double2* P = reinterpret_cast<const double2*>(part);
  double2 s = make_double2(0.0, 0.0);
  for (int r = 0; r < parts; ++r) {
    const double2 v = P[(int64_t)r * per * N + t];
    s.x += v.x;
    s.y += v.y;
  }
  const double2 wj = reinterpret_cast<const double2*>(w)[j];
  reinterpret_cast<double2*>(Bhat)[t] = make_double2(wj.x * s.x - wj.y * s.y, wj.x * s.y + wj.y * s.x);
}

__global__ void mixed_av_kernel(int64_t n, int n_pad, int nu, int N, int S, int acc_cols, int C,
                                const float* __restrict__ Yp, double* __restrict__ AV) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)N * nu * n) return;
  const int64_t i = t % n;
  const int b = (int)((t / n) % nu);
  const int j = (int)(t / (n * (int64_t)nu));
  const int colr = (b / C) * 2 * C + (b % C);
  double re = 0.0, im = 0.0;
  for (int s = 0; s < S; ++s) {
    const float* base = Yp + ((size_t)s * N + j) * acc_cols * (size_t)n_pad;
    re += base[(size_t)colr * n_pad + i];
    im += base[(size_t)(colr + C) * n_pad + i];
  }
  reinterpret_cast<double2*>(AV)[t] = make_double2(re, im);
}

// Column splits: the fewest that fill whole waves of the device to >= 90 %.
int choose_splits(int64_t units1, int nK, int sms) {
  int best = 1;
  double best_eff = 0.0;
  const int smax = std::max(1, std::min(8, nK / 4));
  for (int S = 1; S <= smax; ++S) {
    const int64_t u = units1 * S;
    const int64_t waves = (u + sms - 1) / sms;
    const double eff = (double)u / (double)(waves * sms);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = S;
    }
    if (eff >= 0.9) break;
  }
  return best;
}

// Everything one mixed projection of one context needs besides its launches.
struct MixedPlan {
  MixedParams p{};
  int64_t units = 0;          // work units of the main kernel
  int slices = 0;             // slices of the FP32 partials: the S column splits, then the
                              // near-field correction when it is active
  int64_t vparts = 0, rows_per_vpart = 0;
  bool pair = false;          // twin pairs across CTA clusters (mixed_pair_kernel)
  uint32_t smem = 0;          // dynamic shared memory of the main kernel
  const double* V = nullptr;
  int64_t ldv = 0;
  float2* V32 = nullptr;
  __nv_bfloat16* Bp = nullptr;
  double* vpart = nullptr;
  SmemLayout L{};
};

// Parameters, scratch and FP32 self terms of one projection; S > 0 forces the number of
// column splits (else the fewest that fill the device's waves), Gmax > 0 caps the nodes per
// work unit (else up to kMaxG); allow_pair lets units of one node run as twin pairs across
// two-CTA clusters when the contour has twin nodes.
bem_status mixed_plan(bem_ctx* ctx, const double* V, int64_t ldv, int nu, int S, int Gmax,
                      MixedPlan& plan, cudaStream_t s, bool allow_pair = false) {
  const int64_t n = ctx->geo.n;
  const int N = ctx->con.N;
  MixedParams& p = plan.p;
  p = MixedParams{};
  p.n = n;
  p.N = N;
  p.nu = nu;
  p.nup = (nu + 7) / 8 * 8;
  p.C = p.nup <= 128 ? p.nup : 128;
  if (p.nup % p.C != 0) p.nup = (p.nup + p.C - 1) / p.C * p.C;
  p.nchunks = p.nup / p.C;
  const int acc_cols = 2 * p.nup;
  p.G = std::max(1, std::min(std::min(N, Gmax > 0 ? std::min(Gmax, kMaxG) : kMaxG), 512 / acc_cols));
  p.nG = (N + p.G - 1) / p.G;
  p.nK = (int)((n + kBK - 1) / kBK);
  p.n_pad = (int)((n + kBM - 1) / kBM * kBM);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  const int64_t rtiles = p.n_pad / kBM;
  plan.pair = allow_pair && p.G == 1 && N >= 2 && ctx->con.twins > 0 && ctx->twin_clusters;
  // CTAs per column split: one per (row tile, node), or two per (row tile, pair of slots)
  const int64_t units1 = plan.pair ? rtiles * 2 * ((N + 1) / 2) : rtiles * p.nG;
  p.S = S > 0 ? std::max(1, std::min(S, std::max(1, p.nK / 4)))
              : choose_splits(units1, p.nK, std::max(1, sms));
  plan.units = units1 * p.S;

  // scratch: basis planes, FP32 partials, FP32 copy of V, V^H Y partials
  const size_t bp_bytes = (size_t)p.nK * 256 * p.nup;
  const size_t bp_off = 0;
  const size_t yp_off = (bp_bytes + 255) / 256 * 256;
  plan.slices = p.S + (near_active(ctx) ? 1 : 0);
  const size_t yp_bytes = (size_t)plan.slices * N * acc_cols * p.n_pad * sizeof(float);
  // V^H Y partials on the tensor core: one wave of (node, row part, chunk quadrant) CTAs,
  // 32-row stages; two CTAs per SM when their shared memory and TMEM columns both fit twice
  {
    const VhyLayout VL = vhy_layout(p.C);
    const int per_sm = (VL.total <= 110 * 1024 && VL.tmem_cols <= 256) ? 2 : 1;
    const int64_t slots = (int64_t)std::max(1, sms) * per_sm;
    const int64_t tparts = std::max<int64_t>(1, slots / ((int64_t)N * p.nchunks * p.nchunks));
    plan.rows_per_vpart = ((n + tparts - 1) / tparts + kVRows - 1) / kVRows * kVRows;
    // at most kVMaxRows rows per FP32 TMEM accumulation: its rounding error grows with the
    // number of accumulated 16-row steps (up to 256 u32 here); the parts are summed in FP64
    plan.rows_per_vpart = std::min<int64_t>(plan.rows_per_vpart, kVMaxRows);
    plan.vparts = (n + plan.rows_per_vpart - 1) / plan.rows_per_vpart;
  }
  const size_t v32_off = (yp_off + yp_bytes + 255) / 256 * 256;
  const size_t v32_bytes = (size_t)n * nu * sizeof(float2);
  const size_t vp_off = (v32_off + v32_bytes + 255) / 256 * 256;
  const size_t vp_bytes = (size_t)plan.vparts * N * nu * nu * 2 * sizeof(double);
  bem_status st = ensure_self32(ctx, s);
  if (st != BEM_OK) return st;
  st = ensure_scratch(ctx, vp_off + vp_bytes);
  if (st != BEM_OK) return st;
  unsigned char* scr = reinterpret_cast<unsigned char*>(ctx->d_scratch);
  plan.Bp = reinterpret_cast<__nv_bfloat16*>(scr + bp_off);
  p.Bp = plan.Bp;
  p.Yp = reinterpret_cast<float*>(scr + yp_off);
  p.cx = ctx->geo.cx;
  p.qp = ctx->geo.qp;
  p.qw = ctx->geo.qw;
  p.self32 = reinterpret_cast<const float2*>(ctx->con.self32);
  p.pack32 = ctx->geo.pack32;
  p.z = ctx->con.z;
  p.order = ctx->con.order;
  p.status = ctx->d_status;
  p.wait_limit = ctx->stage_wait_limit;
  p.op = ctx->op;
  plan.V = V;
  plan.ldv = ldv;
  plan.V32 = reinterpret_cast<float2*>(scr + v32_off);
  plan.vpart = reinterpret_cast<double*>(scr + vp_off);
  plan.L = smem_layout(p.G, p.nup);
  plan.smem = plan.pair ? pair_layout(p.nup).total : plan.L.total;
  return BEM_OK;
}

// Basis planes and FP32 copy of V (before the main kernel).
void mixed_pre(bem_ctx* ctx, const MixedPlan& plan, cudaStream_t s) {
  const MixedParams& p = plan.p;
  const int64_t prep_total = (int64_t)p.nK * kBK * p.nup;
  prep_basis_planes_kernel<<<(unsigned)((prep_total + 255) / 256), 256, 0, s>>>(
      plan.V, plan.ldv, p.n, p.nu, p.nup, p.C, p.nK, plan.Bp, plan.V32, p.status);
  ctx->launches++;
}

// V^H Y, weights, optional Y (after the main kernel).
void mixed_post(bem_ctx* ctx, const MixedPlan& plan, double* Bhat, double* AV, cudaStream_t s) {
  const MixedParams& p = plan.p;
  const int acc_cols = 2 * p.nup;
  {
    const dim3 grid((unsigned)p.N, (unsigned)plan.vparts, (unsigned)(p.nchunks * p.nchunks));
    const uint32_t sm = vhy_layout(p.C).total;
    auto* kern = p.C <= 32 ? mixed_vhy_tc_kernel<1>
                           : (p.C <= 64 ? mixed_vhy_tc_kernel<2> : mixed_vhy_tc_kernel<4>);
    kern<<<grid, kVThreads, sm, s>>>(plan.Bp, p.Yp, p.n, p.n_pad, p.nu, p.C, p.nchunks, p.N,
                                     p.nK, plan.slices, plan.rows_per_vpart, plan.vpart, p.status);
  }
  const int64_t outs = (int64_t)p.N * p.nu * p.nu;
  mixed_vhy_reduce_kernel<<<(unsigned)((outs + 255) / 256), 256, 0, s>>>(
      plan.vpart, (int)plan.vparts, p.N, p.nu, ctx->con.w, Bhat);
  ctx->launches += 2;
  if (AV) {
    const int64_t tot = (int64_t)p.N * p.nu * p.n;
    mixed_av_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(p.n, p.n_pad, p.nu, p.N,
                                                                  plan.slices, acc_cols, p.C, p.Yp,
                                                                  AV);
    ctx->launches++;
  }
}

using MixedKernel = void (*)(MixedParams);

// The fused kernel with np polynomial points (0..kPolyPointsMax), single layer or general
// operator.
MixedKernel mixed_kernel(bool general, int np) {
  static const MixedKernel single[kPolyPointsMax + 1] = {
      mixed_apply_kernel<false, 0>, mixed_apply_kernel<false, 1>, mixed_apply_kernel<false, 2>,
      mixed_apply_kernel<false, 3>, mixed_apply_kernel<false, 4>};
  static const MixedKernel op[kPolyPointsMax + 1] = {
      mixed_apply_kernel<true, 0>, mixed_apply_kernel<true, 1>, mixed_apply_kernel<true, 2>,
      mixed_apply_kernel<true, 3>, mixed_apply_kernel<true, 4>};
  np = std::max(0, std::min(np, kPolyPointsMax));
  return general ? op[np] : single[np];
}

MixedKernel mixed_pair(bool general, int np) {
  static const MixedKernel single[kPolyPointsMax + 1] = {
      mixed_pair_kernel<false, 0>, mixed_pair_kernel<false, 1>, mixed_pair_kernel<false, 2>,
      mixed_pair_kernel<false, 3>, mixed_pair_kernel<false, 4>};
  static const MixedKernel op[kPolyPointsMax + 1] = {
      mixed_pair_kernel<true, 0>, mixed_pair_kernel<true, 1>, mixed_pair_kernel<true, 2>,
      mixed_pair_kernel<true, 3>, mixed_pair_kernel<true, 4>};
  np = std::max(0, std::min(np, kPolyPointsMax));
  return general ? op[np] : single[np];
}

// Polynomial points of a projection with G nodes per unit: the context's override, else the
// measured default of the unit shape.
int poly_points(const bem_ctx* ctx, int G) {
  if (ctx->poly_points >= 0) return std::min(ctx->poly_points, kPolyPointsMax);
  return G > 1 ? kPolyPointsMulti : kPolyPointsSingle;
}

bem_status set_mixed_smem(bem_ctx* ctx, uint32_t bytes) {
  bem_status st = BEM_OK;
  for (int np = 0; np <= kPolyPointsMax && st == BEM_OK; ++np)
    for (bool general : {false, true}) {
      st = cuda_check(ctx, cudaFuncSetAttribute(mixed_kernel(general, np),
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)bytes),
                      "mixed kernel attribute");
      if (st != BEM_OK) return st;
      st = cuda_check(ctx, cudaFuncSetAttribute(mixed_pair(general, np),
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)bytes),
                      "mixed kernel attribute");
      if (st != BEM_OK) return st;
    }
  for (const void* f : {(const void*)mixed_vhy_tc_kernel<1>, (const void*)mixed_vhy_tc_kernel<2>,
                        (const void*)mixed_vhy_tc_kernel<4>}) {
    st = cuda_check(ctx, cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)vhy_layout(128).total),
                    "mixed kernel attribute");
    if (st != BEM_OK) return st;
  }
  return cuda_check(ctx, cudaFuncSetAttribute(mixed_apply_grouped_kernel,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)bytes),
                    "mixed kernel attribute");
}

// ---------------------------------------------------------------------------------------
// Node-summed form of the fused kernel (Algorithm 1, Eq. linsyssim): Y = sum_j c_j A(z_j) X_j
// with one X_j per node (the right-hand side b of an inverse power step) or one X for all
// nodes (the Schur complement S = sum_j c_j A(z_j) applied to X). Same evaluation and
// BF16x3 tcgen05 contraction as the projection; the G nodes of a unit accumulate into one
// TMEM accumulator, the units of node group gg and split write slice gg S + split, and the
// slices are summed in a fixed order.

// X (FP32 complex, column-major with leading dimension ldx, node blocks node_stride apart)
// -> BF16 hi/lo basis planes, one set of nK * 256 * nup bytes per node.
__global__ void prep_planes32_kernel(const float2* __restrict__ X, int64_t ldx,
                                     int64_t node_stride, int64_t n, int nu, int nup, int C,
                                     int nK, int nnodes, __nv_bfloat16* __restrict__ Bp) {
  const int64_t rows = (int64_t)nK * kBK;
  const int64_t per = rows * nup;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= per * nnodes) return;
  const int node = (int)(t / per);
  const int64_t l = (t % per) % rows;
  const int col = (int)((t % per) / rows);
  float vr = 0.f, vi = 0.f;
  if (l < n && col < nu) {
    const float2 v = X[node * node_stride + (int64_t)col * ldx + l];
    vr = v.x;
    vi = v.y;
  }
  const __nv_bfloat16 vr_hi = __float2bfloat16(vr), vi_hi = __float2bfloat16(vi);
  const __nv_bfloat16 vr_lo = __float2bfloat16(vr - __bfloat162float(vr_hi));
  const __nv_bfloat16 vi_lo = __float2bfloat16(vi - __bfloat162float(vi_hi));
  const __nv_bfloat16 vals[4][2] = {{vr_hi, vi_hi}, {vr_lo, vi_lo}, {__hneg(vi_hi), vr_hi},
                                    {__hneg(vi_lo), vr_lo}};
  const int kb = (int)(l / kBK), kin = (int)(l % kBK);
  const int kg = kin / 8, k8 = kin % 8;
  const int c = col / C, rc = col % C;
  const int nchunks = nup / C, ngroups = 2 * C / 8;
  __nv_bfloat16* B = Bp + (size_t)node * (size_t)nK * 128 * nup;
#pragma unroll
  for (int pl = 0; pl < 4; ++pl)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int rowN = h * C + rc;
      const int64_t idx =
          (((((int64_t)kb * nchunks + c) * 4 + pl) * ngroups + rowN / 8) * 2 + kg) * 64 +
          (rowN % 8) * 8 + k8;
      B[idx] = vals[pl][h];
    }
}

// out (FP32 complex, n x nu, leading dimension n) = sum over the slices, in slice order
__global__ void sum_slices_kernel(const float* __restrict__ Yp, int slices, int acc_cols, int C,
                                  int64_t n, int n_pad, int nu, float2* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * nu) return;
  const int64_t i = t % n;
  const int c = (int)(t / n);
  const int colr = (c / C) * 2 * C + c % C;
  float re = 0.f, im = 0.f;
  for (int sl = 0; sl < slices; ++sl) {
    const float* base = Yp + (size_t)sl * acc_cols * n_pad;
    re += base[(size_t)colr * n_pad + i];
    im += base[(size_t)(colr + C) * n_pad + i];
  }
  out[t] = make_float2(re, im);
}

constexpr uint32_t kSmemMax = 227 * 1024;

struct SumPlan {
  MixedParams p{};
  int64_t units = 0;
  int slices = 0;
  int nnodes = 1;            // basis plane sets (N with one X per node)
  SmemLayout L{};
  size_t bp_off = 0, yp_off = 0, cf_off = 0, bytes = 0;
};

SumPlan sum_plan(bem_ctx* ctx, int nu, bool per_node) {
  SumPlan plan;
  MixedParams& p = plan.p;
  const int64_t n = ctx->geo.n;
  const int N = ctx->con.N;
  p.n = n;
  p.N = N;
  p.nu = nu;
  p.nup = (nu + 7) / 8 * 8;
  p.C = p.nup <= 128 ? p.nup : 128;
  if (p.nup % p.C != 0) p.nup = (p.nup + p.C - 1) / p.C * p.C;
  p.nchunks = p.nup / p.C;
  // nodes per unit: 4, else 2, else 1 (even counts keep twin pairs together), within the
  // shared memory (per-node basis planes take a set per node and stage)
  int G = std::min(N, kMaxG);
  while (G > 1 && smem_layout(G, p.nup, per_node ? G : 1).total > kSmemMax) G = G > 2 ? 2 : 1;
  p.G = G;
  p.nG = (N + G - 1) / G;
  p.nK = (int)((n + kBK - 1) / kBK);
  p.n_pad = (int)((n + kBM - 1) / kBM * kBM);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  const int64_t rtiles = p.n_pad / kBM;
  // units: row tiles x column splits, and chunks of node groups only when those are too few
  // to fill the device (every chunk and split is a slice of FP32 partials)
  sms = std::max(1, sms);
  int64_t ngc = 1;
  p.S = choose_splits(rtiles, p.nK, sms);
  if (rtiles * p.S < sms) {
    ngc = std::min<int64_t>(p.nG, (sms + rtiles * p.S - 1) / (rtiles * p.S));
    p.S = choose_splits(rtiles * ngc, p.nK, sms);
  }
  p.gchunk = (int)((p.nG + ngc - 1) / ngc);
  p.ngc = (p.nG + p.gchunk - 1) / p.gchunk;
  plan.units = rtiles * p.ngc * p.S;
  plan.slices = p.ngc * p.S;
  plan.nnodes = per_node ? N : 1;
  p.sum = 1;
  const size_t set_bytes = (size_t)p.nK * 256 * p.nup;
  p.b_node_stride = per_node ? (int64_t)set_bytes : 0;
  plan.bp_off = 0;
  plan.yp_off = (plan.nnodes * set_bytes + 255) / 256 * 256;
  plan.cf_off = plan.yp_off +
                ((size_t)plan.slices * 2 * p.nup * p.n_pad * sizeof(float) + 255) / 256 * 256;
  plan.bytes = plan.cf_off + (size_t)N * sizeof(float2);
  plan.L = smem_layout(G, p.nup, per_node ? G : 1);
  return plan;
}

}  // namespace

size_t mixed_sum_work_bytes(bem_ctx* ctx, int nu, bool per_node) {
  return sum_plan(ctx, nu, per_node).bytes;
}

bem_status mixed_sum_apply(bem_ctx* ctx, const float2* X, int64_t ldx, int64_t node_stride,
                           bool per_node, int nu, const double* coef_host, float2* out,
                           void* work, cudaStream_t s) {
  SumPlan plan = sum_plan(ctx, nu, per_node);
  MixedParams& p = plan.p;
  unsigned char* w = reinterpret_cast<unsigned char*>(work);
  __nv_bfloat16* Bp = reinterpret_cast<__nv_bfloat16*>(w + plan.bp_off);
  p.Bp = Bp;
  p.Yp = reinterpret_cast<float*>(w + plan.yp_off);
  float2* cf = reinterpret_cast<float2*>(w + plan.cf_off);
  p.coef = cf;
  p.cx = ctx->geo.cx;
  p.qp = ctx->geo.qp;
  p.qw = ctx->geo.qw;
  p.pack32 = ctx->geo.pack32;
  p.z = ctx->con.z;
  p.order = ctx->con.order;
  p.status = ctx->d_status;
  p.wait_limit = ctx->stage_wait_limit;
  p.op = ctx->op;
  bem_status st = ensure_self32(ctx, s);
  if (st != BEM_OK) return st;
  p.self32 = reinterpret_cast<const float2*>(ctx->con.self32);
  std::vector<float2> ch(p.N);
  for (int j = 0; j < p.N; ++j) ch[j] = make_float2((float)coef_host[2 * j], (float)coef_host[2 * j + 1]);
  st = cuda_check(ctx, cudaMemcpyAsync(cf, ch.data(), p.N * sizeof(float2), cudaMemcpyHostToDevice, s),
                  "coefficient copy");
  if (st != BEM_OK) return st;
  const int64_t prep = (int64_t)plan.nnodes * p.nK * kBK * p.nup;
  prep_planes32_kernel<<<(unsigned)((prep + 255) / 256), 256, 0, s>>>(
      X, ldx, node_stride, p.n, nu, p.nup, p.C, p.nK, plan.nnodes, Bp);
  auto* sum_kern = op_single(ctx->op) ? mixed_sum_kernel<false> : mixed_sum_kernel<true>;
  st = cuda_check(ctx, cudaFuncSetAttribute(sum_kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)plan.L.total),
                  "mixed kernel attribute");
  if (st != BEM_OK) return st;
  sum_kern<<<(unsigned)plan.units, kThreads, plan.L.total, s>>>(p);
  sum_slices_kernel<<<(unsigned)((p.n * nu + 255) / 256), 256, 0, s>>>(
      p.Yp, plan.slices, 2 * p.nup, p.C, p.n, p.n_pad, nu, out);
  ctx->launches += 3;
  return cuda_check(ctx, cudaGetLastError(), "node-summed apply");
}

// A projection whose products Y_j = T(z_j) V are formed elsewhere (the low-rank far field)
// into the mixed path's FP32 partials, one column split: begin plans the scratch, prepares
// the basis planes and hands out slice 0; end adds the FP32 near-field corrections (slice
// 1) and forms B_j = w_j V^H Y_j (and Y_j on request) exactly as the mixed projection.
bem_status external_begin(bem_ctx* ctx, const double* V, int64_t ldv, int nu, ExtFrame& f,
                          cudaStream_t s) {
  MixedPlan* plan = new MixedPlan();
  bem_status st = mixed_plan(ctx, V, ldv, nu, 1, 0, *plan, s);
  if (st != BEM_OK) {
    delete plan;
    return st;
  }
  if ((st = set_mixed_smem(ctx, plan->L.total)) != BEM_OK) {   // the V^H Y kernels' smem
    delete plan;
    return st;
  }
  mixed_pre(ctx, *plan, s);
  f.impl = plan;
  f.Yp = plan->p.Yp;
  f.acc_cols = 2 * plan->p.nup;
  f.C = plan->p.C;
  f.n_pad = plan->p.n_pad;
  return cuda_check(ctx, cudaGetLastError(), "external projection set-up");
}

void external_release(ExtFrame& f) {
  delete static_cast<MixedPlan*>(f.impl);
  f.impl = nullptr;
}

bem_status external_end(bem_ctx* ctx, ExtFrame& f, int nu, double* Bhat, double* AV,
                        cudaStream_t s) {
  MixedPlan* plan = static_cast<MixedPlan*>(f.impl);
  bem_status st = BEM_OK;
  if (plan->slices > plan->p.S)
    st = near_apply32(ctx, plan->V32, nu, plan->p.nup, plan->p.C, plan->p.n_pad, plan->p.Yp,
                      plan->p.S, s);
  if (st == BEM_OK) mixed_post(ctx, *plan, Bhat, AV, s);
  delete plan;
  f.impl = nullptr;
  if (st != BEM_OK) return st;
  return cuda_check(ctx, cudaGetLastError(), "external projection kernels");
}

bem_status project_mixed(bem_ctx* ctx, const double* V, int64_t ldv, int nu, double* Bhat,
                         double* AV, cudaStream_t s) {
  MixedPlan plan;
  bem_status st = mixed_plan(ctx, V, ldv, nu, 0, 0, plan, s, true);
  if (st != BEM_OK) return st;
  mixed_pre(ctx, plan, s);
  if ((st = set_mixed_smem(ctx, plan.smem)) != BEM_OK) return st;
  const int np = poly_points(ctx, plan.pair ? 2 : plan.p.G);
  ctx->last_mixed_G = plan.p.G;
  ctx->last_mixed_pair = plan.pair ? 1 : 0;
  ctx->last_mixed_S = plan.p.S;
  ctx->last_mixed_ctas = plan.units;
  timing_begin(ctx, s);
  (plan.pair ? mixed_pair : mixed_kernel)(!op_single(ctx->op), np)
      <<<(unsigned)plan.units, plan.pair ? kPairThreads : kThreads, plan.smem, s>>>(plan.p);
  timing_end(ctx, s);
  ctx->launches++;
  st = cuda_check(ctx, cudaGetLastError(), "mixed apply kernel");
  if (st != BEM_OK) return st;
  if (plan.slices > plan.p.S) {
    st = near_apply32(ctx, plan.V32, nu, plan.p.nup, plan.p.C, plan.p.n_pad, plan.p.Yp, plan.p.S, s);
    if (st != BEM_OK) return st;
  }
  mixed_post(ctx, plan, Bhat, AV, s);
  return cuda_check(ctx, cudaGetLastError(), "mixed projection kernels");
}

}  // namespace bem

// ---------------------------------------------------------------------------------------
// Batched projection: several contexts (meshes, contours, bases) in one grouped launch of
// the fused kernel, the per-problem preparation and reductions around it, recorded once as
// a CUDA graph and replayed.

struct bem_batch {
  int device = 0;
  int nprob = 0;
  std::vector<bem_ctx*> ctx;
  std::vector<const double*> V;
  std::vector<int64_t> ldv;
  std::vector<int> nu;
  std::vector<double*> Bhat;
  std::vector<int64_t> mesh_ver, contour_ver;
  std::vector<double*> scratch;
  std::vector<int64_t> launches;      // launches per run, per context
  bem::MixedParams* d_plist = nullptr;
  int* d_ustart = nullptr;
  cudaStream_t cs = nullptr;          // private capture stream
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int* d_next = nullptr;              // work counter of the persistent kernel
  int sms = 0;
  int S = 0;                          // column splits (0: per-problem default)
  int G = 0;                          // nodes per unit cap (0: default)
  int64_t units = 0;                  // blocks of the grouped launch
  double tuned_ms = 0.0;              // time of one run at the chosen S (autotune), else 0
};

namespace bem {
namespace {

void batch_release_graph(bem_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// Plan every problem at split count S and node cap G, and record the graph.
bem_status batch_record(bem_batch* b, int S, int G) {
  bem_ctx* c0 = b->ctx[0];
  batch_release_graph(b);
  std::vector<MixedPlan> plan(b->nprob);
  uint32_t smem = 0, tcols = 32;
  for (int k = 0; k < b->nprob; ++k) {
    bem_status st = mixed_plan(b->ctx[k], b->V[k], b->ldv[k], b->nu[k], S, G, plan[k], b->cs);
    if (st != BEM_OK) return st;
    smem = std::max(smem, plan[k].L.total);
    while (tcols < (uint32_t)plan[k].p.G * 2u * plan[k].p.nup) tcols <<= 1;
  }
  // largest problems first; the unit offsets of the grouped launch
  std::vector<int> order(b->nprob);
  for (int k = 0; k < b->nprob; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return plan[x].units > plan[y].units; });
  std::vector<MixedParams> plist(b->nprob);
  std::vector<int> ustart(b->nprob);
  int64_t total = 0;
  for (int k = 0; k < b->nprob; ++k) {
    plist[k] = plan[order[k]].p;
    ustart[k] = (int)total;
    total += plan[order[k]].units;
  }
  if (total > 0x7fffffff) return fail(c0, BEM_EINVAL, "bem_batch_create: too many work units");
  b->units = total;
  b->S = S;
  b->G = G;
  bem_status st = cuda_check(c0, cudaMemcpyAsync(b->d_plist, plist.data(),
                                                 b->nprob * sizeof(MixedParams),
                                                 cudaMemcpyHostToDevice, b->cs), "batch copy");
  if (st == BEM_OK)
    st = cuda_check(c0, cudaMemcpyAsync(b->d_ustart, ustart.data(), b->nprob * sizeof(int),
                                        cudaMemcpyHostToDevice, b->cs), "batch copy");
  if (st == BEM_OK) st = cuda_check(c0, cudaStreamSynchronize(b->cs), "batch copy");
  if (st == BEM_OK) st = set_mixed_smem(c0, smem);
  if (st != BEM_OK) return st;
  std::vector<int64_t> before(b->nprob);
  for (int k = 0; k < b->nprob; ++k) before[k] = b->ctx[k]->launches;
  st = cuda_check(c0, cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal),
                  "batch capture");
  if (st != BEM_OK) return st;
  for (int k = 0; k < b->nprob; ++k) mixed_pre(b->ctx[k], plan[k], b->cs);
  cudaMemsetAsync(b->d_next, 0, sizeof(int), b->cs);
  const unsigned grid = (unsigned)std::min<int64_t>(total, std::max(1, b->sms));
  mixed_apply_grouped_kernel<<<grid, kThreads, smem, b->cs>>>(b->d_plist, b->d_ustart, b->nprob,
                                                            (int)total, b->d_next, tcols);
  c0->launches++;
  for (int k = 0; k < b->nprob; ++k) mixed_post(b->ctx[k], plan[k], b->Bhat[k], nullptr, b->cs);
  const cudaError_t le = cudaGetLastError();
  const cudaError_t ce = cudaStreamEndCapture(b->cs, &b->graph);
  for (int k = 0; k < b->nprob; ++k) {   // counted per replay instead
    b->launches[k] = b->ctx[k]->launches - before[k];
    b->ctx[k]->launches = before[k];
  }
  st = cuda_check(c0, le != cudaSuccess ? le : ce, "batch capture");
  if (st == BEM_OK) st = cuda_check(c0, cudaGraphInstantiate(&b->exec, b->graph, 0), "batch graph");
  if (st != BEM_OK) return st;
  for (int k = 0; k < b->nprob; ++k) {
    b->mesh_ver[k] = b->ctx[k]->mesh_version;
    b->contour_ver[k] = b->ctx[k]->contour_version;
    b->scratch[k] = b->ctx[k]->d_scratch;
  }
  return BEM_OK;
}

bem_status batch_launch(bem_batch* b, cudaStream_t s) {
  bem_ctx* c0 = b->ctx[0];
  for (int k = 0; k < b->nprob; ++k)
    if (b->ctx[k]->mesh_version != b->mesh_ver[k] ||
        b->ctx[k]->contour_version != b->contour_ver[k] ||
        b->ctx[k]->d_scratch != b->scratch[k] || !b->ctx[k]->con.self32_ready ||
        !op_single(b->ctx[k]->op))
      return fail(c0, BEM_ESTATE,
                  "bem_batch_run: a context's mesh, contour or workspace changed since the "
                  "batch was created");
  cudaSetDevice(b->device);
  bem_status st = cuda_check(c0, cudaGraphLaunch(b->exec, s), "bem_batch_run");
  if (st != BEM_OK) return st;
  for (int k = 0; k < b->nprob; ++k) b->ctx[k]->launches += b->launches[k];
  return BEM_OK;
}

// Time `reps` runs on the private stream (after one untimed run).
bem_status batch_time(bem_batch* b, int reps, double* ms) {
  bem_ctx* c0 = b->ctx[0];
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  bem_status st = batch_launch(b, b->cs);
  if (st == BEM_OK) st = cuda_check(c0, cudaEventRecord(e0, b->cs), "batch timing");
  for (int r = 0; r < reps && st == BEM_OK; ++r) st = batch_launch(b, b->cs);
  if (st == BEM_OK) st = cuda_check(c0, cudaEventRecord(e1, b->cs), "batch timing");
  if (st == BEM_OK) st = cuda_check(c0, cudaEventSynchronize(e1), "batch timing");
  float t = 0.f;
  if (st == BEM_OK) cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = t / reps;
  for (int k = 0; k < b->nprob && st == BEM_OK; ++k)
    st = take_status(b->ctx[k], b->cs, "bem_batch_create");
  return st;
}

}  // namespace
}  // namespace bem

extern "C" {

void bem_batch_destroy(bem_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->cs) cudaStreamSynchronize(b->cs);
  bem::batch_release_graph(b);
  cudaFree(b->d_plist);
  cudaFree(b->d_ustart);
  cudaFree(b->d_next);
  if (b->cs) cudaStreamDestroy(b->cs);
  delete b;
}

bem_status bem_batch_create(bem_ctx* const* ctxs, int nprob, const double* const* V_dev,
                            const int64_t* ldv, const int* nu, double* const* Bhat_dev,
                            int precision, int autotune, bem_batch** out, void* stream) {
  if (!out) return BEM_EINVAL;
  *out = nullptr;
  if (!ctxs || nprob < 1 || !ctxs[0]) return BEM_EINVAL;
  bem_ctx* c0 = ctxs[0];
  if (nprob > 4096 || !V_dev || !ldv || !nu || !Bhat_dev)
    return bem::fail(c0, BEM_EINVAL, "bem_batch_create: need 1..4096 problems and all arrays");
  if (precision != BEM_PREC_MIXED)
    return bem::fail(c0, BEM_EINVAL, "bem_batch_create: the grouped launch is the mixed path");
  for (int k = 0; k < nprob; ++k) {
    bem_ctx* c = ctxs[k];
    if (!c || c->device != c0->device)
      return bem::fail(c0, BEM_EINVAL, "bem_batch_create: contexts must exist and share a device");
    for (int q = 0; q < k; ++q)
      if (ctxs[q] == c) return bem::fail(c0, BEM_EINVAL, "bem_batch_create: a context appears twice");
    if (c->geo.n == 0 || c->con.N == 0)
      return bem::fail(c0, BEM_ESTATE, "bem_batch_create: every context needs a mesh and a contour");
    if (c->near_mode != 0)
      return bem::fail(c0, BEM_EINVAL, "bem_batch_create: near-field treatment is not batched");
    if (!bem::op_single(c->op))
      return bem::fail(c0, BEM_EINVAL, "bem_batch_create: the batched launch covers the single layer");
    if (!V_dev[k] || !Bhat_dev[k] || nu[k] < 1 || nu[k] > bem::kMaxNu || ldv[k] < c->geo.n ||
        nu[k] > c->geo.n)
      return bem::fail(c0, BEM_EINVAL, "bem_batch_create: bad V, Bhat, ldv or nu");
  }
  cudaSetDevice(c0->device);
  bem_batch* b = new bem_batch();
  b->device = c0->device;
  b->nprob = nprob;
  b->ctx.assign(ctxs, ctxs + nprob);
  b->V.assign(V_dev, V_dev + nprob);
  b->ldv.assign(ldv, ldv + nprob);
  b->nu.assign(nu, nu + nprob);
  b->Bhat.assign(Bhat_dev, Bhat_dev + nprob);
  b->mesh_ver.resize(nprob);
  b->contour_ver.resize(nprob);
  b->scratch.resize(nprob);
  b->launches.resize(nprob);
  bem_status st = bem::cuda_check(c0, cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking),
                                  "bem_batch_create");
  if (st == BEM_OK)
    st = bem::cuda_check(c0, cudaMalloc(&b->d_plist, nprob * sizeof(bem::MixedParams)),
                         "bem_batch_create");
  if (st == BEM_OK)
    st = bem::cuda_check(c0, cudaMalloc(&b->d_ustart, nprob * sizeof(int)), "bem_batch_create");
  if (st == BEM_OK)
    st = bem::cuda_check(c0, cudaMalloc(&b->d_next, sizeof(int)), "bem_batch_create");
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
  // the caller's stream may still be writing V: order the private stream after it
  if (st == BEM_OK) st = bem::cuda_check(c0, cudaStreamSynchronize((cudaStream_t)stream), "bem_batch_create");
  if (st == BEM_OK && autotune) {
    // autotuner: the work-unit shape of the grouped launch (column splits S, nodes per
    // unit G), by measurement of whole runs
    int best_S = 0, best_G = 0;
    double best = 1e300;
    for (int G : {0, 2}) {
      for (int S : {0, 1, 2, 3, 4}) {
        double ms = 0.0;
        st = bem::batch_record(b, S, G);
        if (st == BEM_OK) st = bem::batch_time(b, 3, &ms);
        if (st != BEM_OK) break;
        if (ms < best) {
          best = ms;
          best_S = S;
          best_G = G;
        }
      }
      if (st != BEM_OK) break;
    }
    if (st == BEM_OK) {
      b->tuned_ms = best;
      st = bem::batch_record(b, best_S, best_G);
    }
  } else if (st == BEM_OK) {
    st = bem::batch_record(b, 0, 0);
  }
  if (st == BEM_OK) st = bem::cuda_check(c0, cudaStreamSynchronize(b->cs), "bem_batch_create");
  if (st != BEM_OK) {
    bem_batch_destroy(b);
    return st;
  }
  *out = b;
  return BEM_OK;
}

bem_status bem_batch_run(bem_batch* b, void* stream) {
  if (!b) return BEM_EINVAL;
  return bem::batch_launch(b, (cudaStream_t)stream);
}

bem_status bem_batch_info(const bem_batch* b, int* splits, int* nodes_per_unit, int64_t* units,
                          double* tuned_ms) {
  if (!b) return BEM_EINVAL;
  if (splits) *splits = b->S;
  if (nodes_per_unit) *nodes_per_unit = b->G;
  if (units) *units = b->units;
  if (tuned_ms) *tuned_ms = b->tuned_ms;
  return BEM_OK;
}

bem_status bem_project_batched(bem_ctx* const* ctxs, int nprob, const double* const* V_dev,
                               const int64_t* ldv, const int* nu, double* const* Bhat_dev,
                               int precision, void* stream) {
  bem_batch* b = nullptr;
  bem_status st = bem_batch_create(ctxs, nprob, V_dev, ldv, nu, Bhat_dev, precision, 0, &b, stream);
  if (st != BEM_OK) return st;
  st = bem_batch_run(b, stream);
  if (st == BEM_OK)
    st = bem::cuda_check(ctxs[0], cudaStreamSynchronize((cudaStream_t)stream), "bem_project_batched");
  for (int k = 0; k < nprob && st == BEM_OK; ++k) st = bem_check(ctxs[k], stream);
  bem_batch_destroy(b);
  return st;
}

}  // extern "C"
