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
// mixed_vhy_part_kernel / mixed_vhy_reduce_kernel then form
// Bhat_j = w_j V^H (sum over column splits of Y_j) with a fixed summation order.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

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
constexpr uint32_t kWaitLimit = 1u << 24;    // polls (with 64 ns sleeps) before giving up
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kInv2Pi = 0.15915494309189535f;
constexpr float kTwoPiHi = 6.28318548202514648f;      // float nearest 2 pi
constexpr float kTwoPiLo = -1.7484555314695172e-7f;   // 2 pi - kTwoPiHi

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
  const __nv_bfloat16* Bp;   // prepared basis planes, tile-native
  float* Yp;          // FP32 partial products [S][N][2 nup][n_pad]
  int* status;
};

struct SmemLayout {
  uint32_t a_off, b_off, graw_off, row_off, col_off, self_off, bar_off, misc_off, total;
  uint32_t a_stage_bytes, b_stage_bytes;
};
constexpr uint32_t kGeoBlockBytes = kBK * 64 * 4;   // packed geometry of one K-block

__host__ __device__ inline SmemLayout smem_layout(int G, int nup) {
  SmemLayout L;
  L.a_stage_bytes = (uint32_t)G * 4 * kPlaneBytes;
  L.b_stage_bytes = (uint32_t)256 * nup;     // 4 planes x 2 nup rows x 16 k x 2 B
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

__device__ __forceinline__ uint32_t pack_bf16(float lo_elem, float hi_elem) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo_elem, hi_elem);   // .x -> low 16 bits
  return *reinterpret_cast<uint32_t*>(&h);
}

// bounded wait that also watches the block's abort flag
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity,
                                              volatile int* abort_flag, int* status) {
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (it > 64) __nanosleep(64);
  }
  atomicOr(status, kStatusTimeout);
  *abort_flag = 1;
  return false;
}

__global__ void __launch_bounds__(kThreads, 1) mixed_apply_kernel(MixedParams p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const SmemLayout L = smem_layout(p.G, p.nup);
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

  // unit -> (row tile, node group, column split)
  const int u = blockIdx.x;
  const int split = u % p.S;
  const int t = u / p.S;
  const int gg = t % p.nG;
  const int rt = t / p.nG;
  const int64_t row0 = (int64_t)rt * kBM;
  const int kb0 = (int)((int64_t)p.nK * split / p.S);
  const int kb1 = (int)((int64_t)p.nK * (split + 1) / p.S);
  const int nkb = kb1 - kb0;
  const int j0 = gg * p.G;
  const int Gv = min(p.G, p.N - j0);
  const uint32_t acc_cols = 2u * p.nup;                 // TMEM columns per node
  uint32_t tmem_cols = 32;
  while (tmem_cols < (uint32_t)p.G * acc_cols) tmem_cols <<= 1;

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
  if (warp == 1) {
    tmem_alloc(tmem_slot, tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

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
    int issued = 0;
    for (int it = 0; it < nkb; ++it) {
      const int s = it % kStages;
      const uint32_t par = (it / kStages) & 1;
      const int kb = kb0 + it;
      int ok = 1;
      if (lane == 0) ok = wait_or_abort(&empty[s], par ^ 1, abort_flag, p.status);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      if (lane == 0) {
        mbar_arrive_expect_tx(&bfull[s], L.b_stage_bytes);
        bulk_g2s(sB + s * L.b_stage_bytes,
                 reinterpret_cast<const unsigned char*>(p.Bp) +
                     (size_t)kb * L.b_stage_bytes,
                 L.b_stage_bytes, &bfull[s]);
        mbar_arrive_expect_tx(&gready[s], kGeoBlockBytes);
        bulk_g2s(smem + L.graw_off + s * kGeoBlockBytes, p.pack32 + (size_t)kb * kBK * 64,
                 kGeoBlockBytes, &gready[s]);
      }
      ++issued;
      // tile-relative FP32 coordinates from the hi/lo pairs: (y_hi - o_hi) + (y_lo - o_lo)
      if (!wait_or_abort(&gready[s], par, abort_flag, p.status)) break;
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
        if (l < p.n && g < Gv && l >= row0 && l < row0 + kBM)
          v = p.self32[(int64_t)(j0 + g) * p.n + l];
        sSelf[x] = v;
      }
      mbar_arrive(&gfull[s]);   // release: the staged values are visible to the waiters
    }
    if (lane == 0 && *abort_flag) {
      // let copies in flight land before the block exits (bounded)
      for (int it = max(0, issued - kStages); it < issued; ++it) {
        mbar_wait(&bfull[it % kStages], (it / kStages) & 1, kWaitLimit);
        mbar_wait(&gready[it % kStages], (it / kStages) & 1, kWaitLimit);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kBM, 2 * p.C);
      // (A plane, B plane) pairs of the split-precision complex product
      const int pa[6] = {0, 0, 1, 2, 2, 3};   // Ar_hi, Ar_hi, Ar_lo, Ai_hi, Ai_hi, Ai_lo
      const int pb[6] = {0, 1, 0, 2, 3, 2};   // [Vr|Vi], [Vr_lo|Vi_lo], [-Vi|Vr], [-Vi_lo|Vr_lo]
      const uint32_t bplane = 2u * p.C * kBK * 2;   // bytes of one basis plane per chunk
      for (int it = 0; it < nkb; ++it) {
        const int s = it % kStages;
        const uint32_t par = (it / kStages) & 1;
        if (!wait_or_abort(&afull[s], par, abort_flag, p.status)) break;
        if (!wait_or_abort(&bfull[s], par, abort_flag, p.status)) break;
        tc_fence_after();
        const uint32_t a_base = smem_u32(sA + s * L.a_stage_bytes);
        const uint32_t b_base = smem_u32(sB + s * L.b_stage_bytes);
        for (int g = 0; g < Gv; ++g) {
          for (int c = 0; c < p.nchunks; ++c) {
            const uint32_t d = tmem_base + g * acc_cols + c * 2 * p.C;
#pragma unroll
            for (int q = 0; q < 6; ++q) {
              const uint64_t ad = smem_desc(a_base + (g * 4 + pa[q]) * kPlaneBytes, 128, 256);
              const uint64_t bd = smem_desc(b_base + (c * 4 + pb[q]) * bplane, 128, 256);
              mma_bf16(d, ad, bd, idesc, (it > 0 || q > 0) ? 1u : 0u);
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
#pragma unroll
    for (int g = 0; g < kMaxG; ++g) {
      const int j = j0 + (g < Gv ? g : 0);
      kr[g] = (float)p.z[2 * j];
      kmi[g] = (float)(-p.z[2 * j + 1]) * kLog2e;
    }
    // this thread's entries: row 8 e + r8, columns 8 kg + 2 kp + {0, 1} for kg = 0, 1
    const int r8 = lane / 4, kp = lane % 4;
    const int row = 8 * e + r8;
    const int64_t i = row0 + row;

    for (int it = 0; it < nkb; ++it) {
      const int s = it % kStages;
      const uint32_t par = (it / kStages) & 1;
      const int kb = kb0 + it;
      const bool ready = wait_or_abort(&gfull[s], par, abort_flag, p.status);
      const float4* sCol = sColAll + s * (kBK * 7);
      const float2* sSelf = sSelfAll + s * (kBK * kMaxG);
      unsigned char* a_stage = sA + s * L.a_stage_bytes;
      const float4 xr = sRow[row];
#pragma unroll 1
      for (int kg = 0; kg < (ready ? 2 : 0); ++kg) {
        const int k0 = 8 * kg + 2 * kp;
        const int64_t l0 = (int64_t)kb * kBK + k0;
        float rr[2][7], am[2][7];
#pragma unroll
        for (int d = 0; d < 2; ++d) {
          const float4* col = sCol + (k0 + d) * 7;
#pragma unroll
          for (int q = 0; q < 7; ++q) {
            const float4 y = col[q];
            const float dx = xr.x - y.x, dy = xr.y - y.y, dz = xr.z - y.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float rs = rsqrtf_mufu(r2);
            rr[d][q] = r2 * rs;
            am[d][q] = y.w * rs;
          }
        }
        const uint32_t off = e * 256 + kg * 128 + r8 * 16 + kp * 4;
#pragma unroll
        for (int g = 0; g < kMaxG; ++g) {
          if (g >= Gv) break;
          float re[2], im[2];
#pragma unroll
          for (int d = 0; d < 2; ++d) {
            float sr = 0.f, si = 0.f;
#pragma unroll
            for (int q = 0; q < 7; ++q) {
              const float a = am[d][q] * ex2f(kmi[g] * rr[d][q]);
              const float ph = kr[g] * rr[d][q];
              const float nrot = fmaf(ph, kInv2Pi, 12582912.0f) - 12582912.0f;
              const float red = fmaf(-nrot, kTwoPiLo, fmaf(-nrot, kTwoPiHi, ph));
              sr = fmaf(a, cosf_mufu(red), sr);
              si = fmaf(a, sinf_mufu(red), si);
            }
            if (i == l0 + d) {   // diagonal: the self term
              const float2 sv = sSelf[(k0 + d) * kMaxG + g];
              sr = sv.x;
              si = sv.y;
            }
            if (i >= p.n || l0 + d >= p.n) {   // padding rows / columns of the tile
              sr = 0.f;
              si = 0.f;
            }
            re[d] = sr;
            im[d] = si;
          }
          const uint32_t hr = pack_bf16(re[0], re[1]);
          const uint32_t hi = pack_bf16(im[0], im[1]);
          const uint32_t lr = pack_bf16(re[0] - __uint_as_float(hr << 16),
                                        re[1] - __uint_as_float(hr & 0xFFFF0000u));
          const uint32_t li = pack_bf16(im[0] - __uint_as_float(hi << 16),
                                        im[1] - __uint_as_float(hi & 0xFFFF0000u));
          unsigned char* ag = a_stage + g * 4 * kPlaneBytes + off;
          *reinterpret_cast<uint32_t*>(ag + 0 * kPlaneBytes) = hr;
          *reinterpret_cast<uint32_t*>(ag + 1 * kPlaneBytes) = lr;
          *reinterpret_cast<uint32_t*>(ag + 2 * kPlaneBytes) = hi;
          *reinterpret_cast<uint32_t*>(ag + 3 * kPlaneBytes) = li;
        }
      }
      fence_proxy_async_smem();
      mbar_arrive(&afull[s]);
      if (!ready) break;
    }

    // ---------------- epilogue: TMEM -> FP32 partial Y ----------------
    const bool ok = !*abort_flag && wait_or_abort(accfull, 0, abort_flag, p.status);
    if (__all_sync(0xffffffffu, ok)) {   // tcgen05.ld is warp-collective
      tc_fence_after();
      const int quarter = warp % 4;              // TMEM lanes this warp may read
      const int part = (warp - 2) / 4;           // four warps per quarter split the columns
      const int erow = quarter * 32 + lane;
      const int64_t ei = row0 + erow;
      const uint32_t cols_total = (uint32_t)Gv * acc_cols;
      for (uint32_t c0 = part * 16; c0 < cols_total; c0 += 64) {
        float v[16];
        tmem_ld16(tmem_base + ((uint32_t)(quarter * 32) << 16) + c0, v);
        const int g = c0 / acc_cols;
        const int col = c0 % acc_cols;
        float* dst = p.Yp + (((size_t)split * p.N + (j0 + g)) * acc_cols + col) * p.n_pad + ei;
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
    tmem_dealloc(tmem_base, tmem_cols);
  }
}

// Basis planes in the tile-native layout the kernel copies per K-block: for K-block kb,
// chunk c, plane pl, the 2C x 16 block in core matrices (row group ng, k group kg) of
// 8 rows x 8 bf16, row stride 16 B, at ng * 256 + kg * 128 bytes.
__global__ void prep_basis_planes_kernel(const double* __restrict__ V, int64_t ldv, int64_t n,
                                         int nu, int nup, int C, int nK,
                                         __nv_bfloat16* __restrict__ Bp) {
  const int64_t total = (int64_t)nK * 4 * 2 * nup * kBK;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= total) return;
  // decode in the order of the layout
  int64_t x = t;
  const int k8 = (int)(x % 8); x /= 8;
  const int r8 = (int)(x % 8); x /= 8;
  const int kg = (int)(x % 2); x /= 2;
  const int ngroups = 2 * C / 8;
  const int ng = (int)(x % ngroups); x /= ngroups;
  const int pl = (int)(x % 4); x /= 4;
  const int nchunks = nup / C;
  const int c = (int)(x % nchunks); x /= nchunks;
  const int kb = (int)x;
  const int rowN = ng * 8 + r8;                 // 0 .. 2C
  const int halfim = rowN >= C;                 // 0: feeds Yr, 1: feeds Yi
  const int col = c * C + (rowN % C);
  const int64_t l = (int64_t)kb * kBK + kg * 8 + k8;
  double vr = 0.0, vi = 0.0;
  if (l < n && col < nu) {
    const double2 v = reinterpret_cast<const double2*>(V)[(int64_t)col * ldv + l];
    vr = v.x;
    vi = v.y;
  }
  const __nv_bfloat16 vr_hi = __double2bfloat16(vr);
  const __nv_bfloat16 vi_hi = __double2bfloat16(vi);
  const __nv_bfloat16 vr_lo = __double2bfloat16(vr - (double)__bfloat162float(vr_hi));
  const __nv_bfloat16 vi_lo = __double2bfloat16(vi - (double)__bfloat162float(vi_hi));
  __nv_bfloat16 out;
  switch (pl) {
    case 0: out = halfim ? vi_hi : vr_hi; break;                    // [Vr | Vi]
    case 1: out = halfim ? vi_lo : vr_lo; break;                    // [Vr_lo | Vi_lo]
    case 2: out = halfim ? vr_hi : __hneg(vi_hi); break;            // [-Vi | Vr]
    default: out = halfim ? vr_lo : __hneg(vi_lo); break;           // [-Vi_lo | Vr_lo]
  }
  Bp[t] = out;
}

// Partial products P_r,j = V^H Y_j over the row range of part r, Y_j = sum over column
// splits of the FP32 partials: FP32 products summed over 32-row chunks, chunk sums added
// in FP64 (the inputs carry ~1e-5 relative error, so FP32 products lose nothing; the FP64
// pipe of this GPU is ~70x slower than its FP32 pipe).
constexpr int kT = 64;    // output tile (64 x 64 of the nu x nu matrix)
constexpr int kTR = 32;   // rows per chunk
__global__ void __launch_bounds__(256)
mixed_vhy_part_kernel(const double* __restrict__ V, int64_t ldv, int nu, int64_t n, int n_pad,
                      int N, int S, int acc_cols, int C, const float* __restrict__ Yp,
                      int64_t rows_per_part, double* __restrict__ part) {
  __shared__ float2 sX[kTR][kT + 1];   // +1: the row-major fill below is then 2-way at most
  __shared__ float2 sY[kTR][kT + 1];
  const int tiles_a = (nu + kT - 1) / kT;
  const int ta = blockIdx.x % tiles_a, tb = blockIdx.x / tiles_a;
  const int j = blockIdx.y;
  const int64_t r_begin = (int64_t)blockIdx.z * rows_per_part;
  const int64_t r_end = min(n, r_begin + rows_per_part);
  const int tid = threadIdx.x;
  const int oa = tid % 16, ob = tid / 16;   // outputs (oa + 16 i, ob + 16 m)
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int m = 0; m < 4; ++m) acc[i][m] = make_double2(0.0, 0.0);
  const double2* Vc = reinterpret_cast<const double2*>(V);
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kTR) {
    __syncthreads();
    for (int x = tid; x < kTR * kT; x += 256) {
      const int rr = x % kTR, cc = x / kTR;
      const int64_t r = r0 + rr;
      const int a = ta * kT + cc;
      float2 v = make_float2(0.f, 0.f);
      if (r < r_end && a < nu) {
        const double2 vd = Vc[(int64_t)a * ldv + r];
        v = make_float2((float)vd.x, (float)vd.y);
      }
      sX[rr][cc] = v;
    }
    // Y rows four at a time (rows_per_part and the chunk start are multiples of 4; rows
    // past n are the zero padding rows of the last tile, rows past r_end are masked)
    for (int x = tid; x < (kTR / 4) * kT; x += 256) {
      const int q4 = x % (kTR / 4), cc = x / (kTR / 4);
      const int64_t r = r0 + 4 * q4;
      const int b = tb * kT + cc;
      float4 yr = make_float4(0.f, 0.f, 0.f, 0.f), yi = yr;
      if (r < r_end && b < nu) {
        const int colr = (b / C) * 2 * C + (b % C);
        for (int s = 0; s < S; ++s) {
          const float* base = Yp + ((size_t)s * N + j) * acc_cols * (size_t)n_pad;
          const float4 a4 = *reinterpret_cast<const float4*>(base + (size_t)colr * n_pad + r);
          const float4 b4 = *reinterpret_cast<const float4*>(base + (size_t)(colr + C) * n_pad + r);
          yr.x += a4.x; yr.y += a4.y; yr.z += a4.z; yr.w += a4.w;
          yi.x += b4.x; yi.y += b4.y; yi.z += b4.z; yi.w += b4.w;
        }
      }
      sY[4 * q4 + 0][cc] = (r + 0 < r_end) ? make_float2(yr.x, yi.x) : make_float2(0.f, 0.f);
      sY[4 * q4 + 1][cc] = (r + 1 < r_end) ? make_float2(yr.y, yi.y) : make_float2(0.f, 0.f);
      sY[4 * q4 + 2][cc] = (r + 2 < r_end) ? make_float2(yr.z, yi.z) : make_float2(0.f, 0.f);
      sY[4 * q4 + 3][cc] = (r + 3 < r_end) ? make_float2(yr.w, yi.w) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2 c[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m) c[i][m] = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int rr = 0; rr < kTR; ++rr) {
      float2 x[4], y[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) x[i] = sX[rr][oa + 16 * i];
#pragma unroll
      for (int m = 0; m < 4; ++m) y[m] = sY[rr][ob + 16 * m];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int m = 0; m < 4; ++m) {   // conj(x) * y
          c[i][m].x = fmaf(x[i].x, y[m].x, fmaf(x[i].y, y[m].y, c[i][m].x));
          c[i][m].y = fmaf(x[i].x, y[m].y, fmaf(-x[i].y, y[m].x, c[i][m].y));
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        acc[i][m].x += c[i][m].x;
        acc[i][m].y += c[i][m].y;
      }
  }
  double2* P = reinterpret_cast<double2*>(part) + ((int64_t)blockIdx.z * N + j) * nu * nu;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = ta * kT + oa + 16 * i;
    if (a >= nu) continue;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int b = tb * kT + ob + 16 * m;
      if (b < nu) P[(int64_t)b * nu + a] = acc[i][m];
    }
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

}  // namespace

bem_status project_mixed(bem_ctx* ctx, const double* V, int64_t ldv, int nu, double* Bhat,
                         double* AV, cudaStream_t s) {
  const int64_t n = ctx->geo.n;
  const int N = ctx->con.N;
  MixedParams p{};
  p.n = n;
  p.N = N;
  p.nu = nu;
  p.nup = (nu + 7) / 8 * 8;
  p.C = p.nup <= 128 ? p.nup : 128;
  if (p.nup % p.C != 0) p.nup = (p.nup + p.C - 1) / p.C * p.C;
  p.nchunks = p.nup / p.C;
  const int acc_cols = 2 * p.nup;
  p.G = std::max(1, std::min(std::min(N, kMaxG), 512 / acc_cols));
  p.nG = (N + p.G - 1) / p.G;
  p.nK = (int)((n + kBK - 1) / kBK);
  p.n_pad = (int)((n + kBM - 1) / kBM * kBM);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  const int64_t rtiles = p.n_pad / kBM;
  p.S = choose_splits(rtiles * p.nG, p.nK, std::max(1, sms));

  // scratch: basis planes, then the FP32 partials
  const size_t bp_bytes = (size_t)p.nK * 256 * p.nup;
  const size_t bp_off = 0;
  const size_t yp_off = (bp_bytes + 255) / 256 * 256;
  const size_t yp_bytes = (size_t)p.S * N * acc_cols * p.n_pad * sizeof(float);
  // V^H Y partials: enough row ranges to fill the device, at least 128 rows each
  const int vtiles = ((nu + kT - 1) / kT) * ((nu + kT - 1) / kT);
  int64_t vparts = std::max<int64_t>(1, std::min<int64_t>((n + 127) / 128,
                                                          (4 * (int64_t)sms + vtiles * N - 1) /
                                                              ((int64_t)vtiles * N)));
  const int64_t rows_per_vpart = ((n + vparts - 1) / vparts + kTR - 1) / kTR * kTR;
  vparts = (n + rows_per_vpart - 1) / rows_per_vpart;
  const size_t vp_off = (yp_off + yp_bytes + 255) / 256 * 256;
  const size_t vp_bytes = (size_t)vparts * N * nu * nu * 2 * sizeof(double);
  bem_status st = ensure_self32(ctx, s);
  if (st != BEM_OK) return st;
  st = ensure_scratch(ctx, vp_off + vp_bytes);
  if (st != BEM_OK) return st;
  unsigned char* scr = reinterpret_cast<unsigned char*>(ctx->d_scratch);
  p.Bp = reinterpret_cast<const __nv_bfloat16*>(scr + bp_off);
  p.Yp = reinterpret_cast<float*>(scr + yp_off);
  p.cx = ctx->geo.cx;
  p.qp = ctx->geo.qp;
  p.qw = ctx->geo.qw;
  p.self32 = reinterpret_cast<const float2*>(ctx->con.self32);
  p.pack32 = ctx->geo.pack32;
  p.z = ctx->con.z;
  p.status = ctx->d_status;

  const int64_t prep_total = (int64_t)p.nK * 4 * 2 * p.nup * kBK;
  prep_basis_planes_kernel<<<(unsigned)((prep_total + 255) / 256), 256, 0, s>>>(
      V, ldv, n, nu, p.nup, p.C, p.nK,
      reinterpret_cast<__nv_bfloat16*>(scr + bp_off));
  ctx->launches++;

  const SmemLayout L = smem_layout(p.G, p.nup);
  st = cuda_check(ctx, cudaFuncSetAttribute(mixed_apply_kernel,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)L.total),
                  "mixed kernel attribute");
  if (st != BEM_OK) return st;
  const int64_t units = rtiles * p.nG * p.S;
  timing_begin(ctx, s);
  mixed_apply_kernel<<<(unsigned)units, kThreads, L.total, s>>>(p);
  timing_end(ctx, s);
  ctx->launches++;
  st = cuda_check(ctx, cudaGetLastError(), "mixed apply kernel");
  if (st != BEM_OK) return st;

  double* vpart = reinterpret_cast<double*>(scr + vp_off);
  mixed_vhy_part_kernel<<<dim3((unsigned)vtiles, (unsigned)N, (unsigned)vparts), 256, 0, s>>>(
      V, ldv, nu, n, p.n_pad, N, p.S, acc_cols, p.C, p.Yp, rows_per_vpart, vpart);
  const int64_t outs = (int64_t)N * nu * nu;
  mixed_vhy_reduce_kernel<<<(unsigned)((outs + 255) / 256), 256, 0, s>>>(vpart, (int)vparts, N, nu,
                                                                         ctx->con.w, Bhat);
  ctx->launches += 2;
  if (AV) {
    const int64_t tot = (int64_t)N * nu * n;
    mixed_av_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, p.n_pad, nu, N, p.S,
                                                                  acc_cols, p.C, p.Yp, AV);
    ctx->launches++;
  }
  return cuda_check(ctx, cudaGetLastError(), "mixed projection kernels");
}

}  // namespace bem
