// Low-rank far field of T(z_j) (the H-matrix route of the paper's largest problems,
// Section 4, Example 3: the samples are stored as H-matrices compressed by adaptive cross
// approximation), applied in the projection of Eq. RR_approx.
//
// Host: a cluster tree of the panels (split at the middle of their order along the longest
// axis of the centroids' box, ties by index, down to `leaf` panels; a cluster's geometry is
// the box of its panels' vertices) and the block partition from (root, root): a pair is far
// when max(diam tau, diam sigma) <= eta dist(tau, sigma) and both hold more than two leaves
// of panels, a pair of leaves that is not far is dense, any other pair splits into its
// children's pairs.
// Device, node by node:
//   hm_aca_kernel        one CTA per far block: adaptive cross approximation with partial
//                        pivoting on FP32 entries (block ~ U W^T, ranks up to rmax, stop at
//                        ||u_k|| ||w_k|| <= eps ||S_k||_F with the exact norm update);
//   hm_wtv_kernel        T_b = W_b^T V_sigma (rank x nu) per far block, as panel products in
//                        shared memory;
//   hm_leaf_kernel       one CTA per leaf row range: the leaf's dense column ranges evaluated
//                        32 panels at a time from geometry staged in shared memory and
//                        multiplied with every basis column, then the rank-1 terms of every
//                        far block above the leaf, 32 at a time, in a fixed order (no
//                        atomics), into the mixed path's FP32 partials of Y_j.
// Geometry, basis and T_b are kept in cluster order, so that a cluster is a contiguous range.
// The mixed path then adds the FP32 near-field corrections (if enabled) and forms
// B_j = w_j V^H Y_j (tensor-core contraction for nu <= 128).
#include <math.h>

#include <algorithm>
#include <numeric>
#include <type_traits>
#include <vector>

#include "internal.h"

namespace bem {

struct HMatrix {
  int leaf = 32;
  double eta = 1.0, eps = 1e-6;
  int rmax = 48;
  int64_t mesh_version = -1;
  // structure (host)
  std::vector<int32_t> perm;   // cluster order -> panel
  struct Cl {
    int32_t b, e, c0, c1;      // panel range in `perm`, children (-1: leaf)
    double lo[3], hi[3];
  };
  std::vector<Cl> cl;
  std::vector<int4> far;       // far blocks: tau range, sigma range
  std::vector<int64_t> uw_off; // per far block: offset of U (m x rmax), then W (n x rmax)
  int64_t uw_total = 0;        // complex elements per node
  int64_t used_total = 0;      // row flags per node (bytes)
  std::vector<int64_t> used_off;
  std::vector<int4> leaves;    // leaf row range, then [near_begin, near_end) in `near`
  std::vector<int32_t> leaf_far_ptr, leaf_far;   // CSR: far blocks above each leaf
  std::vector<int2> near;      // dense column ranges of a leaf (contiguous in cluster order)
  std::vector<int32_t> near_ptr;
  int64_t dense_blocks = 0;    // leaf-leaf dense blocks of the partition
  int nbig = 0;                // far blocks (the first ones) of at least kAcaBig rows + columns
  // device copies
  int32_t* d_perm = nullptr;
  int4* d_far = nullptr;
  int64_t* d_uw_off = nullptr;
  int64_t* d_used_off = nullptr;
  int4* d_leaves = nullptr;
  int32_t* d_leaf_far_ptr = nullptr;
  int32_t* d_leaf_far = nullptr;
  int2* d_near = nullptr;
  int32_t* d_near_ptr = nullptr;
  float4* d_gq = nullptr;      // geometry in cluster order: 7 n points, n normals, n centroids
  float4* d_gn = nullptr;
  float4* d_gc = nullptr;
  // per-node work (grown on demand)
  float2* d_uw = nullptr;
  size_t uw_bytes = 0;
  uint8_t* d_used = nullptr;
  size_t used_bytes = 0;
  int32_t* d_rank = nullptr;
  int64_t* d_toff = nullptr;
  size_t rank_cap = 0;
  float2* d_t = nullptr;
  size_t t_bytes = 0;
  float2* d_vp = nullptr;      // V in cluster order, row-major (CW per panel, zero-padded), FP32
  size_t vp_bytes = 0;
  double* d_y = nullptr;       // Y_j, FP64, column-major per node
  size_t y_bytes = 0;
  // statistics of the last projection
  double mean_rank = 0.0;
  int max_rank = 0;
  double far_fraction = 0.0;
  // algorithmic work per node (averaged over the nodes of the last projection): dense
  // entries evaluated and multiplied, rank-1 terms times rows (U T) and times columns (W^T V)
  double dense_entries = 0.0, far_row_terms = 0.0, far_col_terms = 0.0;
};

namespace {

void free_dev(HMatrix& h) {
  cudaFree(h.d_perm); cudaFree(h.d_far); cudaFree(h.d_uw_off); cudaFree(h.d_used_off);
  cudaFree(h.d_leaves); cudaFree(h.d_leaf_far_ptr); cudaFree(h.d_leaf_far); cudaFree(h.d_near);
  cudaFree(h.d_near_ptr); cudaFree(h.d_gq);
  h.d_gq = h.d_gn = h.d_gc = nullptr;
  h.d_perm = nullptr; h.d_far = nullptr; h.d_uw_off = nullptr; h.d_used_off = nullptr;
  h.d_leaves = nullptr; h.d_leaf_far_ptr = nullptr; h.d_leaf_far = nullptr; h.d_near = nullptr;
  h.d_near_ptr = nullptr;
}

void free_work(HMatrix& h) {
  cudaFree(h.d_uw); cudaFree(h.d_used); cudaFree(h.d_rank); cudaFree(h.d_toff); cudaFree(h.d_t);
  cudaFree(h.d_vp); cudaFree(h.d_y);
  h.d_uw = nullptr; h.d_used = nullptr; h.d_rank = nullptr; h.d_toff = nullptr; h.d_t = nullptr;
  h.d_vp = nullptr; h.d_y = nullptr;
  h.uw_bytes = h.used_bytes = h.rank_cap = h.t_bytes = h.vp_bytes = h.y_bytes = 0;
}

double box_diam(const HMatrix::Cl& c) {
  double s = 0.0;
  for (int d = 0; d < 3; ++d) s += (c.hi[d] - c.lo[d]) * (c.hi[d] - c.lo[d]);
  return sqrt(s);
}

double box_dist(const HMatrix::Cl& a, const HMatrix::Cl& b) {
  double s = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double g = std::max(0.0, std::max(a.lo[d] - b.hi[d], b.lo[d] - a.hi[d]));
    s += g * g;
  }
  return sqrt(s);
}

// Cluster tree over perm[b, e); returns the cluster's number.
int build_cluster(HMatrix& h, const std::vector<double>& cen, const std::vector<double>& xyz,
                  const std::vector<int32_t>& tri, int32_t b, int32_t e) {
  const int me = (int)h.cl.size();
  HMatrix::Cl c;
  c.b = b;
  c.e = e;
  c.c0 = c.c1 = -1;
  for (int d = 0; d < 3; ++d) {
    c.lo[d] = 1e300;
    c.hi[d] = -1e300;
  }
  double clo[3] = {1e300, 1e300, 1e300}, chi[3] = {-1e300, -1e300, -1e300};
  for (int32_t t = b; t < e; ++t) {
    const int32_t l = h.perm[t];
    for (int v = 0; v < 3; ++v)
      for (int d = 0; d < 3; ++d) {
        const double x = xyz[3 * (int64_t)tri[3 * (int64_t)l + v] + d];
        c.lo[d] = std::min(c.lo[d], x);
        c.hi[d] = std::max(c.hi[d], x);
      }
    for (int d = 0; d < 3; ++d) {
      clo[d] = std::min(clo[d], cen[3 * (int64_t)l + d]);
      chi[d] = std::max(chi[d], cen[3 * (int64_t)l + d]);
    }
  }
  h.cl.push_back(c);
  if (e - b > h.leaf) {
    int axis = 0;
    for (int d = 1; d < 3; ++d)
      if (chi[d] - clo[d] > chi[axis] - clo[axis]) axis = d;
    std::sort(h.perm.begin() + b, h.perm.begin() + e, [&](int32_t p, int32_t q) {
      const double xp = cen[3 * (int64_t)p + axis], xq = cen[3 * (int64_t)q + axis];
      return xp < xq || (xp == xq && p < q);
    });
    const int32_t mid = b + (e - b) / 2;
    const int c0 = build_cluster(h, cen, xyz, tri, b, mid);
    const int c1 = build_cluster(h, cen, xyz, tri, mid, e);
    h.cl[me].c0 = c0;
    h.cl[me].c1 = c1;
  }
  return me;
}

void build_blocks(HMatrix& h, int t, int s, std::vector<int2>& far_cl,
                  std::vector<int2>& near_cl) {
  const HMatrix::Cl& A = h.cl[t];
  const HMatrix::Cl& B = h.cl[s];
  // far: admissible and larger than two leaves both ways (smaller admissible blocks are
  // cheaper evaluated densely, leaf by leaf)
  if (std::max(box_diam(A), box_diam(B)) <= h.eta * box_dist(A, B) &&
      std::min(A.e - A.b, B.e - B.b) > 2 * h.leaf) {
    far_cl.push_back(make_int2(t, s));
    return;
  }
  const bool la = A.c0 < 0, lb = B.c0 < 0;
  if (la && lb) {
    near_cl.push_back(make_int2(t, s));
    return;
  }
  const int ta[2] = {la ? t : A.c0, la ? -1 : A.c1};
  const int sb[2] = {lb ? s : B.c0, lb ? -1 : B.c1};
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      if (ta[i] >= 0 && sb[j] >= 0) build_blocks(h, ta[i], sb[j], far_cl, near_cl);
}

}  // namespace

namespace {

// Geometry in cluster order (structure of arrays, coalesced for consecutive panels of a
// cluster): the 7 quadrature points (x, y, z, W/4pi) of cluster panel t at q * n + t, the
// unit normal at t, the centroid (x, y, z, panel index as int bits) at t. FP32 values of the
// mixed path's geometry, permuted once per block structure.
struct HmGeom {
  const float4* q;
  const float4* nrm;
  const float4* cen;
  int64_t n;
};

__global__ void hm_geom_kernel(Geometry g, const int32_t* __restrict__ perm, float4* __restrict__ q,
                               float4* __restrict__ nrm, float4* __restrict__ cen) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = g.n;
  if (t >= n) return;
  const int64_t l = perm[t];
#pragma unroll
  for (int k = 0; k < 7; ++k)
    q[k * n + t] = make_float4(g.qp32[k * n + l], g.qp32[(7 + k) * n + l], g.qp32[(14 + k) * n + l],
                               g.qw32[k * n + l]);
  const float* pk = g.pack32 + l * 64;
  nrm[t] = make_float4(pk[56], pk[57], pk[58], 0.f);
  cen[t] = make_float4(g.cx32[l], g.cx32[n + l], g.cx32[2 * n + l], __int_as_float((int)l));
}

__device__ __forceinline__ float hm_ex2(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// T_il(z) in FP32 for i != l: the 7-point rule at collocation point x_i over the points
// q[k * stride] (k = 0..6) of panel l, with the general operator's factor (normal nl) when
// op is not the single layer; coordinates relative to x_i.
template <bool general>
__device__ __forceinline__ float2 hm_eval(float xi, float yi, float zi, const float4* q,
                                          int64_t stride, float4 nl, float kr, float ki,
                                          const OpCoef& op) {
  const float kmi = -ki * 1.4426950408889634f;
  float sr = 0.f, si = 0.f;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const float4 y = q[k * stride];
    const float dx = y.x - xi, dy = y.y - yi, dz = y.z - zi;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float rs = rsqrtf(r2);
    const float r = r2 * rs;
    const float a = y.w * rs * hm_ex2(kmi * r);
    float sn, cs;
    __sincosf(kr * r, &sn, &cs);
    if constexpr (general) {
      float fr, fi;
      op_factor(op, (dx * nl.x + dy * nl.y + dz * nl.z) * rs * rs, kr * r, ki * r, fr, fi);
      sr += a * (cs * fr - sn * fi);
      si += a * (cs * fi + sn * fr);
    } else {
      sr = fmaf(a, cs, sr);
      si = fmaf(a, sn, si);
    }
  }
  return make_float2(sr, si);
}

// Entry of cluster row t against cluster column u (t != u as panels).
template <bool general>
__device__ __forceinline__ float2 hm_entry(const HmGeom& g, int64_t t, int64_t u, float kr,
                                           float ki, const OpCoef& op) {
  const float4 x = g.cen[t];
  const float4 nl = general ? g.nrm[u] : make_float4(0.f, 0.f, 0.f, 0.f);
  return hm_eval<general>(x.x, x.y, x.z, g.q + u, g.n, nl, kr, ki, op);
}

constexpr int kAcaThreads = 128;      // threads per far block
constexpr int kAcaThreadsBig = 256;   // for blocks of at least kAcaBig rows + columns
constexpr int kAcaBig = 1024;
constexpr int kMaxRank = 128;

// Block-wide argmax of (v, i) over NT threads: the largest v, the smallest i among equals.
template <int NT>
__device__ __forceinline__ void block_argmax(float& v, int& idx, float* sv, int* si) {
  for (int off = 16; off > 0; off >>= 1) {
    const float ov = __shfl_down_sync(0xffffffffu, v, off);
    const int oi = __shfl_down_sync(0xffffffffu, idx, off);
    if (ov > v || (ov == v && oi < idx)) {
      v = ov;
      idx = oi;
    }
  }
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (lane == 0) {
    sv[w] = v;
    si[w] = idx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < NT / 32; ++k)
      if (sv[k] > sv[0] || (sv[k] == sv[0] && si[k] < si[0])) {
        sv[0] = sv[k];
        si[0] = si[k];
      }
  }
  __syncthreads();
  v = sv[0];
  idx = si[0];
  __syncthreads();
}

// Block-wide sums of a and b over NT threads (warp partials in sa, sb; the same order on
// every thread).
template <int NT>
__device__ __forceinline__ void block_sum2(float& a, float& b, float* sa, float* sb) {
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, off);
    b += __shfl_down_sync(0xffffffffu, b, off);
  }
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (lane == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  a = b = 0.f;
  for (int k = 0; k < NT / 32; ++k) {
    a += sa[k];
    b += sb[k];
  }
  __syncthreads();
}

// One CTA per far block: adaptive cross approximation with partial pivoting.
template <bool general, int NT>
__global__ void __launch_bounds__(NT)
hm_aca_kernel(int base, HmGeom g, const int4* __restrict__ far,
              const int64_t* __restrict__ uw_off, const int64_t* __restrict__ used_off,
              float kr, float ki, OpCoef op, float eps, int rmax, float2* __restrict__ uw,
              uint8_t* __restrict__ used, int32_t* __restrict__ rank) {
  __shared__ float sv[NT / 32], sv2[NT / 32];
  __shared__ int si[NT / 32];
  __shared__ float2 ui[kMaxRank], wj[kMaxRank], au[kMaxRank], aw[kMaxRank];
  __shared__ float2 piv;
  const int b = base + (int)blockIdx.x, tid = threadIdx.x;
  const int4 f = far[b];
  const int m = f.y - f.x, n = f.w - f.z;
  float2* U = uw + uw_off[b];
  float2* W = U + (int64_t)m * rmax;
  uint8_t* fl = used + used_off[b];
  for (int i = tid; i < m; i += NT) fl[i] = 0;
  const int rcap = min(rmax, min(m, n));
  int k = 0, istar = 0, guard = 0;
  float norm2 = 0.f;
  __syncthreads();
  while (k < rcap && guard++ < m + rcap) {
    if (tid == 0) fl[istar] = 1;
    for (int p = tid; p < k; p += NT) ui[p] = U[istar + (int64_t)p * m];
    __syncthreads();
    // residual row i* into W[:, k]
    float best = -1.f;
    int bj = 0x7fffffff;
    for (int l = tid; l < n; l += NT) {
      float2 v = hm_entry<general>(g, f.x + istar, f.z + l, kr, ki, op);
      for (int p = 0; p < k; ++p) {
        const float2 a = ui[p], w = W[l + (int64_t)p * n];
        v.x -= a.x * w.x - a.y * w.y;
        v.y -= a.x * w.y + a.y * w.x;
      }
      W[l + (int64_t)k * n] = v;
      const float mag = v.x * v.x + v.y * v.y;
      if (mag > best) {
        best = mag;
        bj = l;
      }
    }
    block_argmax<NT>(best, bj, sv, si);
    if (!(best > 0.f)) {   // a zero residual row: the next unused row, if any
      float fv = -1.f;
      int fi = 0x7fffffff;
      for (int i = tid; i < m; i += NT)
        if (!fl[i] && fv < 0.f) {
          fv = 0.f;
          fi = i;
        }
      block_argmax<NT>(fv, fi, sv, si);
      if (fv < 0.f) break;
      istar = fi;
      continue;
    }
    if (tid == 0) piv = W[bj + (int64_t)k * n];
    __syncthreads();
    const float2 pv = piv;
    const float ipd = 1.f / (pv.x * pv.x + pv.y * pv.y);
    float nw = 0.f;
    for (int l = tid; l < n; l += NT) {   // w_k = r / r[j*]
      const float2 v = W[l + (int64_t)k * n];
      const float2 q = make_float2((v.x * pv.x + v.y * pv.y) * ipd, (v.y * pv.x - v.x * pv.y) * ipd);
      W[l + (int64_t)k * n] = q;
      nw += q.x * q.x + q.y * q.y;
    }
    for (int p = tid; p < k; p += NT) wj[p] = W[bj + (int64_t)p * n];
    __syncthreads();
    // residual column j* into U[:, k]
    float nu2 = 0.f;
    for (int i = tid; i < m; i += NT) {
      float2 v = hm_entry<general>(g, f.x + i, f.z + bj, kr, ki, op);
      for (int p = 0; p < k; ++p) {
        const float2 a = U[i + (int64_t)p * m], w = wj[p];
        v.x -= a.x * w.x - a.y * w.y;
        v.y -= a.x * w.y + a.y * w.x;
      }
      U[i + (int64_t)k * m] = v;
      nu2 += v.x * v.x + v.y * v.y;
    }
    __syncthreads();
    block_sum2<NT>(nu2, nw, sv, sv2);
    // (U^H u)_p and (W^H w)_p for p < k: warps take p in turn, lanes sum over the rows
    {
      const int wp = tid / 32, lane = tid % 32;
      for (int p = wp; p < k; p += NT / 32) {
        float2 a = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
        for (int i = lane; i < m; i += 32) {
          const float2 x = U[i + (int64_t)p * m], y = U[i + (int64_t)k * m];
          a.x += x.x * y.x + x.y * y.y;
          a.y += x.x * y.y - x.y * y.x;
        }
        for (int l = lane; l < n; l += 32) {
          const float2 x = W[l + (int64_t)p * n], y = W[l + (int64_t)k * n];
          c.x += x.x * y.x + x.y * y.y;
          c.y += x.x * y.y - x.y * y.x;
        }
        for (int off = 16; off > 0; off >>= 1) {
          a.x += __shfl_down_sync(0xffffffffu, a.x, off);
          a.y += __shfl_down_sync(0xffffffffu, a.y, off);
          c.x += __shfl_down_sync(0xffffffffu, c.x, off);
          c.y += __shfl_down_sync(0xffffffffu, c.y, off);
        }
        if (lane == 0) {
          au[p] = a;
          aw[p] = c;
        }
      }
    }
    __syncthreads();
    float cross = 0.f;
    for (int p = 0; p < k; ++p) cross += au[p].x * aw[p].x - au[p].y * aw[p].y;
    norm2 += 2.f * cross + nu2 * nw;
    ++k;
    if (sqrtf(nu2 * nw) <= eps * sqrtf(fmaxf(norm2, 0.f))) break;
    // next row: the largest |u_k| among the unused rows
    float bv = -1.f;
    int bi = 0x7fffffff;
    for (int i = tid; i < m; i += NT) {
      if (fl[i]) continue;
      const float2 v = U[i + (int64_t)(k - 1) * m];
      const float mag = v.x * v.x + v.y * v.y;
      if (mag > bv) {
        bv = mag;
        bi = i;
      }
    }
    block_argmax<NT>(bv, bi, sv, si);
    if (bv < 0.f) break;
    istar = bi;
  }
  if (tid == 0) rank[b] = k;
}

constexpr int kLeafMax = 32;   // rows of a leaf (the leaf size is capped to it)
constexpr int kPanelK = 32;    // depth of a staged panel
constexpr int kHmThreads = 256;

// Panel products on 256 threads: A (up to 32 rows x K) times B (K rows x CW = 64 NCH complex
// columns, row-major in shared memory) accumulated into acc. Two thread mappings with one
// interface (accumulator NR x NC per thread, its rows row(i) and columns col(e), the A slot
// aidx(row, k)); PanelFor picks the faster one per width (measured).
//
// PanelTile (CW = 256): warp w covers the 32 column
// pairs 32 (w % NCH) + lane (columns 2 p and 2 p + 1) for the rows rg + RG i (i < RPT) of
// its row group rg = w / NCH, RG = 8 / NCH, RPT = 32 / RG. A is kept in shared memory as
// a[k][slot], slot = (row % RG) RPT + row / RG, so that a thread's rows are contiguous: one
// broadcast 16-byte read gives two of them, and a warp reads B once for all its rows.
template <int NCH>
struct PanelTile {
  static constexpr int CW = 64 * NCH;
  static constexpr int RG = 8 / NCH;         // row groups
  static constexpr int RPT = kLeafMax / RG;  // rows per thread (even)
  static constexpr int kAS = kLeafMax + 2;   // A row stride (float2; even, 16-byte rows)
  static_assert(RPT % 2 == 0, "row pairs");
  static __device__ __forceinline__ int aidx(int row, int kk) {
    return kk * kAS + (row % RG) * RPT + row / RG;
  }
  static __device__ __forceinline__ int rg() { return ((int)threadIdx.x / 32) / NCH; }
  static __device__ __forceinline__ int pair() {
    return 32 * (((int)threadIdx.x / 32) % NCH) + (int)threadIdx.x % 32;
  }
  static constexpr int NR = RPT, NC = 2;   // accumulator: rows x columns per thread
  static constexpr int ASZ = kPanelK * kAS;  // A tile, float2
  static __device__ __forceinline__ int row(int i) { return rg() + RG * i; }
  static __device__ __forceinline__ int col(int e) { return 2 * pair() + e; }
  // the products for the thread's first 2 NP rows (those beyond the row count are computed
  // on whatever A holds there and never written out)
  template <int NP>
  static __device__ __forceinline__ void mac_rows(const float2* a, const float2* b, int K,
                                                  float2 (&acc)[RPT][2]) {
    const float2* ab = a + rg() * RPT;
    const float2* bb = b + 2 * pair();
#pragma unroll 2
    for (int kk = 0; kk < K; ++kk) {
      const float4 v = *reinterpret_cast<const float4*>(bb + kk * CW);
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const float4 x = *reinterpret_cast<const float4*>(ab + kk * kAS + 2 * j);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float xr = h ? x.z : x.x, xi = h ? x.w : x.y;
          float2& p = acc[2 * j + h][0];
          float2& q = acc[2 * j + h][1];
          p.x = fmaf(xr, v.x, fmaf(-xi, v.y, p.x));
          p.y = fmaf(xr, v.y, fmaf(xi, v.x, p.y));
          q.x = fmaf(xr, v.z, fmaf(-xi, v.w, q.x));
          q.y = fmaf(xr, v.w, fmaf(xi, v.z, q.y));
        }
      }
    }
  }
  static __device__ __forceinline__ void mac(const float2* a, const float2* b, int K, int rows,
                                             float2 (&acc)[RPT][2]) {
    const int g = rg();   // the thread's rows g + RG i, active while below the row count
    const int na = g >= rows ? 0 : min(RPT, (rows - g + RG - 1) / RG);
    const int np = (na + 1) / 2;
    if (np == RPT / 2) mac_rows<RPT / 2>(a, b, K, acc);
    else if (np == 1) mac_rows<1>(a, b, K, acc);
    else if constexpr (RPT >= 6) {
      if (np == 2) mac_rows<2>(a, b, K, acc);
      else if constexpr (RPT >= 8) {
        if (np == 3) mac_rows<3>(a, b, K, acc);
        else if constexpr (RPT >= 16) {
          if (np == 4) mac_rows<4>(a, b, K, acc);
          else if (np == 5) mac_rows<5>(a, b, K, acc);
          else if (np == 6) mac_rows<6>(a, b, K, acc);
          else if (np == 7) mac_rows<7>(a, b, K, acc);
        }
      }
    }
  }
  template <int R, int C2>
  static __device__ __forceinline__ void zero(float2 (&acc)[R][C2]) {
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int e = 0; e < C2; ++e) acc[i][e] = make_float2(0.f, 0.f);
  }
  // B rows [0, K) from rows src + kk * CW (16-byte aligned, CW complex each)
  static __device__ __forceinline__ void stage_b(float2* b, const float2* __restrict__ src, int K) {
    const float4* s = reinterpret_cast<const float4*>(src);
    float4* d = reinterpret_cast<float4*>(b);
    for (int t = threadIdx.x; t < K * (CW / 2); t += kHmThreads) d[t] = s[t];
  }
  static constexpr size_t smem_bytes() {
    return (size_t)kPanelK * CW * sizeof(float2) + kPanelK * (kLeafMax + 2) * sizeof(float2) +
           kPanelK * 8 * sizeof(float4) + kLeafMax * sizeof(float4) + kPanelK * sizeof(int2) +
           (kFarGroup + 1) * sizeof(int);
  }
  static constexpr int kFarGroup = 128;
};

// PanelRows (CW = 64, 128): a warp owns one row per item: thread t owns rows t / 32 + 8 k
// (k < 4) and the column pairs lane + 32 e (e < NCH); A kept as a[row][k] (row stride
// kPanelK + 1). Reads B once per row, but its warps stay busy on short leaves.
template <int NCH>
struct PanelRows : PanelTile<NCH> {
  using Base = PanelTile<NCH>;
  static constexpr int CW = Base::CW;
  static constexpr int NR = 4, NC = 2 * NCH;
  static constexpr int ASZ = kLeafMax * (kPanelK + 1);
  static __device__ __forceinline__ int aidx(int row, int kk) { return row * (kPanelK + 1) + kk; }
  static __device__ __forceinline__ int row(int k) { return (int)threadIdx.x / 32 + 8 * k; }
  static __device__ __forceinline__ int col(int e) {
    return 2 * ((int)threadIdx.x % 32 + 32 * (e / 2)) + e % 2;
  }
  template <int NA>
  static __device__ __forceinline__ void mac_rows(const float2* a, const float2* b, int K,
                                                  float2 (&acc)[NR][NC]) {
    const int cg = (int)threadIdx.x % 32, r0 = (int)threadIdx.x / 32;
#pragma unroll 2
    for (int kk = 0; kk < K; ++kk) {
      float4 v[NCH];
#pragma unroll
      for (int e = 0; e < NCH; ++e)
        v[e] = *reinterpret_cast<const float4*>(b + (int64_t)kk * CW + 2 * (cg + 32 * e));
#pragma unroll
      for (int k = 0; k < NA; ++k) {
        const float2 x = a[(r0 + 8 * k) * (kPanelK + 1) + kk];
#pragma unroll
        for (int e = 0; e < NCH; ++e) {
          float2& p = acc[k][2 * e];
          float2& q = acc[k][2 * e + 1];
          p.x = fmaf(x.x, v[e].x, fmaf(-x.y, v[e].y, p.x));
          p.y = fmaf(x.x, v[e].y, fmaf(x.y, v[e].x, p.y));
          q.x = fmaf(x.x, v[e].z, fmaf(-x.y, v[e].w, q.x));
          q.y = fmaf(x.x, v[e].w, fmaf(x.y, v[e].z, q.y));
        }
      }
    }
  }
  static __device__ __forceinline__ void mac(const float2* a, const float2* b, int K, int rows,
                                             float2 (&acc)[NR][NC]) {
    const int r0 = (int)threadIdx.x / 32;   // the thread's rows r0 + 8 k increase with k
    const int na = r0 >= rows ? 0 : min(NR, (rows - r0 + 7) / 8);
    if (na == 4) mac_rows<4>(a, b, K, acc);
    else if (na == 3) mac_rows<3>(a, b, K, acc);
    else if (na == 2) mac_rows<2>(a, b, K, acc);
    else if (na == 1) mac_rows<1>(a, b, K, acc);
  }
};

template <int NCH>
using PanelFor = typename std::conditional<NCH >= 4, PanelTile<NCH>, PanelRows<NCH>>::type;

// Y_j for the rows of one leaf and every basis column (one CTA per leaf):
//   dense part: the leaf's dense column ranges (contiguous in cluster order), 32 panels at a
//   time: their quadrature points staged, the block T(z_j)[leaf, panels] evaluated into
//   shared memory (self entries from the FP32 self terms), times the staged basis rows;
//   far part: the rank-1 terms u_p w_p^T of every far block above the leaf, as rows of
//   [U_b | ...] (the leaf's rows of U_b) and [T_b; ...] (T_b = W_b^T V), 32 terms a panel;
// in a fixed order (deterministic), then written into the FP32 partials of the mixed path.
// vp: V in cluster order, row-major with CW columns (zero beyond nu); T rows CW wide too.
template <int NCH, bool general>
__global__ void __launch_bounds__(kHmThreads, NCH >= 4 ? 2 : 4)
hm_leaf_kernel(HmGeom g, const int4* __restrict__ leaves, const int2* __restrict__ near,
               const int32_t* __restrict__ leaf_far_ptr, const int32_t* __restrict__ leaf_far,
               const int4* __restrict__ far, const int64_t* __restrict__ uw_off,
               const int32_t* __restrict__ rank, const int64_t* __restrict__ toff,
               const float2* __restrict__ uw, const float2* __restrict__ T,
               const float2* __restrict__ vp, int nu, const float2* __restrict__ self32,
               float kr, float ki, OpCoef op, float* __restrict__ Yp, int C, int64_t n_pad) {
  using P = PanelFor<NCH>;
  extern __shared__ float4 hm_smem[];
  float2* sB = reinterpret_cast<float2*>(hm_smem);
  float2* sA = sB + kPanelK * P::CW;                          // A tile, slots P::aidx
  float4* sQ = reinterpret_cast<float4*>(sA + kPanelK * (kLeafMax + 2));   // [kk][8]: 7 points, normal
  float4* sX = sQ + kPanelK * 8;
  int2* sMap = reinterpret_cast<int2*>(sX + kLeafMax);
  int* sPre = reinterpret_cast<int*>(sMap + kPanelK);
  const int L = blockIdx.x;
  const int tid = threadIdx.x;
  const int4 lf = leaves[L];   // rows [x, y), dense ranges [z, w)
  const int mL = lf.y - lf.x;
  const int64_t n = g.n;
  if (tid < kLeafMax) sX[tid] = tid < mL ? g.cen[lf.x + tid] : make_float4(0.f, 0.f, 0.f, 0.f);
  float2 acc[P::NR][P::NC];
  P::zero(acc);
  for (int nb = lf.z; nb < lf.w; ++nb) {
    const int2 sg = near[nb];
    for (int k0 = sg.x; k0 < sg.y; k0 += kPanelK) {
      const int K = min(kPanelK, sg.y - k0);
      __syncthreads();
      for (int t = tid; t < 8 * kPanelK; t += kHmThreads) {
        const int kk = t % kPanelK, q = t / kPanelK;
        if (kk < K)
          sQ[kk * 8 + q] = q < 7 ? g.q[q * n + k0 + kk]
                                 : (general ? g.nrm[k0 + kk] : make_float4(0.f, 0.f, 0.f, 0.f));
      }
      P::stage_b(sB, vp + (int64_t)k0 * P::CW, K);
      __syncthreads();
      for (int t = tid; t < mL * K; t += kHmThreads) {
        const int rr = t % mL, kk = t / mL;
        const float4 x = sX[rr];
        sA[P::aidx(rr, kk)] = (lf.x + rr == k0 + kk)
                         ? self32[__float_as_int(x.w)]
                         : hm_eval<general>(x.x, x.y, x.z, sQ + kk * 8, 1, sQ[kk * 8 + 7], kr, ki, op);
      }
      __syncthreads();
      P::mac(sA, sB, K, mL, acc);
    }
  }
  const int fe = leaf_far_ptr[L + 1];
  for (int g0 = leaf_far_ptr[L]; g0 < fe; g0 += P::kFarGroup) {
    const int gn = min(P::kFarGroup, fe - g0);
    __syncthreads();
    if (tid == 0) {   // term offsets of the group's far blocks
      int s = 0;
      for (int e = 0; e < gn; ++e) {
        sPre[e] = s;
        s += rank[leaf_far[g0 + e]];
      }
      sPre[gn] = s;
    }
    __syncthreads();
    const int Kt = sPre[gn];
    for (int k0 = 0; k0 < Kt; k0 += kPanelK) {
      const int K = min(kPanelK, Kt - k0);
      if (tid < K) {   // term k0 + tid: far block and rank index
        const int want = k0 + tid;
        int lo = 0, hi = gn - 1;   // the last e with sPre[e] <= want
        while (lo < hi) {
          const int mid = (lo + hi + 1) / 2;
          if (sPre[mid] <= want) lo = mid; else hi = mid - 1;
        }
        sMap[tid] = make_int2(leaf_far[g0 + lo], want - sPre[lo]);
      }
      __syncthreads();
      for (int t = tid; t < K * (P::CW / 2); t += kHmThreads) {
        const int kk = t / (P::CW / 2), c = t % (P::CW / 2);
        const int2 bp = sMap[kk];
        reinterpret_cast<float4*>(sB)[t] =
            reinterpret_cast<const float4*>(T + toff[bp.x] + (int64_t)bp.y * P::CW)[c];
      }
      for (int t = tid; t < K * mL; t += kHmThreads) {
        const int rr = t % mL, kk = t / mL;
        const int2 bp = sMap[kk];
        const int4 f = far[bp.x];
        sA[P::aidx(rr, kk)] = uw[uw_off[bp.x] + (lf.x - f.x + rr) + (int64_t)bp.y * (f.y - f.x)];
      }
      __syncthreads();
      P::mac(sA, sB, K, mL, acc);
      __syncthreads();
    }
  }
#pragma unroll
  for (int k = 0; k < P::NR; ++k) {
    const int r = P::row(k);
    if (r >= mL) continue;
    const int64_t i = __float_as_int(sX[r].w);
#pragma unroll
    for (int e = 0; e < P::NC; ++e) {
      const int c = P::col(e);
      if (c < nu) {   // real part at column (c / C) 2 C + c % C, imaginary part C further
        const int64_t colr = (int64_t)(c / C) * 2 * C + c % C;
        Yp[colr * n_pad + i] = acc[k][e].x;
        Yp[(colr + C) * n_pad + i] = acc[k][e].y;
      }
    }
  }
}

// T_b = W_b^T V_sigma (rank x CW, row-major) per far block (one CTA each), 32 ranks and 32
// panels of sigma per panel product.
template <int NCH>
__global__ void __launch_bounds__(kHmThreads, NCH >= 4 ? 2 : 3)
hm_wtv_kernel(const int4* __restrict__ far, const int64_t* __restrict__ uw_off,
              const int32_t* __restrict__ rank, const int64_t* __restrict__ toff, int rmax,
              const float2* __restrict__ uw, const float2* __restrict__ vp,
              float2* __restrict__ T) {
  using P = PanelFor<NCH>;
  extern __shared__ float4 hm_smem[];
  float2* sB = reinterpret_cast<float2*>(hm_smem);
  float2* sA = sB + kPanelK * P::CW;   // A tile, slots P::aidx
  const int b = blockIdx.x, tid = threadIdx.x;
  const int4 f = far[b];
  const int m = f.y - f.x, n = f.w - f.z;
  const int r = rank[b];
  const float2* W = uw + uw_off[b] + (int64_t)m * rmax;
  float2* Tb = T + toff[b];
  for (int p0 = 0; p0 < r; p0 += kLeafMax) {
    const int rows = min(kLeafMax, r - p0);
    float2 acc[P::NR][P::NC];
    P::zero(acc);
    for (int l0 = 0; l0 < n; l0 += kPanelK) {
      const int K = min(kPanelK, n - l0);
      __syncthreads();
      for (int t = tid; t < rows * kPanelK; t += kHmThreads) {
        const int kk = t % kPanelK, pp = t / kPanelK;
        if (kk < K) sA[P::aidx(pp, kk)] = W[(l0 + kk) + (int64_t)(p0 + pp) * n];
      }
      P::stage_b(sB, vp + (int64_t)(f.z + l0) * P::CW, K);
      __syncthreads();
      P::mac(sA, sB, K, rows, acc);
    }
#pragma unroll
    for (int k = 0; k < P::NR; ++k) {
      const int pr = P::row(k);
      if (pr >= rows) continue;
#pragma unroll
      for (int e = 0; e < P::NC; e += 2)   // columns col(e), col(e) + 1
        reinterpret_cast<float4*>(Tb + (int64_t)(p0 + pr) * P::CW)[P::col(e) / 2] =
            make_float4(acc[k][e].x, acc[k][e].y, acc[k][e + 1].x, acc[k][e + 1].y);
    }
  }
}

// vp[t][c] = V[perm[t], c] in FP32 (cluster order, row-major, cw columns, zero beyond nu)
__global__ void hm_vperm_kernel(const double2* __restrict__ V, int64_t ldv, int64_t n, int nu,
                                int cw, const int32_t* __restrict__ perm, float2* __restrict__ vp) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * cw) return;
  const int64_t row = t / cw;
  const int c = (int)(t % cw);
  float2 o = make_float2(0.f, 0.f);
  if (c < nu) {
    const double2 v = V[(int64_t)c * ldv + perm[row]];
    o = make_float2((float)v.x, (float)v.y);
  }
  vp[t] = o;
}

}  // namespace

namespace {

template <typename T>
bem_status upload(bem_ctx* ctx, T*& dst, const std::vector<T>& src) {
  cudaFree(dst);
  dst = nullptr;
  const size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
  if (cudaMalloc(&dst, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, BEM_ENOMEM, "low-rank far field: device allocation failed");
  }
  if (!src.empty())
    return cuda_check(ctx, cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice),
                      "low-rank far field copy");
  return BEM_OK;
}

template <typename T>
bem_status grow(bem_ctx* ctx, T*& p, size_t& cap, size_t bytes) {
  if (bytes <= cap) return BEM_OK;
  cudaFree(p);
  p = nullptr;
  cap = 0;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, BEM_ENOMEM, "low-rank far field: device allocation failed");
  }
  cap = bytes;
  return BEM_OK;
}

// The cluster tree, the block partition and the per-leaf lists of the current mesh.
bem_status build_structure(bem_ctx* ctx, cudaStream_t s) {
  HMatrix& h = *ctx->hm;
  const int64_t n = ctx->geo.n;
  const std::vector<double>& xyz = ctx->h_xyz;
  const std::vector<int32_t>& tri = ctx->h_tri;
  std::vector<double> cen(3 * n);
  for (int64_t l = 0; l < n; ++l)
    for (int d = 0; d < 3; ++d)
      cen[3 * l + d] = (xyz[3 * (int64_t)tri[3 * l] + d] + xyz[3 * (int64_t)tri[3 * l + 1] + d] +
                        xyz[3 * (int64_t)tri[3 * l + 2] + d]) / 3.0;
  h.perm.resize(n);
  std::iota(h.perm.begin(), h.perm.end(), 0);
  h.cl.clear();
  build_cluster(h, cen, xyz, tri, 0, (int32_t)n);
  std::vector<int2> far_cl, near_cl;
  build_blocks(h, 0, 0, far_cl, near_cl);
  // far blocks largest first (rows + columns; ties keep the partition's order)
  auto fsize = [&](const int2& fb) {
    return (h.cl[fb.x].e - h.cl[fb.x].b) + (h.cl[fb.y].e - h.cl[fb.y].b);
  };
  std::stable_sort(far_cl.begin(), far_cl.end(),
                   [&](const int2& a, const int2& b) { return fsize(a) > fsize(b); });
  h.nbig = 0;
  while (h.nbig < (int)far_cl.size() && fsize(far_cl[h.nbig]) >= kAcaBig) ++h.nbig;
  // far blocks and their storage
  h.far.clear();
  h.uw_off.clear();
  h.used_off.clear();
  h.uw_total = h.used_total = 0;
  double far_entries = 0.0;
  for (const int2& fb : far_cl) {
    const HMatrix::Cl& A = h.cl[fb.x];
    const HMatrix::Cl& B = h.cl[fb.y];
    h.far.push_back(make_int4(A.b, A.e, B.b, B.e));
    h.uw_off.push_back(h.uw_total);
    h.uw_total += (int64_t)(A.e - A.b + B.e - B.b) * h.rmax;
    h.used_off.push_back(h.used_total);
    h.used_total += A.e - A.b;
    far_entries += (double)(A.e - A.b) * (B.e - B.b);
  }
  h.far_fraction = far_entries / ((double)n * n);
  // leaves in cluster order, their dense blocks and the far blocks above them
  std::vector<int> leaf_id(h.cl.size(), -1);
  h.leaves.clear();
  for (size_t c = 0; c < h.cl.size(); ++c)
    if (h.cl[c].c0 < 0) leaf_id[c] = 0;
  std::vector<int> leaf_cl;
  for (size_t c = 0; c < h.cl.size(); ++c)
    if (h.cl[c].c0 < 0) leaf_cl.push_back((int)c);
  std::sort(leaf_cl.begin(), leaf_cl.end(), [&](int a, int b) { return h.cl[a].b < h.cl[b].b; });
  for (size_t t = 0; t < leaf_cl.size(); ++t) leaf_id[leaf_cl[t]] = (int)t;
  std::vector<std::vector<int2>> lnear(leaf_cl.size());
  for (const int2& nb : near_cl)
    lnear[leaf_id[nb.x]].push_back(make_int2(h.cl[nb.y].b, h.cl[nb.y].e));
  h.dense_blocks = (int64_t)near_cl.size();
  for (std::vector<int2>& r : lnear) {   // ranges sorted, adjacent ones merged
    std::sort(r.begin(), r.end(), [](int2 a, int2 b) { return a.x < b.x; });
    size_t w = 0;
    for (size_t e = 0; e < r.size(); ++e) {
      if (w && r[w - 1].y == r[e].x) r[w - 1].y = r[e].y;
      else r[w++] = r[e];
    }
    r.resize(w);
  }
  std::vector<std::vector<int32_t>> lfar(leaf_cl.size());
  // the leaves inside a far block's row cluster are consecutive (leaves sorted by start)
  std::vector<int32_t> leaf_start(leaf_cl.size());
  for (size_t t = 0; t < leaf_cl.size(); ++t) leaf_start[t] = h.cl[leaf_cl[t]].b;
  for (size_t b = 0; b < h.far.size(); ++b) {
    const int4 f = h.far[b];
    size_t t = std::lower_bound(leaf_start.begin(), leaf_start.end(), f.x) - leaf_start.begin();
    for (; t < leaf_cl.size() && h.cl[leaf_cl[t]].e <= f.y; ++t) lfar[t].push_back((int32_t)b);
  }
  h.near.clear();
  h.dense_entries = 0.0;
  h.leaf_far.clear();
  h.leaf_far_ptr.assign(1, 0);
  for (size_t t = 0; t < leaf_cl.size(); ++t) {
    const HMatrix::Cl& Lc = h.cl[leaf_cl[t]];
    const int nb0 = (int)h.near.size();
    for (const int2& s : lnear[t]) h.near.push_back(s);
    h.leaves.push_back(make_int4(Lc.b, Lc.e, nb0, (int)h.near.size()));
    for (const int2& r : lnear[t]) h.dense_entries += (double)(Lc.e - Lc.b) * (r.y - r.x);
    for (int32_t b : lfar[t]) h.leaf_far.push_back(b);
    h.leaf_far_ptr.push_back((int32_t)h.leaf_far.size());
  }
  bem_status st = upload(ctx, h.d_perm, h.perm);
  if (st == BEM_OK) st = upload(ctx, h.d_far, h.far);
  if (st == BEM_OK) st = upload(ctx, h.d_uw_off, h.uw_off);
  if (st == BEM_OK) st = upload(ctx, h.d_used_off, h.used_off);
  if (st == BEM_OK) st = upload(ctx, h.d_leaves, h.leaves);
  if (st == BEM_OK) st = upload(ctx, h.d_leaf_far_ptr, h.leaf_far_ptr);
  if (st == BEM_OK) st = upload(ctx, h.d_leaf_far, h.leaf_far);
  if (st == BEM_OK) st = upload(ctx, h.d_near, h.near);
  if (st != BEM_OK) return st;
  cudaFree(h.d_gq);
  h.d_gq = h.d_gn = h.d_gc = nullptr;
  if (cudaMalloc(&h.d_gq, (size_t)n * 9 * sizeof(float4)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, BEM_ENOMEM, "low-rank far field: device allocation failed");
  }
  h.d_gn = h.d_gq + 7 * n;
  h.d_gc = h.d_gq + 8 * n;
  hm_geom_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ctx->geo, h.d_perm, h.d_gq, h.d_gn, h.d_gc);
  ctx->launches++;
  h.mesh_version = ctx->mesh_version;
  return BEM_OK;
}

unsigned nblocks(int64_t count, int t = 256) { return (unsigned)((count + t - 1) / t); }

// The W^T V and leaf kernels for CW = 64 NCH basis columns (the dynamic shared memory of
// NCH = 4 exceeds the default 48 KB and is opted in).
template <int NCH, bool general>
bem_status hm_apply_kernels(bem_ctx* ctx, HMatrix& h, bool wtv, int j, int nu, float kr, float ki,
                            const ExtFrame& fr, cudaStream_t s) {
  const size_t smem = PanelFor<NCH>::smem_bytes();
  if (cudaFuncSetAttribute(hm_leaf_kernel<NCH, general>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(hm_wtv_kernel<NCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return cuda_check(ctx, cudaGetLastError(), "low-rank far field kernel attributes");
  const int64_t n = ctx->geo.n;
  const HmGeom g{h.d_gq, h.d_gn, h.d_gc, n};
  if (wtv) {
    hm_wtv_kernel<NCH><<<(unsigned)h.far.size(), kHmThreads, smem, s>>>(
        h.d_far, h.d_uw_off, h.d_rank, h.d_toff, h.rmax, h.d_uw, h.d_vp, h.d_t);
    ctx->launches++;
  }
  timing_begin(ctx, s);
  hm_leaf_kernel<NCH, general><<<(unsigned)h.leaves.size(), kHmThreads, smem, s>>>(
      g, h.d_leaves, h.d_near, h.d_leaf_far_ptr, h.d_leaf_far, h.d_far, h.d_uw_off, h.d_rank,
      h.d_toff, h.d_uw, h.d_t, h.d_vp, nu,
      reinterpret_cast<const float2*>(ctx->con.self32) + (int64_t)j * n, kr, ki, ctx->op,
      fr.Yp + (int64_t)j * fr.acc_cols * fr.n_pad, fr.C, fr.n_pad);
  timing_end(ctx, s);
  ctx->launches++;
  return cuda_check(ctx, cudaGetLastError(), "low-rank far field kernels");
}

}  // namespace

void free_hmatrix(bem_ctx* ctx) {
  if (!ctx->hm) return;
  free_dev(*ctx->hm);
  free_work(*ctx->hm);
  delete ctx->hm;
  ctx->hm = nullptr;
}

bem_status project_hmatrix(bem_ctx* ctx, const double* V, int64_t ldv, int nu, double* Bhat,
                           double* AV, cudaStream_t s) {
  if (!ctx->hm) return fail(ctx, BEM_ESTATE, "bem_project: no low-rank far field set (bem_set_hmatrix)");
  HMatrix& h = *ctx->hm;
  const int64_t n = ctx->geo.n;
  const int N = ctx->con.N;
  if (ctx->h_xyz.empty()) return fail(ctx, BEM_ESTATE, "bem_project: no mesh set");
  bem_status st = BEM_OK;
  if (h.mesh_version != ctx->mesh_version && (st = build_structure(ctx, s)) != BEM_OK) return st;
  if ((st = ensure_self32(ctx, s)) != BEM_OK) return st;
  const size_t nfar = h.far.size();
  if ((st = grow(ctx, h.d_uw, h.uw_bytes, std::max<size_t>(1, h.uw_total) * sizeof(float2))) != BEM_OK ||
      (st = grow(ctx, h.d_used, h.used_bytes, std::max<size_t>(1, h.used_total))) != BEM_OK ||
      (st = grow(ctx, h.d_vp, h.vp_bytes, (size_t)n * 256 * sizeof(float2))) != BEM_OK)
    return st;
  const int nch = nu <= 64 ? 1 : nu <= 128 ? 2 : 4;   // basis columns padded to CW = 64 nch
  const int cw = 64 * nch;
  size_t rc = h.rank_cap, tc = h.rank_cap;
  if ((st = grow(ctx, h.d_rank, rc, std::max<size_t>(1, nfar) * sizeof(int32_t))) != BEM_OK ||
      (st = grow(ctx, h.d_toff, tc, std::max<size_t>(1, nfar) * sizeof(int64_t))) != BEM_OK)
    return st;
  h.rank_cap = std::min(rc, tc);
  // the mixed path's FP32 partials (slice 0 of one column split), zeroed: the leaf kernels
  // write every row < n and column < nu
  ExtFrame fr;
  if ((st = external_begin(ctx, V, ldv, nu, fr, s)) != BEM_OK) return st;
  st = cuda_check(ctx, cudaMemsetAsync(fr.Yp, 0, (size_t)N * fr.acc_cols * fr.n_pad * sizeof(float), s),
                  "partials clear");
  if (st != BEM_OK) {
    external_release(fr);
    return st;
  }
  hm_vperm_kernel<<<nblocks(n * cw), 256, 0, s>>>(reinterpret_cast<const double2*>(V), ldv, n, nu,
                                                  cw, h.d_perm, h.d_vp);
  ctx->launches++;
  std::vector<int32_t> ranks(nfar);
  std::vector<int64_t> toff(nfar);
  const bool single = op_single(ctx->op);
  double rank_sum = 0.0, row_terms = 0.0, col_terms = 0.0;
  int rank_max = 0;
  for (int j = 0; j < N; ++j) {
    const float kr = (float)ctx->con.z_host[2 * j], ki = (float)ctx->con.z_host[2 * j + 1];
    if (nfar) {
      // the far blocks are ordered by size, largest first: those of at least kAcaBig rows +
      // columns take the wider kernel
      const HmGeom hg{h.d_gq, h.d_gn, h.d_gc, n};
      const int nbig = h.nbig, nsmall = (int)nfar - h.nbig;
#define HM_ACA(GEN, NT, BASE, COUNT)                                                          \
  hm_aca_kernel<GEN, NT><<<(unsigned)(COUNT), NT, 0, s>>>(BASE, hg, h.d_far, h.d_uw_off,      \
                                                        h.d_used_off, kr, ki, ctx->op,        \
                                                        (float)h.eps, h.rmax, h.d_uw, h.d_used, \
                                                        h.d_rank)
      if (single) {
        if (nbig) HM_ACA(false, kAcaThreadsBig, 0, nbig);
        if (nsmall) HM_ACA(false, kAcaThreads, nbig, nsmall);
      } else {
        if (nbig) HM_ACA(true, kAcaThreadsBig, 0, nbig);
        if (nsmall) HM_ACA(true, kAcaThreads, nbig, nsmall);
      }
#undef HM_ACA
      ctx->launches += (nbig > 0) + (nsmall > 0) - 1;
      ctx->launches++;
      st = cuda_check(ctx, cudaMemcpyAsync(ranks.data(), h.d_rank, nfar * sizeof(int32_t),
                                           cudaMemcpyDeviceToHost, s), "rank copy");
      if (st == BEM_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), "rank copy");
      if (st != BEM_OK) {
        external_release(fr);
        return st;
      }
      int64_t tot = 0;
      for (size_t b = 0; b < nfar; ++b) {
        toff[b] = tot;
        tot += (int64_t)ranks[b] * cw;
        rank_sum += ranks[b];
        row_terms += (double)ranks[b] * (h.far[b].y - h.far[b].x);
        col_terms += (double)ranks[b] * (h.far[b].w - h.far[b].z);
        rank_max = std::max(rank_max, ranks[b]);
      }
      if ((st = grow(ctx, h.d_t, h.t_bytes, std::max<int64_t>(1, tot) * sizeof(float2))) != BEM_OK) {
        external_release(fr);
        return st;
      }
      st = cuda_check(ctx, cudaMemcpyAsync(h.d_toff, toff.data(), nfar * sizeof(int64_t),
                                           cudaMemcpyHostToDevice, s), "offset copy");
      if (st != BEM_OK) {
        external_release(fr);
        return st;
      }
    }
    if (single)
      st = nch == 1   ? hm_apply_kernels<1, false>(ctx, h, nfar > 0, j, nu, kr, ki, fr, s)
           : nch == 2 ? hm_apply_kernels<2, false>(ctx, h, nfar > 0, j, nu, kr, ki, fr, s)
                      : hm_apply_kernels<4, false>(ctx, h, nfar > 0, j, nu, kr, ki, fr, s);
    else
      st = nch == 1   ? hm_apply_kernels<1, true>(ctx, h, nfar > 0, j, nu, kr, ki, fr, s)
           : nch == 2 ? hm_apply_kernels<2, true>(ctx, h, nfar > 0, j, nu, kr, ki, fr, s)
                      : hm_apply_kernels<4, true>(ctx, h, nfar > 0, j, nu, kr, ki, fr, s);
    if (st != BEM_OK) {
      external_release(fr);
      return st;
    }
  }
  h.mean_rank = nfar ? rank_sum / ((double)nfar * N) : 0.0;
  h.max_rank = rank_max;
  h.far_row_terms = row_terms / N;
  h.far_col_terms = col_terms / N;
  return external_end(ctx, fr, nu, Bhat, AV, s);
}

}  // namespace bem

using namespace bem;

extern "C" bem_status bem_set_hmatrix(bem_ctx* ctx, int leaf, double eta, double eps, int rmax) {
  if (!ctx) return BEM_EINVAL;
  if (leaf < 1 || leaf > kLeafMax || !(eta > 0.0) || !(eps > 0.0) || eps >= 1.0 || rmax < 1 ||
      rmax > kMaxRank)
    return fail(ctx, BEM_EINVAL,
                "bem_set_hmatrix: need 1 <= leaf <= 32, eta > 0, 0 < eps < 1, 1 <= rmax <= 128");
  if (!ctx->hm) ctx->hm = new HMatrix();
  HMatrix& h = *ctx->hm;
  h.leaf = leaf;
  h.eta = eta;
  h.eps = eps;
  h.rmax = rmax;
  h.mesh_version = -1;   // rebuilt (and its storage re-laid out) by the next projection
  free_work(h);
  return BEM_OK;
}

extern "C" bem_status bem_hmatrix_work(const bem_ctx* ctx, double* dense_entries,
                                       double* far_row_terms, double* far_col_terms) {
  if (!ctx) return BEM_EINVAL;
  if (!ctx->hm) return BEM_ESTATE;
  const HMatrix& h = *ctx->hm;
  if (dense_entries) *dense_entries = h.dense_entries;
  if (far_row_terms) *far_row_terms = h.far_row_terms;
  if (far_col_terms) *far_col_terms = h.far_col_terms;
  return BEM_OK;
}

extern "C" bem_status bem_hmatrix_stats(const bem_ctx* ctx, int64_t* far_blocks,
                                        int64_t* dense_blocks, double* far_fraction,
                                        double* mean_rank, int* max_rank) {
  if (!ctx) return BEM_EINVAL;
  if (!ctx->hm) return BEM_ESTATE;
  const HMatrix& h = *ctx->hm;
  if (far_blocks) *far_blocks = (int64_t)h.far.size();
  if (dense_blocks) *dense_blocks = h.dense_blocks;
  if (far_fraction) *far_fraction = h.far_fraction;
  if (mean_rank) *mean_rank = h.mean_rank;
  if (max_rank) *max_rank = h.max_rank;
  return BEM_OK;
}
