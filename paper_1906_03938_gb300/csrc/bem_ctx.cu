// Context, error handling, mesh and contour set-up, and the projection entry point.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "internal.h"

namespace bem {

bem_status fail(bem_ctx* ctx, bem_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

bem_status cuda_check(bem_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return BEM_OK;
  return fail(ctx, BEM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bem_status ensure_scratch(bem_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->scratch_bytes) return BEM_OK;
  if (ctx->d_scratch) cudaFree(ctx->d_scratch);
  ctx->d_scratch = nullptr;
  ctx->scratch_bytes = 0;
  if (cudaMalloc(&ctx->d_scratch, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, BEM_ENOMEM, "scratch allocation of " + std::to_string(bytes) + " bytes failed");
  }
  ctx->scratch_bytes = bytes;
  return BEM_OK;
}

bem_status ensure_small(bem_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->small_bytes) return BEM_OK;
  if (ctx->d_small) cudaFree(ctx->d_small);
  ctx->d_small = nullptr;
  ctx->small_bytes = 0;
  if (cudaMalloc(&ctx->d_small, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, BEM_ENOMEM, "workspace allocation failed");
  }
  ctx->small_bytes = bytes;
  return BEM_OK;
}

bem_status take_status(bem_ctx* ctx, cudaStream_t stream, const char* where) {
  int h = 0;
  bem_status st = cuda_check(ctx, cudaMemcpyAsync(&h, ctx->d_status, sizeof(int),
                                                  cudaMemcpyDeviceToHost, stream), where);
  if (st != BEM_OK) return st;
  st = cuda_check(ctx, cudaStreamSynchronize(stream), where);
  if (st != BEM_OK) return st;
  if (h == 0) return BEM_OK;
  cudaMemsetAsync(ctx->d_status, 0, sizeof(int), stream);
  cudaStreamSynchronize(stream);
  std::string m = std::string(where) + ": device reported";
  if (h & kStatusBadIndex) m += " vertex-index-out-of-range";
  if (h & kStatusZeroArea) m += " zero-area-triangle";
  if (h & kStatusNotSPD) m += " Gram-matrix-not-positive-definite";
  if (h & kStatusNonFinite) m += " non-finite-value";
  if (h & kStatusTimeout) m += " wait-timeout";
  if (h & kStatusTimeout) return fail(ctx, BEM_ETIMEOUT, m);
  return fail(ctx, (h & (kStatusBadIndex | kStatusZeroArea)) ? BEM_EINVAL : BEM_EKERNEL, m);
}

static void free_geometry(Geometry& g) {
  cudaFree(g.xyz); cudaFree(g.tri); cudaFree(g.cx); cudaFree(g.qp); cudaFree(g.qw);
  cudaFree(g.cx32); cudaFree(g.qp32); cudaFree(g.qw32); cudaFree(g.edge32); cudaFree(g.pack32);
  cudaFree(g.mom32); cudaFree(g.rho32); cudaFree(g.diam); cudaFree(g.nrm);
  g = Geometry();
}

static void free_contour(Contour& c) {
  cudaFree(c.z); cudaFree(c.w); cudaFree(c.self); cudaFree(c.self32); cudaFree(c.order);
  c.z = c.w = c.self = nullptr;
  c.order = nullptr;
  c.twins = 0;
  c.self32 = nullptr;
  c.self64_ready = c.self32_ready = false;
  c.N = 0;
  c.cap_N = 0;
  c.cap_self = 0;
}

bem_status ensure_self64(bem_ctx* ctx, cudaStream_t s) {
  if (ctx->con.self64_ready) return BEM_OK;
  bem_status st = cuda_check(ctx, launch_self_terms(ctx, s), "self-term kernel");
  if (st == BEM_OK) ctx->con.self64_ready = true;
  return st;
}

bem_status ensure_self32(bem_ctx* ctx, cudaStream_t s) {
  if (ctx->con.self32_ready) return BEM_OK;
  bem_status st = cuda_check(ctx, launch_self_terms32(ctx, s), "self-term kernel");
  if (st == BEM_OK) ctx->con.self32_ready = true;
  return st;
}

// Node schedule of the mixed evaluation. Nodes whose real parts round to the same FP32
// value (the conjugate nodes of a contour symmetric about a horizontal line) evaluate the
// same phase Re(z) r at every quadrature point, so the kernel computes its sine and cosine
// once for both: twins first, in pairs at even slots (the first flagged), then the rest.
static void build_node_order(Contour& c) {
  const int N = c.N;
  std::vector<char> used(N, 0);
  std::vector<int> single;
  int slot = 0;
  c.twins = 0;
  for (int j = 0; j < N; ++j) {
    if (used[j]) continue;
    used[j] = 1;
    const float rj = (float)c.z_host[2 * j];
    int m = -1;
    for (int k = j + 1; k < N && m < 0; ++k)
      if (!used[k] && (float)c.z_host[2 * k] == rj) m = k;
    if (m < 0) {
      single.push_back(j);
      continue;
    }
    used[m] = 1;
    c.order_host[slot++] = j | kTwinBit;
    c.order_host[slot++] = m;
    c.twins++;
  }
  for (int j : single) c.order_host[slot++] = j;
}

// A pinned staging buffer of at least `bytes`, free to be rewritten (the copy behind its
// event has completed).
static bem_status stage_buffer(bem_ctx* ctx, void*& buf, size_t& cap, cudaEvent_t& ev,
                               size_t bytes) {
  if (ev) cudaEventSynchronize(ev);
  else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
    return cuda_check(ctx, cudaGetLastError(), "staging event");
  if (bytes > cap) {
    cudaFreeHost(buf);
    buf = nullptr;
    cap = 0;
    if (cudaMallocHost(&buf, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, BEM_ENOMEM, "pinned staging allocation failed");
    }
    cap = bytes;
  }
  return BEM_OK;
}

// Nodes and weights of a contour, on the host (the device receives these values).
// Circle / ellipse: theta_j = pi (2 j + 1) / N with the lower half the exact mirror of the
// upper (theta_{N-1-j} = 2 pi - theta_j), so conjugate nodes have equal real parts.
void contour_nodes(int kind, double c_re, double c_im, double a, double b, int N, double* z,
                   double* w) {
  const double pi = 3.14159265358979323846;
  for (int j = 0; j < N; ++j) {
    if (kind == BEM_CONTOUR_CHEBYSHEV) {
      z[2 * j] = c_re + a * cos(pi * (j + 0.5) / N);
      z[2 * j + 1] = c_im;
      w[2 * j] = 1.0;
      w[2 * j + 1] = 0.0;
      continue;
    }
    const int m = 2 * j + 1 > N ? N - 1 - j : j;
    const double th = pi * (2.0 * m + 1.0) / N;
    double sn = sin(th);
    const double cs = cos(th);
    if (2 * m + 1 == N) sn = 0.0;   // theta = pi exactly
    if (m != j) sn = -sn;
    z[2 * j] = c_re + a * cs;
    z[2 * j + 1] = c_im + b * sn;
    w[2 * j] = b * cs / N;
    w[2 * j + 1] = a * sn / N;
  }
}

}  // namespace bem

using namespace bem;

extern "C" {

const char* bem_version(void) { return "bem_gb300 0.1 (sm_103a)"; }

bem_status bem_create(bem_ctx** out, int device) {
  if (!out) return BEM_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
    cudaGetLastError();
    return BEM_ECUDA;
  }
  if (device < 0 || device >= count) return BEM_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return BEM_ECUDA;
  bem_ctx* ctx = new bem_ctx();
  ctx->device = device;
  if (cudaMalloc(&ctx->d_status, sizeof(int)) != cudaSuccess ||
      cudaMemset(ctx->d_status, 0, sizeof(int)) != cudaSuccess) {
    delete ctx;
    return BEM_ECUDA;
  }
  *out = ctx;
  return BEM_OK;
}

void bem_destroy(bem_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  free_geometry(ctx->geo);
  free_contour(ctx->con);
  cudaFree(ctx->d_status);
  cudaFree(ctx->d_scratch);
  cudaFree(ctx->d_small);
  cudaFree(ctx->d_piv_val);
  cudaFree(ctx->d_piv_idx);
  cudaFree(ctx->d_lu_work);
  cudaFree(ctx->d_zgemm);
  release_cublas(ctx);
  cudaFree(ctx->d_solve);
  cudaFree(ctx->d_near_ptr);
  cudaFree(ctx->d_near_cols);
  cudaFree(ctx->d_near_work);
  cudaFree(ctx->d_sur_usage);
  cudaFree(ctx->d_net);
  free_hmatrix(ctx);
  for (auto& e : ctx->ev) cudaEventDestroy(e);
  if (ctx->mesh_ev) cudaEventSynchronize(ctx->mesh_ev);
  if (ctx->con_ev) cudaEventSynchronize(ctx->con_ev);
  cudaFreeHost(ctx->h_mesh);
  cudaFreeHost(ctx->h_con);
  if (ctx->mesh_ev) cudaEventDestroy(ctx->mesh_ev);
  if (ctx->con_ev) cudaEventDestroy(ctx->con_ev);
  delete ctx;
}

const char* bem_last_error(const bem_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

int64_t bem_kernel_launches(const bem_ctx* ctx) { return ctx ? ctx->launches : 0; }

bem_status bem_set_operator(bem_ctx* ctx, double cg_re, double cg_im, double ch_re,
                            double ch_im) {
  if (!ctx) return BEM_EINVAL;
  if (!isfinite(cg_re) || !isfinite(cg_im) || !isfinite(ch_re) || !isfinite(ch_im) ||
      (cg_re == 0.0 && cg_im == 0.0 && ch_re == 0.0 && ch_im == 0.0))
    return fail(ctx, BEM_EINVAL, "bem_set_operator: coefficients must be finite and not both zero");
  const bool has_h = ch_re != 0.0 || ch_im != 0.0;
  if (has_h && ctx->near_mode == 2)
    return fail(ctx, BEM_EINVAL,
                "bem_set_operator: the surrogate near field (mode 2) covers the single layer only");
  ctx->op.cgr = cg_re;
  ctx->op.cgi = cg_im;
  ctx->op.chr = ch_re;
  ctx->op.chi = ch_im;
  ctx->op_version++;
  ctx->con.self64_ready = ctx->con.self32_ready = false;   // T's self entries change
  return BEM_OK;
}

bem_status bem_set_async(bem_ctx* ctx, int on) {
  if (!ctx) return BEM_EINVAL;
  ctx->async = on != 0;
  return BEM_OK;
}

bem_status bem_set_wait_limit(bem_ctx* ctx, uint32_t polls) {
  if (!ctx) return BEM_EINVAL;
  ctx->stage_wait_limit = polls;
  return BEM_OK;
}

bem_status bem_set_eval_split(bem_ctx* ctx, int poly_points) {
  if (!ctx || poly_points < -1 || poly_points > 4)
    return fail(ctx, BEM_EINVAL, "bem_set_eval_split: poly_points must be -1 or 0..4");
  ctx->poly_points = poly_points;
  return BEM_OK;
}

bem_status bem_set_twin_clusters(bem_ctx* ctx, int on) {
  if (!ctx || (on != 0 && on != 1))
    return fail(ctx, BEM_EINVAL, "bem_set_twin_clusters: on must be 0 or 1");
  ctx->twin_clusters = on;
  return BEM_OK;
}

bem_status bem_mixed_shape(const bem_ctx* ctx, int* nodes_per_unit, int* paired, int* splits,
                           int64_t* ctas) {
  if (!ctx) return BEM_EINVAL;
  if (nodes_per_unit) *nodes_per_unit = ctx->last_mixed_G;
  if (paired) *paired = ctx->last_mixed_pair;
  if (splits) *splits = ctx->last_mixed_S;
  if (ctas) *ctas = ctx->last_mixed_ctas;
  return BEM_OK;
}

bem_status bem_set_refine_residual(bem_ctx* ctx, int arith) {
  if (!ctx || (arith != 0 && arith != 1))
    return fail(ctx, BEM_EINVAL, "bem_set_refine_residual: arith must be 0 (FP64) or 1");
  ctx->final_residual_arith = arith;
  return BEM_OK;
}

bem_status bem_check(bem_ctx* ctx, void* stream) {
  if (!ctx) return BEM_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  bem_status st = cuda_check(ctx, cudaGetLastError(), "bem_check");
  if (st != BEM_OK) return st;
  return take_status(ctx, s, "bem_check");
}

bem_status bem_set_mesh(bem_ctx* ctx, int64_t nv, const double* xyz_host, int64_t nt,
                        const int32_t* tri_host, void* stream) {
  if (!ctx) return BEM_EINVAL;
  if (!xyz_host || !tri_host || nv < 3 || nt < 1 || nt > (int64_t)1 << 26)
    return fail(ctx, BEM_EINVAL, "bem_set_mesh: need nv >= 3, 1 <= nt <= 2^26 and non-null arrays");
  for (int64_t t = 0; t < 3 * nv; ++t)
    if (!isfinite(xyz_host[t])) return fail(ctx, BEM_EINVAL, "bem_set_mesh: non-finite vertex coordinate");
  // validation on the host (the geometry kernel repeats it into the status word): indices in
  // range, and no triangle whose area is below 1e-12 of its squared longest edge
  for (int64_t l = 0; l < nt; ++l) {
    const int32_t* t3 = tri_host + 3 * l;
    for (int e = 0; e < 3; ++e)
      if (t3[e] < 0 || t3[e] >= nv)
        return fail(ctx, BEM_EINVAL, "bem_set_mesh: vertex-index-out-of-range");
    const double* v0 = xyz_host + 3 * (int64_t)t3[0];
    const double* v1 = xyz_host + 3 * (int64_t)t3[1];
    const double* v2 = xyz_host + 3 * (int64_t)t3[2];
    const double e1[3] = {v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2]};
    const double e2[3] = {v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2]};
    const double e3[3] = {v2[0] - v1[0], v2[1] - v1[1], v2[2] - v1[2]};
    const double nx = e1[1] * e2[2] - e1[2] * e2[1];
    const double ny = e1[2] * e2[0] - e1[0] * e2[2];
    const double nz = e1[0] * e2[1] - e1[1] * e2[0];
    const double area = 0.5 * sqrt(nx * nx + ny * ny + nz * nz);
    const double l2 = fmax(fmax(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2],
                                e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]),
                           e3[0] * e3[0] + e3[1] * e3[1] + e3[2] * e3[2]);
    if (!(area > 1e-12 * l2) || !isfinite(area))
      return fail(ctx, BEM_EINVAL, "bem_set_mesh: zero-area-triangle");
  }
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  ctx->con.N = 0;   // self terms depend on the mesh: the contour must be set again
  Geometry& g = ctx->geo;
  if (nt > g.cap_n || nv > g.cap_nv) {   // buffers only grow; same-size meshes reuse them
    free_geometry(g);
    bool ok = cudaMalloc(&g.xyz, 3 * nv * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&g.tri, 3 * nt * sizeof(int32_t)) == cudaSuccess &&
              cudaMalloc(&g.cx, 3 * nt * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&g.qp, 21 * nt * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&g.qw, 7 * nt * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&g.cx32, 3 * nt * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&g.qp32, 21 * nt * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&g.qw32, 7 * nt * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&g.edge32, 9 * nt * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&g.mom32, kSelfMoments * nt * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&g.rho32, nt * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&g.diam, nt * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&g.nrm, 3 * nt * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&g.pack32, (nt + 15) / 16 * 16 * 64 * sizeof(float)) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      free_geometry(g);
      return fail(ctx, BEM_ENOMEM, "bem_set_mesh: device allocation failed");
    }
    g.cap_n = nt;
    g.cap_nv = nv;
  }
  // the kernels index the q-major arrays with the current n, so n must equal the capacity
  // they were laid out for: re-layout by reallocating when a smaller mesh follows a larger
  if (nt != g.cap_n) {
    free_geometry(g);
    return bem_set_mesh(ctx, nv, xyz_host, nt, tri_host, stream);
  }
  g.n = nt;
  g.nv = nv;
  ctx->h_xyz.assign(xyz_host, xyz_host + 3 * nv);
  ctx->h_tri.assign(tri_host, tri_host + 3 * nt);
  // asynchronous upload through the pinned staging buffer
  const size_t xb = 3 * nv * sizeof(double), tb = 3 * nt * sizeof(int32_t);
  bem_status st = stage_buffer(ctx, ctx->h_mesh, ctx->h_mesh_bytes, ctx->mesh_ev, xb + tb);
  if (st != BEM_OK) return st;
  unsigned char* hb = reinterpret_cast<unsigned char*>(ctx->h_mesh);
  memcpy(hb, xyz_host, xb);
  memcpy(hb + xb, tri_host, tb);
  st = cuda_check(ctx, cudaMemcpyAsync(g.xyz, hb, xb, cudaMemcpyHostToDevice, s), "bem_set_mesh copy");
  if (st == BEM_OK)
    st = cuda_check(ctx, cudaMemcpyAsync(g.tri, hb + xb, tb, cudaMemcpyHostToDevice, s),
                    "bem_set_mesh copy");
  if (st == BEM_OK) st = cuda_check(ctx, cudaEventRecord(ctx->mesh_ev, s), "bem_set_mesh event");
  if (st == BEM_OK) st = cuda_check(ctx, launch_geometry(ctx, s), "geometry kernel");
  if (st != BEM_OK) {
    free_geometry(g);
    return st;
  }
  ctx->mesh_version++;
  return BEM_OK;
}

bem_status bem_set_contour(bem_ctx* ctx, int kind, double c_re, double c_im, double a,
                           double b, int N, double* z_host, double* w_host, void* stream) {
  if (!ctx) return BEM_EINVAL;
  if (ctx->geo.n == 0) return fail(ctx, BEM_ESTATE, "bem_set_contour: no mesh set");
  if (kind != BEM_CONTOUR_CIRCLE && kind != BEM_CONTOUR_ELLIPSE && kind != BEM_CONTOUR_CHEBYSHEV)
    return fail(ctx, BEM_EINVAL, "bem_set_contour: unknown contour kind");
  if (kind == BEM_CONTOUR_CIRCLE || kind == BEM_CONTOUR_CHEBYSHEV) b = a;
  if (!(a > 0.0) || !(b > 0.0) || !isfinite(a) || !isfinite(b) || !isfinite(c_re) ||
      !isfinite(c_im))
    return fail(ctx, BEM_EINVAL, "bem_set_contour: semi-axes must be positive and finite");
  if (N < 1 || N > kMaxNodes) return fail(ctx, BEM_EINVAL, "bem_set_contour: N out of [1, 4096]");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  Contour& c = ctx->con;
  const int64_t need_self = ctx->geo.n * (int64_t)N;
  if (N > c.cap_N || need_self > c.cap_self) {
    free_contour(c);
    bool ok = cudaMalloc(&c.z, 2 * N * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&c.w, 2 * N * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&c.self, 2 * need_self * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&c.self32, 2 * need_self * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&c.order, N * sizeof(int)) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      free_contour(c);
      return fail(ctx, BEM_ENOMEM, "bem_set_contour: device allocation failed");
    }
    c.cap_N = N;
    c.cap_self = need_self;
  }
  c.N = N; c.kind = kind; c.c_re = c_re; c.c_im = c_im; c.a = a; c.b = b;
  c.self64_ready = c.self32_ready = false;   // filled by the first projection that needs them
  // nodes, weights and node schedule on the host; asynchronous upload through the pinned
  // staging buffer
  contour_nodes(kind, c_re, c_im, a, b, N, c.z_host, c.w_host);
  build_node_order(c);
  const size_t zb = 2 * N * sizeof(double), ob = N * sizeof(int);
  bem_status st = stage_buffer(ctx, ctx->h_con, ctx->h_con_bytes, ctx->con_ev, 2 * zb + ob);
  if (st != BEM_OK) {
    free_contour(c);
    return st;
  }
  unsigned char* hb = reinterpret_cast<unsigned char*>(ctx->h_con);
  memcpy(hb, c.z_host, zb);
  memcpy(hb + zb, c.w_host, zb);
  memcpy(hb + 2 * zb, c.order_host, ob);
  st = cuda_check(ctx, cudaMemcpyAsync(c.z, hb, zb, cudaMemcpyHostToDevice, s), "contour copy");
  if (st == BEM_OK)
    st = cuda_check(ctx, cudaMemcpyAsync(c.w, hb + zb, zb, cudaMemcpyHostToDevice, s), "contour copy");
  if (st == BEM_OK)
    st = cuda_check(ctx, cudaMemcpyAsync(c.order, hb + 2 * zb, ob, cudaMemcpyHostToDevice, s),
                    "node order copy");
  if (st == BEM_OK) st = cuda_check(ctx, cudaEventRecord(ctx->con_ev, s), "contour event");
  if (st != BEM_OK) {
    free_contour(c);
    return st;
  }
  ctx->contour_version++;
  for (int t = 0; t < 2 * N; ++t) {
    if (z_host) z_host[t] = c.z_host[t];
    if (w_host) w_host[t] = c.w_host[t];
  }
  return BEM_OK;
}

bem_status bem_node_order(const bem_ctx* ctx, int* order_host, int* twins) {
  if (!ctx) return BEM_EINVAL;
  if (ctx->con.N == 0) return BEM_ESTATE;
  if (order_host)
    for (int t = 0; t < ctx->con.N; ++t) order_host[t] = ctx->con.order_host[t] & kNodeMask;
  if (twins) *twins = ctx->con.twins;
  return BEM_OK;
}

bem_status bem_project(bem_ctx* ctx, const double* V_dev, int64_t ldv, int nu,
                       double* Bhat_dev, double* AV_dev, int precision, void* stream) {
  if (!ctx) return BEM_EINVAL;
  if (ctx->geo.n == 0) return fail(ctx, BEM_ESTATE, "bem_project: no mesh set");
  if (ctx->con.N == 0) return fail(ctx, BEM_ESTATE, "bem_project: no contour set");
  const int64_t n = ctx->geo.n;
  if (!V_dev || !Bhat_dev || nu < 1 || nu > kMaxNu || ldv < n)
    return fail(ctx, BEM_EINVAL, "bem_project: need V and Bhat, 1 <= nu <= 256, ldv >= n");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int N = ctx->con.N;
  if (precision != BEM_PREC_MIXED && precision != BEM_PREC_FP64 && precision != BEM_PREC_HMATRIX)
    return fail(ctx, BEM_EINVAL, "bem_project: unknown precision");
  bem_status st0 = ensure_near(ctx, s);
  if (st0 != BEM_OK) return st0;
  if (precision == BEM_PREC_MIXED) return project_mixed(ctx, V_dev, ldv, nu, Bhat_dev, AV_dev, s);
  if (precision == BEM_PREC_HMATRIX)
    return project_hmatrix(ctx, V_dev, ldv, nu, Bhat_dev, AV_dev, s);
  st0 = ensure_self64(ctx, s);
  if (st0 != BEM_OK) return st0;
  double* Y = AV_dev;
  if (!Y) {
    bem_status st = ensure_scratch(ctx, (size_t)N * n * nu * 2 * sizeof(double));
    if (st != BEM_OK) return st;
    Y = ctx->d_scratch;
  }
  timing_begin(ctx, s);
  bem_status st = cuda_check(ctx, launch_apply_fp64(ctx, V_dev, ldv, nu, Y, s), "apply kernel");
  timing_end(ctx, s);
  if (st != BEM_OK) return st;
  if (near_active(ctx)) {
    st = near_apply64(ctx, V_dev, ldv, nu, Y, s);
    if (st != BEM_OK) return st;
  }
  return cuda_check(ctx, launch_xhy_fp64(ctx, V_dev, ldv, nu, Y, n, n * nu, nu, n, N, ctx->con.w,
                                         Bhat_dev, s),
                    "projection kernel");
}

}  // extern "C"
