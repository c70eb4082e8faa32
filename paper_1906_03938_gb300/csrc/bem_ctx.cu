// Context, error handling, mesh and contour set-up, and the projection entry point.
#include <math.h>
#include <stdio.h>

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
  cudaFree(g.mom32); cudaFree(g.rho32); cudaFree(g.diam);
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
  cudaFree(ctx->d_solve);
  cudaFree(ctx->d_near_ptr);
  cudaFree(ctx->d_near_cols);
  cudaFree(ctx->d_near_work);
  cudaFree(ctx->d_net);
  for (auto& e : ctx->ev) cudaEventDestroy(e);
  delete ctx;
}

const char* bem_last_error(const bem_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

int64_t bem_kernel_launches(const bem_ctx* ctx) { return ctx ? ctx->launches : 0; }

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
  bem_status st = cuda_check(ctx, cudaMemcpyAsync(g.xyz, xyz_host, 3 * nv * sizeof(double),
                                                  cudaMemcpyHostToDevice, s), "bem_set_mesh copy");
  if (st == BEM_OK)
    st = cuda_check(ctx, cudaMemcpyAsync(g.tri, tri_host, 3 * nt * sizeof(int32_t),
                                         cudaMemcpyHostToDevice, s), "bem_set_mesh copy");
  if (st == BEM_OK) st = cuda_check(ctx, launch_geometry(ctx, s), "geometry kernel");
  if (st == BEM_OK) st = take_status(ctx, s, "bem_set_mesh");
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
  bem_status st = cuda_check(ctx, launch_contour(ctx, s), "contour kernel");
  if (st == BEM_OK)
    st = cuda_check(ctx, cudaMemcpyAsync(c.z_host, c.z, 2 * N * sizeof(double),
                                         cudaMemcpyDeviceToHost, s), "contour copy");
  if (st == BEM_OK)
    st = cuda_check(ctx, cudaMemcpyAsync(c.w_host, c.w, 2 * N * sizeof(double),
                                         cudaMemcpyDeviceToHost, s), "contour copy");
  if (st == BEM_OK) st = take_status(ctx, s, "bem_set_contour");
  if (st == BEM_OK) {
    build_node_order(c);
    st = cuda_check(ctx, cudaMemcpyAsync(c.order, c.order_host, N * sizeof(int),
                                         cudaMemcpyHostToDevice, s), "node order copy");
  }
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
  if (precision != BEM_PREC_MIXED && precision != BEM_PREC_FP64)
    return fail(ctx, BEM_EINVAL, "bem_project: unknown precision");
  bem_status st0 = ensure_near(ctx, s);
  if (st0 != BEM_OK) return st0;
  if (precision == BEM_PREC_MIXED) return project_mixed(ctx, V_dev, ldv, nu, Bhat_dev, AV_dev, s);
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
