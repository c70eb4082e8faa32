// Context state: statistics, and a checkpoint of everything that defines the operator and
// the contour (mesh, contour, near-field mode, surrogate network) for resuming elsewhere.
//
// Checkpoint layout (little-endian host bytes): the 8-byte tag "BEMSTAT2", then int64 nv,
// int64 nt, int64 N, int64 contour kind, int64 near-field mode, int64 network floats (0 or
// the network size), double c_re, c_im, a, b, double c_G (re, im), c_H (re, im) of the
// operator; then xyz (3 nv doubles), tri (3 nt int32), the network's master parameters
// (floats). States written before the operator existed ("BEMSTAT1": the same without the
// operator's four doubles) load as the single layer. Workspaces, self-term tables, pair
// lists and timing records are rebuilt, not stored.
#include <string.h>

#include <vector>

#include "internal.h"
#include "surrogate.cuh"

using namespace bem;

namespace {

constexpr char kTag[8] = {'B', 'E', 'M', 'S', 'T', 'A', 'T', '2'};
constexpr char kTag1[8] = {'B', 'E', 'M', 'S', 'T', 'A', 'T', '1'};

struct Header1 {
  char tag[8];
  int64_t nv, nt, N, kind, near_mode, net_floats;
  double c_re, c_im, a, b;
};
struct Header {
  char tag[8];
  int64_t nv, nt, N, kind, near_mode, net_floats;
  double c_re, c_im, a, b;
  double op[4];   // c_G (re, im), c_H (re, im)
};

}  // namespace

extern "C" {

bem_status bem_stats(const bem_ctx* ctx, bem_stats_t* out) {
  if (!ctx || !out) return BEM_EINVAL;
  out->device = ctx->device;
  out->n = ctx->geo.n;
  out->nv = ctx->geo.nv;
  out->N = ctx->con.N;
  out->near_mode = ctx->near_mode;
  out->near_pairs = near_active(ctx) ? ctx->near_nnz : -1;
  out->launches = ctx->launches;
  out->workspace_bytes = (int64_t)(ctx->scratch_bytes + ctx->small_bytes + ctx->solve_bytes +
                                   ctx->near_work_bytes);
  out->surrogate_ready = ctx->net_ready ? 1 : 0;
  return BEM_OK;
}

bem_status bem_save_state(bem_ctx* ctx, void* buf, size_t* len, void* stream) {
  if (!ctx || !len) return BEM_EINVAL;
  if (ctx->geo.n == 0) return fail(ctx, BEM_ESTATE, "bem_save_state: no mesh set");
  const int64_t nv = ctx->geo.nv, nt = ctx->geo.n;
  const int64_t nf = ctx->net_ready ? kNetFloats : 0;
  const size_t need = sizeof(Header) + (size_t)3 * nv * sizeof(double) +
                      (size_t)3 * nt * sizeof(int32_t) + (size_t)nf * sizeof(float);
  if (!buf) {
    *len = need;
    return BEM_OK;
  }
  if (*len < need) {
    *len = need;
    return fail(ctx, BEM_EINVAL, "bem_save_state: buffer too small (*len set to the size)");
  }
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  Header h;
  memcpy(h.tag, kTag, 8);
  h.nv = nv;
  h.nt = nt;
  h.N = ctx->con.N;
  h.kind = ctx->con.kind;
  h.near_mode = ctx->near_mode;
  h.net_floats = nf;
  h.c_re = ctx->con.c_re;
  h.c_im = ctx->con.c_im;
  h.a = ctx->con.a;
  h.b = ctx->con.b;
  h.op[0] = ctx->op.cgr;
  h.op[1] = ctx->op.cgi;
  h.op[2] = ctx->op.chr;
  h.op[3] = ctx->op.chi;
  unsigned char* p = static_cast<unsigned char*>(buf);
  memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  bem_status st = cuda_check(ctx, cudaMemcpyAsync(p, ctx->geo.xyz, 3 * nv * sizeof(double),
                                                  cudaMemcpyDeviceToHost, s), "bem_save_state");
  p += 3 * nv * sizeof(double);
  if (st == BEM_OK)
    st = cuda_check(ctx, cudaMemcpyAsync(p, ctx->geo.tri, 3 * nt * sizeof(int32_t),
                                         cudaMemcpyDeviceToHost, s), "bem_save_state");
  p += 3 * nt * sizeof(int32_t);
  if (st == BEM_OK && nf)
    st = cuda_check(ctx, cudaMemcpyAsync(p, ctx->d_net, nf * sizeof(float), cudaMemcpyDeviceToHost, s),
                    "bem_save_state");
  if (st == BEM_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), "bem_save_state");
  if (st == BEM_OK) *len = need;
  return st;
}

bem_status bem_load_state(bem_ctx* ctx, const void* buf, size_t len, void* stream) {
  if (!ctx) return BEM_EINVAL;
  if (!buf || len < sizeof(Header1)) return fail(ctx, BEM_EINVAL, "bem_load_state: truncated state");
  Header h;
  size_t hsize = sizeof(Header);
  if (memcmp(buf, kTag1, 8) == 0) {   // written before the operator existed: single layer
    Header1 h1;
    memcpy(&h1, buf, sizeof(h1));
    memcpy(&h, &h1, sizeof(h1));
    h.op[0] = 1.0;
    h.op[1] = h.op[2] = h.op[3] = 0.0;
    hsize = sizeof(Header1);
  } else {
    if (len < sizeof(Header)) return fail(ctx, BEM_EINVAL, "bem_load_state: truncated state");
    memcpy(&h, buf, sizeof(h));
    if (memcmp(h.tag, kTag, 8) != 0) return fail(ctx, BEM_EINVAL, "bem_load_state: not a saved state");
  }
  if (h.nv < 3 || h.nt < 1 || h.nv > (int64_t)1 << 31 || h.nt > (int64_t)1 << 31 || h.N < 0 ||
      h.N > kMaxNodes || h.near_mode < 0 || h.near_mode > 2 ||
      (h.net_floats != 0 && h.net_floats != kNetFloats))
    return fail(ctx, BEM_EINVAL, "bem_load_state: corrupt header");
  const size_t need = hsize + (size_t)3 * h.nv * sizeof(double) +
                      (size_t)3 * h.nt * sizeof(int32_t) + (size_t)h.net_floats * sizeof(float);
  if (len < need) return fail(ctx, BEM_EINVAL, "bem_load_state: truncated state");
  const unsigned char* p = static_cast<const unsigned char*>(buf) + hsize;
  std::vector<double> xyz(3 * h.nv);
  std::vector<int32_t> tri(3 * h.nt);
  memcpy(xyz.data(), p, xyz.size() * sizeof(double));
  p += xyz.size() * sizeof(double);
  memcpy(tri.data(), p, tri.size() * sizeof(int32_t));
  p += tri.size() * sizeof(int32_t);
  // the mesh first (this clears the contour), then the network, contour and near field
  bem_status st = bem_set_mesh(ctx, h.nv, xyz.data(), h.nt, tri.data(), stream);
  if (st != BEM_OK) return st;
  if (ctx->near_mode == 2) {   // mode 2 would refuse a double-layer operator: reset it first
    st = bem_set_near_field(ctx, 0, stream);
    if (st != BEM_OK) return st;
  }
  st = bem_set_operator(ctx, h.op[0], h.op[1], h.op[2], h.op[3]);
  if (st != BEM_OK) return st;
  if (h.net_floats) {
    std::vector<float> net(h.net_floats);
    memcpy(net.data(), p, net.size() * sizeof(float));
    st = bem_surrogate_set(ctx, net.data(), h.net_floats, stream);
    if (st != BEM_OK) return st;
  }
  if (h.N > 0) {
    st = bem_set_contour(ctx, (int)h.kind, h.c_re, h.c_im, h.a, h.b, (int)h.N, nullptr, nullptr,
                         stream);
    if (st != BEM_OK) return st;
  }
  return bem_set_near_field(ctx, (int)h.near_mode, stream);
}

}  // extern "C"
