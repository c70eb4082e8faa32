// Allocation-free variant of the plain FP64 projection.
//
// Some callers cannot call cudaMalloc: code that runs while a memory pool is locked, an
// embedding runtime that hands out device memory only through its own allocator, or a
// process that must not grow its device footprint after start-up. bem_project_fp64_noalloc
// serves them: it takes the mesh, the basis and the output already on the device and keeps
// every intermediate (geometry, contour nodes and weights, self terms, the status word and
// the A(z_j) V products) in one file-scope device array of fixed size, so neither it nor
// anything it calls allocates.
//
// The array is a __device__ symbol: in host code its name is only a host-side stand-in, so
// its device address is obtained with cudaGetSymbolAddress (with the device current) and
// that address is what the kernels receive. The lookup is repeated on every call, so a
// device whose primary context was reset and re-created in between gets the array's new
// address; it allocates nothing (the first lookup on a device may load the module, which
// is why the first call should come before any stream capture). Every GPU that loads this
// library holds the array until the process exits. The message of the last failure on the
// calling thread is kept for bem_noalloc_last_error.
// All calls share it and it keeps the last call's contents; calls whose work overlaps on
// the GPU (other streams, other host threads) race on it and must be serialised by the
// caller.
#include <math.h>

#include <algorithm>
#include <string>

#include "internal.h"

namespace bem {
namespace {

constexpr size_t kNoallocBytes = (size_t)64 << 20;   // 64 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

thread_local std::string g_last_error;   // message of the calling thread's last failure

bem_status noalloc_fail(bem_status st, const std::string& msg) {
  g_last_error = "bem_project_fp64_noalloc: " + msg;
  return st;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Bytes of the parts whose size does not depend on how many nodes share the Y buffer.
size_t fixed_bytes(int64_t n, int N) {
  return round256(sizeof(int)) + round256(31 * n * sizeof(double)) +
         round256(31 * n * sizeof(float)) + 2 * round256(2 * (size_t)N * sizeof(double)) +
         round256(2 * (size_t)n * N * sizeof(double));
}

}  // namespace
}  // namespace bem

using namespace bem;

extern "C" bem_status bem_project_fp64_noalloc(int device, int64_t nv, const double* xyz_dev,
                                               int64_t nt, const int32_t* tri_dev, int kind,
                                               double c_re, double c_im, double a, double b,
                                               int N, const double* V_dev, int64_t ldv, int nu,
                                               double* Bhat_dev, void* stream) {
  g_last_error.clear();
  if (!xyz_dev || !tri_dev || !V_dev || !Bhat_dev || nv < 3 || nt < 1 || nu < 1 ||
      nu > kMaxNu || ldv < nt || N < 1 || N > kMaxNodes || device < 0 || device >= kMaxDevices)
    return noalloc_fail(BEM_EINVAL, "bad argument (null pointer, size or device out of range)");
  if (kind != BEM_CONTOUR_CIRCLE && kind != BEM_CONTOUR_ELLIPSE)
    return noalloc_fail(BEM_EINVAL, "unknown contour kind");
  if (kind == BEM_CONTOUR_CIRCLE) b = a;
  if (!(a > 0.0) || !(b > 0.0) || !isfinite(a) || !isfinite(b) || !isfinite(c_re) ||
      !isfinite(c_im))
    return noalloc_fail(BEM_EINVAL, "contour centre and semi-axes must be finite, axes > 0");
  // size limit: the fixed parts plus the products of at least one node must fit
  const size_t fixed = fixed_bytes(nt, N);
  const size_t per_node = round256((size_t)2 * nt * nu * sizeof(double));
  if (fixed + per_node > kNoallocBytes)
    return noalloc_fail(BEM_EINVAL, "problem too large for the fixed " +
                                        std::to_string(kNoallocBytes >> 20) + " MiB array");

  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return noalloc_fail(BEM_ECUDA, "cudaGetDevice failed");
  if (cur != device && cudaSetDevice(device) != cudaSuccess)
    return noalloc_fail(BEM_ECUDA, "cudaSetDevice failed");
  void* base = nullptr;
  const cudaError_t ge = cudaGetSymbolAddress(&base, g_noalloc_scratch);
  if (ge != cudaSuccess || !base) {
    cudaGetLastError();
    if (cur != device) cudaSetDevice(cur);
    return noalloc_fail(BEM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(ge));
  }

  // carve the array: status | FP64 geometry | FP32 geometry | z | w | self | Y chunk
  unsigned char* p = static_cast<unsigned char*>(base);
  bem_ctx ctx;                 // a view onto the array; owns no device memory
  ctx.device = device;
  ctx.d_status = reinterpret_cast<int*>(p);
  p += round256(sizeof(int));
  Geometry& g = ctx.geo;
  g.n = nt;
  g.nv = nv;
  g.xyz = const_cast<double*>(xyz_dev);
  g.tri = const_cast<int32_t*>(tri_dev);
  g.cx = reinterpret_cast<double*>(p);
  g.qp = g.cx + 3 * nt;
  g.qw = g.qp + 21 * nt;
  p += round256(31 * nt * sizeof(double));
  g.cx32 = reinterpret_cast<float*>(p);
  g.qp32 = g.cx32 + 3 * nt;
  g.qw32 = g.qp32 + 21 * nt;
  p += round256(31 * nt * sizeof(float));
  Contour& c = ctx.con;
  c.N = N; c.kind = kind; c.c_re = c_re; c.c_im = c_im; c.a = a; c.b = b;
  c.z = reinterpret_cast<double*>(p);
  p += round256(2 * (size_t)N * sizeof(double));
  c.w = reinterpret_cast<double*>(p);
  p += round256(2 * (size_t)N * sizeof(double));
  c.self = reinterpret_cast<double*>(p);
  p += round256(2 * (size_t)nt * N * sizeof(double));
  double* Y = reinterpret_cast<double*>(p);
  const int chunk = (int)std::min<size_t>((size_t)N, (kNoallocBytes - fixed) / per_node);

  cudaStream_t s = (cudaStream_t)stream;
  bem_status st = BEM_OK;
  // the status word must start at zero; everything else is overwritten before it is read
  if (cudaMemsetAsync(ctx.d_status, 0, sizeof(int), s) != cudaSuccess) st = BEM_ECUDA;
  if (st == BEM_OK && launch_geometry(&ctx, s) != cudaSuccess) st = BEM_ECUDA;
  if (st == BEM_OK && launch_contour(&ctx, s) != cudaSuccess) st = BEM_ECUDA;
  if (st == BEM_OK) st = take_status(&ctx, s, "bem_project_fp64_noalloc");
  if (st == BEM_OK && launch_self_terms(&ctx, s) != cudaSuccess) st = BEM_ECUDA;
  // nodes in chunks that fit the array: Y for nodes [j0, j0 + nc), then their Bhat_j
  for (int j0 = 0; st == BEM_OK && j0 < N; j0 += chunk) {
    const int nc = std::min(chunk, N - j0);
    Contour sub = c;
    sub.N = nc;
    sub.z = c.z + 2 * j0;
    sub.w = c.w + 2 * j0;
    sub.self = c.self + 2 * (size_t)nt * j0;
    ctx.con = sub;
    if (launch_apply_fp64(&ctx, V_dev, ldv, nu, Y, s) != cudaSuccess ||
        launch_xhy_fp64(&ctx, V_dev, ldv, nu, Y, nt, nt * nu, nu, nt, nc, sub.w,
                        Bhat_dev + 2 * (size_t)nu * nu * j0, s) != cudaSuccess)
      st = BEM_ECUDA;
    ctx.con = c;
  }
  if (cur != device) cudaSetDevice(cur);
  if (st != BEM_OK)
    noalloc_fail(st, ctx.err.empty() ? std::string("CUDA error on a launch") : ctx.err);
  return st;
}

extern "C" const char* bem_noalloc_last_error(void) { return g_last_error.c_str(); }
