// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "bem_gb300.h"
#include "operator.cuh"

namespace bem {

// Maximum sizes the kernels are written for.
constexpr int kMaxNu = 256;
constexpr int kMaxNodes = 4096;
// Launches of the projection's main kernel whose duration is kept when timing is on.
constexpr int kMaxTimed = 256;
// Contour nodes the dense / matrix-free FP32 solver kernels accept.
constexpr int kMaxNodesSolve = 64;

// Terms kept of the Taylor expansion of the FP32 self term in i k rho.
constexpr int kSelfMoments = 24;

// Bits of the device status word.
enum : int {
  kStatusBadIndex = 1,     // a triangle references a vertex out of range
  kStatusZeroArea = 2,     // a triangle of zero area
  kStatusNotSPD = 4,       // a Gram matrix that is not numerically positive definite
  kStatusNonFinite = 8,    // a non-finite value where a finite one is required
  kStatusTimeout = 16,     // a bounded device wait gave up (the kernel aborted cleanly)
};
// polls (with 64 ns sleeps after the first 64: about a second) of a bounded device wait
constexpr uint32_t kStageWaitDefault = 1u << 24;


// Device geometry, structure-of-arrays, FP64 (plain path) and FP32 (mixed path).
// Quadrature arrays are q-major: element (q, l) at q * n + l, so that consecutive
// panels are consecutive in memory.
struct Geometry {
  int64_t n = 0;           // triangles = unknowns
  int64_t nv = 0;          // vertices
  int64_t cap_n = 0;       // allocated sizes (buffers are reused by same-size meshes)
  int64_t cap_nv = 0;
  double* xyz = nullptr;   // 3 nv
  int32_t* tri = nullptr;  // 3 n
  double* cx = nullptr;    // centroids, 3 n: x[0..n), y[n..2n), z[2n..3n)
  double* qp = nullptr;    // 21 n: x of point q at q*n + l, y at (7+q)*n + l, z at (14+q)*n + l
  double* qw = nullptr;    // 7 n: W_lq / (4 pi) at q*n + l
  float* cx32 = nullptr;   // FP32 copies of the above for the mixed path
  float* qp32 = nullptr;
  float* qw32 = nullptr;
  float* edge32 = nullptr; // 9 n, optional: self-term edge data (d, u_p, u_q per edge) at
                           // (3 e + f) * n + l, for the FP32 self terms of the mixed path
  double* diam = nullptr;  // optional, n: panel diameter (longest edge), FP64
  float* mom32 = nullptr;  // optional, kSelfMoments * n: moments of the FP32 self term at
                           // m * n + l (see self_moments32_kernel)
  float* rho32 = nullptr;  // optional, n: largest centroid-to-vertex distance of panel l
  float* pack32 = nullptr; // optional, 64 floats per panel, rows padded to a multiple of 16
                           // panels: 7 x (x_hi, y_hi, z_hi, w) then 7 x (x_lo, y_lo, z_lo, 0)
                           // (hi + lo = the FP64 quadrature point; w = W_lq / 4 pi), then the
                           // unit normal (nx, ny, nz) at 56..58
  double* nrm = nullptr;   // optional, 3 n: unit normal of panel l (vertex order) at c * n + l
};

struct Contour {
  int N = 0;
  int kind = 0;
  double c_re = 0, c_im = 0, a = 0, b = 0;
  double* z = nullptr;     // 2 N, device
  double* w = nullptr;     // 2 N, device
  double* self = nullptr;  // 2 n N, device: A_ll(z_j) at j * n + l (complex)
  float* self32 = nullptr; // 2 n N, device: the same in FP32 (mixed path)
  bool self64_ready = false;   // tables are filled on first use after bem_set_contour
  bool self32_ready = false;
  int cap_N = 0;           // allocated sizes
  int64_t cap_self = 0;
  double z_host[2 * kMaxNodes];
  double w_host[2 * kMaxNodes];
  // Node schedule of the mixed evaluation: slot -> node, twin nodes (equal FP32 real parts,
  // which share their sine and cosine) at slots 2 P, 2 P + 1 with kTwinBit on slot 2 P.
  int* order = nullptr;    // N, device
  int order_host[kMaxNodes];
  int twins = 0;           // twin pairs in the schedule
};
constexpr int kTwinBit = 1 << 30;
constexpr int kNodeMask = kTwinBit - 1;

}  // namespace bem

namespace bem {
struct HMatrix;   // low-rank far field (hmatrix.cu)
}  // namespace bem

struct bem_ctx {
  int device = 0;
  std::string err;
  bem::Geometry geo;
  bem::Contour con;
  int* d_status = nullptr;       // device status word
  double* d_scratch = nullptr;   // reusable FP64 workspace
  size_t scratch_bytes = 0;
  double* d_small = nullptr;     // small FP64 workspace (Gram / Cholesky / norms)
  void* cublas = nullptr;        // cuBLAS handle of the dense LU's trailing updates (lazy)
  float* d_piv_val = nullptr;    // LU pivot search: per-block partial maxima and their rows
  int* d_piv_idx = nullptr;
  double* d_zgemm = nullptr;     // split-k partial products of the small complex GEMMs
  size_t zgemm_bytes = 0;
  float* d_lu_work = nullptr;    // the LU's trailing-update operands in real form
  size_t lu_work_bytes = 0;
  size_t small_bytes = 0;
  int64_t launches = 0;
  int64_t mesh_version = 0;         // bumped by every successful bem_set_mesh
  int64_t contour_version = 0;      // bumped by every successful bem_set_contour
  // buffers of bem_solve (grown on demand, owned by the context)
  double* d_solve = nullptr;
  size_t solve_bytes = 0;
  bool timing = false;              // record events around the main projection kernel
  std::vector<cudaEvent_t> ev;      // 2 * kMaxTimed events (start, stop)
  int n_timed = 0;
  // near field: mode (0 off, 1 64-point rule, 2 surrogate network) and the pair list (CSR)
  int near_mode = 0;
  int64_t near_mesh_version = -1;   // mesh the list was built for
  int64_t near_nnz = 0;
  int32_t* d_near_ptr = nullptr;    // n + 1
  int32_t* d_near_cols = nullptr;   // nnz
  int64_t near_cap_n = 0, near_cap_nnz = 0;
  unsigned long long* d_sur_usage = nullptr;   // (network, plain rule) samples since the last read
  void* d_near_work = nullptr;      // row-major copy of the basis for the near products
  size_t near_work_bytes = 0;
  // surrogate network of the near field (weights on the device, see surrogate.cu)
  float* d_net = nullptr;
  int64_t net_floats = 0;
  bool net_ready = false;
  // pinned host staging of the mesh and contour uploads (asynchronous copies); a buffer is
  // rewritten only after the event recorded behind its last copy has completed
  void* h_mesh = nullptr;
  size_t h_mesh_bytes = 0;
  cudaEvent_t mesh_ev = nullptr;
  void* h_con = nullptr;
  size_t h_con_bytes = 0;
  cudaEvent_t con_ev = nullptr;
  // asynchronous mode: bem_cholqr2 does not wait for its status word (bem_check reports it)
  bool async = false;
  // polls of each pipeline-stage wait of the fused projection kernel before it gives up
  // (bem_set_wait_limit); the drains before a block releases its memory keep the full bound
  uint32_t stage_wait_limit = bem::kStageWaitDefault;
  // quadrature points per entry whose sine and cosine the fused kernel takes from the FMA-
  // pipe polynomials (bem_set_eval_split); -1: the measured default of the unit shape
  int poly_points = -1;
  // twin pairs on two-CTA clusters when a unit holds one node (bem_set_twin_clusters)
  int twin_clusters = 1;
  // work decomposition of the last mixed projection (bem_mixed_shape)
  int last_mixed_G = 0, last_mixed_pair = 0, last_mixed_S = 0;
  int64_t last_mixed_ctas = 0;
  // arithmetic of the residuals bem_refine (and bem_solve) report: 0 FP64, 1 double-FP32
  int final_residual_arith = 0;
  // the boundary operator T = c_G G + c_H (1/2 I + K) (single layer by default)
  bem::OpCoef op;
  int64_t op_version = 0;   // bumped by every bem_set_operator
  // host copy of the mesh (the cluster tree of the low-rank far field is built from it)
  std::vector<double> h_xyz;
  std::vector<int32_t> h_tri;
  // low-rank far field (hmatrix.cu); null until bem_set_hmatrix
  bem::HMatrix* hm = nullptr;
};

namespace bem {

// Set the context's error message and return `st`.
bem_status fail(bem_ctx* ctx, bem_status st, const std::string& msg);
// Map a CUDA error to BEM_ECUDA with a message; BEM_OK if `e` is cudaSuccess.
bem_status cuda_check(bem_ctx* ctx, cudaError_t e, const char* what);
// Make sure the context's scratch holds at least `bytes`.
bem_status ensure_scratch(bem_ctx* ctx, size_t bytes);
bem_status ensure_small(bem_ctx* ctx, size_t bytes);
void release_cublas(bem_ctx* ctx);
// nodes z and weights w (2 N doubles each, interleaved) of a contour, on the host
void contour_nodes(int kind, double c_re, double c_im, double a, double b, int N, double* z,
                   double* w);
// Events around the main kernel of a projection (no-ops unless timing is enabled).
inline void timing_begin(bem_ctx* ctx, cudaStream_t s) {
  if (ctx->timing && ctx->n_timed < kMaxTimed) cudaEventRecord(ctx->ev[2 * ctx->n_timed], s);
}
inline void timing_end(bem_ctx* ctx, cudaStream_t s) {
  if (ctx->timing && ctx->n_timed < kMaxTimed) cudaEventRecord(ctx->ev[2 * ctx->n_timed++ + 1], s);
}
// Read and clear the device status word (synchronises `stream`).
bem_status take_status(bem_ctx* ctx, cudaStream_t stream, const char* where);

// Kernel launchers (each returns the launch error, if any).
cudaError_t launch_geometry(bem_ctx* ctx, cudaStream_t s);
cudaError_t launch_contour(bem_ctx* ctx, cudaStream_t s);
cudaError_t launch_self_terms(bem_ctx* ctx, cudaStream_t s);
cudaError_t launch_self_terms32(bem_ctx* ctx, cudaStream_t s);
// FP32 self terms of the mesh at nk wavenumbers kz (device, complex) into out (nk x n).
cudaError_t launch_self32(bem_ctx* ctx, int nk, const double* kz, float* out, cudaStream_t s);
// R[:, c] = A(lam_c) X[:, c] (deriv: A'(lam_c) X[:, c]), FP64, matrix-free (residual.cu);
// R has leading dimension n. lam_dev: m complex on the device.
cudaError_t launch_apply_percol64(bem_ctx* ctx, int m, const double* lam_dev, const double* X,
                                  int64_t ldx, double* R, bool deriv, cudaStream_t s);
// R = A(lambda_c) x_c and, if Rd, Rd = A'(lambda_c) x_c in double-FP32 arithmetic (entries
// to ~1e-13; single layer; the general operator uses the FP64 kernels), near field added
cudaError_t launch_apply_ff(bem_ctx* ctx, int m, const double* lam_dev, const double* X,
                            int64_t ldx, double* R, double* Rd, cudaStream_t s);
// R_c[i] = the self entry of T(lambda_c) (or of its k-derivative)
cudaError_t launch_self_at(bem_ctx* ctx, int m, const double* lam_dev, double* R, bool deriv,
                           cudaStream_t s);
// out[2c] = ||R[:, c]||^2, out[2c+1] = ||X[:, c]||^2 (fixed-order sums)
cudaError_t launch_colnorms(bem_ctx* ctx, const double* R, int64_t ldr, const double* X,
                            int64_t ldx, int64_t n, int m, double* out, cudaStream_t s);
// dense FP32 operator and LU (dense32.cu)
bem_status assemble32(bem_ctx* ctx, int nk, const double* kz_host, const double* coef_host,
                      float2* M, cudaStream_t s);
bem_status lu32(bem_ctx* ctx, float2* A, int64_t n, int* ipiv, cudaStream_t s);
bem_status lu32_solve(bem_ctx* ctx, const float2* LU, const int* ipiv, int64_t n, float2* B,
                      int64_t m, cudaStream_t s);
cudaError_t launch_zgemm(bem_ctx* ctx, int m, int n, int k, const double* A, int64_t lda,
                         const double* B, int64_t ldb, double* C, int64_t ldc, cudaStream_t s);
// Fill the FP64 / FP32 self-term table of the current contour if not done yet.
bem_status ensure_self64(bem_ctx* ctx, cudaStream_t s);
bem_status ensure_self32(bem_ctx* ctx, cudaStream_t s);
// Y_j = A(z_j) V for all nodes (FP64), Y node-major with leading dimension n.
cudaError_t launch_apply_fp64(bem_ctx* ctx, const double* V, int64_t ldv, int nu, double* Y,
                              cudaStream_t s);
// C_j = scale_j * X^H Y_j for a batch of nb right-hand blocks (FP64, deterministic).
// X: n x p (ldx), Y_j at Y + j * strideY (ldy), C_j at C + j * p * q (p x q, col-major).
// scale: nullptr (1) or 2 nb doubles (complex, device).
cudaError_t launch_xhy_fp64(bem_ctx* ctx, const double* X, int64_t ldx, int p, const double* Y,
                            int64_t ldy, int64_t strideY, int q, int64_t n, int nb,
                            const double* scale, double* C, cudaStream_t s);
// CholeskyQR2 with caller-provided work space (asynchronous; status word on failure).
// refresh_seed != 0: columns whose first-pass pivot collapses (rank deficiency) are
// replaced by pseudo-random columns before the second pass instead of failing; R is then
// not a factor of the input.
size_t cholqr2_work_bytes(bem_ctx* ctx, int64_t n, int nu);
bem_status cholqr2_impl(bem_ctx* ctx, double* V, int64_t n, int64_t ldv, int nu, double* R,
                        void* work, cudaStream_t s, uint64_t refresh_seed);
// Near field (near.cu). near_active: a mode is set and the pair list is current (build it
// with ensure_near first).
bem_status ensure_near(bem_ctx* ctx, cudaStream_t s);
inline bool near_active(const bem_ctx* ctx) {
  return ctx->near_mode != 0 && ctx->near_mesh_version == ctx->mesh_version;
}
// Y_j += (A_near - A_7)(z_j) V over the near pairs, FP64 (Y node-major, leading dim. n).
bem_status near_apply64(bem_ctx* ctx, const double* V, int64_t ldv, int nu, double* Y,
                        cudaStream_t s);
// The same correction in FP32 into slice `slice` of the mixed path's partial products
// (layout [slice][N][2 nup][n_pad], basis column b at (b / C) 2C + b % C, imaginary part C
// further); V32 is the FP32 copy of V (column-major, leading dimension n). Every row and
// column of the slice is written.
bem_status near_apply32(bem_ctx* ctx, const float2* V32, int nu, int nup, int C, int n_pad,
                        float* Yp, int slice, cudaStream_t s);
// R[:, c] += (A_near - A_7)(lam_c) X[:, c] (deriv: the k-derivatives), FP64.
cudaError_t launch_near_percol64(bem_ctx* ctx, int m, const double* lam_dev, const double* X,
                                 int64_t ldx, double* R, bool deriv, cudaStream_t s);
// Node-summed fused apply (tcgen05; project_mixed.cu): out = sum_j c_j A(z_j) X_j, X_j at
// X + j node_stride (per_node) or X itself, FP32 complex, column-major with leading dimension
// ldx; out n x nu (leading dimension n). work: mixed_sum_work_bytes(ctx, nu, per_node) bytes.
size_t mixed_sum_work_bytes(bem_ctx* ctx, int nu, bool per_node);
bem_status mixed_sum_apply(bem_ctx* ctx, const float2* X, int64_t ldx, int64_t node_stride,
                           bool per_node, int nu, const double* coef_host, float2* out,
                           void* work, cudaStream_t s);
// Restarted GMRES (gmres.cu) for (sum_j c_j A(z_j)) X = B, FP32 n x nu blocks (leading
// dimension n), every column at once; work: gmres_sum_work_bytes(ctx, nu, restart) bytes.
// relres_host (nu doubles, may be null): final true relative residuals.
size_t gmres_sum_work_bytes(bem_ctx* ctx, int nu, int restart);
bem_status gmres_sum32(bem_ctx* ctx, const double* coef_host, const float2* B, float2* X, int nu,
                       double tol, int max_iter, int restart, void* work, cudaStream_t s,
                       int* iters_out, double* relres_host);
// Products formed outside the fused kernel, finished by the mixed path (project_mixed.cu):
// Yp is slice 0 of the FP32 partials [slice][N][acc_cols][n_pad], basis column c's real part
// at column (c / C) 2 C + c % C, its imaginary part C further; every entry must be written.
struct ExtFrame {
  float* Yp = nullptr;
  int acc_cols = 0, C = 0, n_pad = 0;
  void* impl = nullptr;
};
bem_status external_begin(bem_ctx* ctx, const double* V, int64_t ldv, int nu, ExtFrame& f,
                          cudaStream_t s);
bem_status external_end(bem_ctx* ctx, ExtFrame& f, int nu, double* Bhat, double* AV,
                        cudaStream_t s);
void external_release(ExtFrame& f);   // on an error between begin and end
// Projection with the low-rank far field (hmatrix.cu); BEM_ESTATE without bem_set_hmatrix.
bem_status project_hmatrix(bem_ctx* ctx, const double* V, int64_t ldv, int nu, double* Bhat,
                           double* AV, cudaStream_t s);
void free_hmatrix(bem_ctx* ctx);
// mixed-precision fused projection (tcgen05); defined in project_mixed.cu
bem_status project_mixed(bem_ctx* ctx, const double* V, int64_t ldv, int nu, double* Bhat,
                         double* AV, cudaStream_t s);

}  // namespace bem
