/*
 * bem_gb300.h -- C ABI of the GB300 hot path of the Cauchy rational-approximation /
 * Rayleigh-Ritz method for the acoustic BEM nonlinear eigenvalue problem A(k) x = 0
 * (El-Guide, Miedlar, Saad, "A rational approximation method for solving acoustic
 * nonlinear eigenvalue problems").
 *
 * Operator. A(k) is the constant-element collocation matrix of the single-layer part of
 * the boundary integral equation (Section 1, Eq. HelmBIM, Eq. GreenFun): for triangles
 * i != l, A_il(k) = sum_q W_lq exp(i k r) / (4 pi r), r = |x_i - y_lq|, with x_i the
 * centroid of triangle i and (y_lq, W_lq) Radon's 7-point degree-5 rule on triangle l;
 * A_ii(k) is the exact integral of the kernel over triangle i, taken in polar
 * coordinates about x_i (radial part in closed form, angular part by 16-point
 * Gauss-Legendre in u = asinh(s/d) on each side of the foot of each edge).
 *
 * Conventions for every entry point:
 *  - Complex numbers are interleaved (re, im) doubles. Matrices are column-major.
 *  - "_dev" pointers are CUDA device pointers on the context's device; "_host" pointers
 *    are host memory. The caller owns every buffer it passes; the context owns only its
 *    internal workspaces (geometry, contour, self-term table, reduction partials).
 *  - Work is enqueued on the given stream (a cudaStream_t passed as void*, NULL = legacy
 *    default stream) and returns without synchronising unless stated otherwise.
 *  - Every call returns a bem_status; on failure bem_last_error() describes it. No C++
 *    exception crosses the ABI. There is no CPU fallback: a missing or failing GPU is an
 *    error (BEM_ECUDA).
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef BEM_GB300_H
#define BEM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bem_ctx bem_ctx;

typedef enum {
    BEM_OK = 0,
    BEM_EINVAL = -1,    /* invalid argument (null pointer, bad size, degenerate mesh) */
    BEM_ENOMEM = -2,    /* device workspace allocation failed */
    BEM_ECUDA = -3,     /* CUDA runtime error (launch failure, no device, ...) */
    BEM_EKERNEL = -4,   /* a kernel reported an error through its status word */
    BEM_ETIMEOUT = -5,  /* a bounded device wait ran out */
    BEM_ENOCONV = -6,   /* an iteration did not converge */
    BEM_ESTATE = -7     /* call out of order (no mesh / no contour set yet) */
} bem_status;

typedef enum {
    BEM_PREC_FP64 = 0,  /* plain path: FP64 evaluation and FP64 contraction */
    BEM_PREC_MIXED = 1, /* FP32 evaluation, BF16x3 split-precision tcgen05 contraction */
    BEM_PREC_HMATRIX = 2 /* low-rank far field (bem_set_hmatrix): FP32 entries and products */
} bem_precision;

typedef enum {
    BEM_CONTOUR_CIRCLE = 0,
    BEM_CONTOUR_ELLIPSE = 1,
    BEM_CONTOUR_CHEBYSHEV = 2   /* Chebyshev points of a real interval (Eq. Chebyshev) */
} bem_contour_kind;

/* Create a context on CUDA device `device`. */
bem_status bem_create(bem_ctx** out, int device);
void bem_destroy(bem_ctx* ctx);
/* Message of the last failing call on this context (never NULL). */
const char* bem_last_error(const bem_ctx* ctx);
/* Library version string. */
const char* bem_version(void);

/*
 * Geometry set-up (the mesh is the discretisation of Section 1; Eq. NEVPHelmholtz).
 * Copies nv vertices (xyz_host: 3*nv doubles, x y z per vertex) and nt triangles
 * (tri_host: 3*nt int32 vertex indices, outward orientation) to the device and computes
 * per-triangle centroids, areas and the 7 quadrature points and weights. n = nt is the
 * number of unknowns. Fails with BEM_EINVAL on an index out of range or a triangle of
 * zero area (area below 1e-12 of its squared longest edge), both checked on the host before
 * anything changes. The arrays are copied into a pinned staging buffer of the context and
 * uploaded asynchronously; the call returns without synchronising.
 */
bem_status bem_set_mesh(bem_ctx* ctx, int64_t nv, const double* xyz_host, int64_t nt,
                        const int32_t* tri_host, void* stream);

/*
 * Contour set-up (Section 2, Eq. Tz, Eq. TzApp). Trapezoid nodes in the angle,
 * theta_j = 2 pi (j + 1/2) / N, j = 0..N-1, on z(theta) = c + a cos(theta) + i b sin(theta)
 * (kind CIRCLE uses b = a):
 *     z_j = c + a cos(theta_j) + i b sin(theta_j),
 *     w_j = (b cos(theta_j) + i a sin(theta_j)) / N,
 * so that A(z) ~ sum_j w_j A(z_j) / (z_j - z) inside the contour. The self terms A_ii(z_j)
 * of the current mesh are evaluated by the first bem_project after this call (in the
 * precision that projection uses) and kept until the mesh or contour changes. z_host /
 * w_host (2*N doubles each) may
 * be NULL; if given they receive the nodes / weights. Requires a mesh. N in [1, 4096],
 * a > 0, b > 0. The nodes and weights are computed on the host (the lower half of the
 * nodes as the exact mirror of the upper, so conjugate nodes have equal real parts) and
 * uploaded asynchronously through a pinned staging buffer; no synchronisation.
 * Kind CHEBYSHEV (Section 2, Eq. Chebyshev): the Chebyshev points of the first kind of the
 * interval [c_re - a, c_re + a] shifted by i c_im, z_k = c + a cos(pi (k + 1/2) / N), and
 * unit weights (bem_project then returns the unweighted V^H A(z_k) V); b is ignored.
 */
bem_status bem_set_contour(bem_ctx* ctx, int kind, double c_re, double c_im, double a,
                           double b, int N, double* z_host, double* w_host, void* stream);

/*
 * The boundary operator (Section 1, Eq. HelmBIM in its general form T = A H - B G, with
 * constant coefficients): T(k) = c_G G(k) + c_H (1/2 I + K(k)), G the single layer
 * (Eq. GreenFun) and K the double layer with kernel
 *     dG/dn_y = exp(i k r) (i k r - 1) (y - x) . n_y / (4 pi r^3),
 * n_y the unit normal of the source triangle in its vertex order (outward for an outward
 * oriented mesh), collocated at centroids with the same 7-point rule; K vanishes on the
 * collocation point's own (flat) panel, whose entry is c_G A_ii + c_H / 2. (c_G, c_H) =
 * (1, 0), the default, is the single layer (Dirichlet conditions); (0, 1) the interior
 * Neumann problem with the boundary values as unknowns; both non-zero a Robin condition.
 * Every projection, residual, refinement, inverse power step and near-field correction
 * uses T from the next call on; the self terms are recomputed. The near-field surrogate
 * (mode 2) and the batched launch cover the single layer only (BEM_EINVAL). Host only.
 */
bem_status bem_set_operator(bem_ctx* ctx, double cg_re, double cg_im, double ch_re,
                            double ch_im);

/*
 * Low-rank far field (the H-matrix route of Section 4, Example 3, where the samples are
 * stored as H-matrices compressed by adaptive cross approximation; the paper does not give
 * its parameters). bem_set_hmatrix configures it; bem_project with precision
 * BEM_PREC_HMATRIX then forms B_j = w_j V^H T(z_j) V with T(z_j) replaced by its
 * H-matrix:
 *   cluster tree: panels split at the middle of their order along the longest axis of
 *     their centroids' box (ties by index) down to `leaf` panels (1..32); a cluster's
 *     geometry is the box of its panels' vertices;
 *   blocks from (root, root): far when max(diam) <= eta dist of the two boxes, dense when
 *     both clusters are leaves, else split into the children's pairs;
 *   far blocks: adaptive cross approximation with partial pivoting on FP32 entries, per
 *     node, to relative accuracy eps (stop at ||u_k|| ||w_k|| <= eps ||S_k||_F, at most
 *     rmax terms, 1..128); dense blocks evaluated in FP32; products in FP32; then the
 *     mixed path's finish: FP32 near-field corrections (bem_set_near_field) and
 *     B_j = w_j V^H Y_j (BF16x3 tensor-core contraction for nu <= 128).
 * The structure is built on the host at the first projection after a mesh change (from a
 * host copy of the mesh kept by bem_set_mesh) and reused; the compression runs at every
 * projection. The AV output holds the H-matrix products. Synchronises the stream (once per
 * node). bem_hmatrix_stats: far and dense block counts, the fraction of entries in far
 * blocks, mean and largest rank of the last projection (host; BEM_ESTATE before
 * bem_set_hmatrix). bem_hmatrix_work: the algorithmic work of one node of the last
 * projection, averaged over its nodes: dense entries (each evaluated once and multiplied
 * into nu columns), sum over far blocks of rank x rows (the U_b T_b products) and of
 * rank x columns (the W_b^T V products); any pointer may be NULL (host; BEM_ESTATE before
 * bem_set_hmatrix). With bem_set_timing on, each node's leaf kernel (dense blocks and
 * U_b T_b) is timed by bem_kernel_times.
 */
bem_status bem_set_hmatrix(bem_ctx* ctx, int leaf, double eta, double eps, int rmax);
bem_status bem_hmatrix_stats(const bem_ctx* ctx, int64_t* far_blocks, int64_t* dense_blocks,
                             double* far_fraction, double* mean_rank, int* max_rank);
bem_status bem_hmatrix_work(const bem_ctx* ctx, double* dense_entries, double* far_row_terms,
                            double* far_col_terms);

/*
 * Node schedule of the mixed projection (an implementation detail of Eq. RR_approx's
 * evaluation; the paper has no counterpart). Nodes whose real parts round to the same FP32
 * value evaluate the same phase Re(z_j) |x - y| at every quadrature point: the conjugate
 * nodes z, conj(z) of a circle or ellipse centred on the real axis (the trapezoid nodes of
 * Eq. quadrature_contour are placed mirror-symmetrically, so their real parts agree
 * exactly). The mixed kernel takes such twins in pairs and computes one sine and one cosine
 * for both; the results are the same as without pairing, bit for bit.
 *   order_host  N ints (host), or NULL: slot s of the schedule holds node order[s]; twin
 *               pairs fill slots 0 .. 2 twins - 1 (slots 2 P, 2 P + 1), the rest follow.
 *   twins       (host), or NULL: number of twin pairs.
 * Set by bem_set_contour; host only. BEM_ESTATE without a contour.
 */
bem_status bem_node_order(const bem_ctx* ctx, int* order_host, int* twins);

/*
 * Fused assembly + Rayleigh-Ritz projection (Section 3, Eq. RR_approx; Algorithm 3,
 * "use U to compute B^_i"): for every contour node z_j,
 *     Bhat_j = w_j * V^H A(z_j) V                                   (nu x nu)
 * without storing A(z_j): its entries are evaluated tile by tile and contracted at once.
 *   V_dev    n x nu complex, column-major, leading dimension ldv >= n.
 *   Bhat_dev N x (nu x nu) complex: node j at offset j*nu*nu, column-major.
 *   AV_dev   optional (NULL to skip): N x (n x nu) complex, node j at offset j*n*nu,
 *            column-major with leading dimension n: Y_j = A(z_j) V (unweighted), the
 *            products the stopping test and the residuals use.
 *   precision  BEM_PREC_FP64, BEM_PREC_MIXED or BEM_PREC_HMATRIX (after bem_set_hmatrix).
 * 1 <= nu <= 256. Requires a mesh and a contour. Asynchronous on `stream`.
 */
bem_status bem_project(bem_ctx* ctx, const double* V_dev, int64_t ldv, int nu,
                       double* Bhat_dev, double* AV_dev, int precision, void* stream);

/*
 * CholeskyQR2 orthonormalisation of a basis (the paper orthonormalises U before the
 * projection, Section 4, Example 1): G = V^H V, R1 = chol(G), V <- V R1^{-1}, repeated
 * once; on return V (n x nu, column-major, leading dimension ldv) has orthonormal
 * columns and, if R_dev is not NULL, R_dev (nu x nu, column-major) holds R = R2 R1 with
 * V_in = V_out R. The second pass is FP64 throughout and sets the final orthogonality;
 * when R_dev is NULL and nu <= 128 the first pass (whose only job is to make V well
 * conditioned) runs its Gram matrix, Cholesky factor and triangular inverse in FP32 and
 * applies the inverse to V in FP64. Fails with BEM_EKERNEL if a Gram matrix is not
 * numerically positive definite (rank-deficient V). Synchronises the stream.
 */
bem_status bem_cholqr2(bem_ctx* ctx, double* V_dev, int64_t n, int64_t ldv, int nu,
                       double* R_dev, void* stream);

/*
 * Residuals of approximate eigenpairs (Section 4: ||T(lambda) u||_2 / ||u||_2), matrix-
 * free in FP64: for each column c, r_c = A(lam_c) x_c.
 *   lam_host   2*m doubles (lambda_c interleaved)
 *   X_dev      n x m complex, column-major, leading dimension ldx
 *   R_dev      optional n x m complex output (leading dimension n), may be NULL
 *   relres_host m doubles receiving ||r_c|| / ||x_c||
 * Synchronises the stream.
 */
bem_status bem_residual(bem_ctx* ctx, int m, const double* lam_host, const double* X_dev,
                        int64_t ldx, double* R_dev, double* relres_host, void* stream);
/*
 * bem_residual with a choice of arithmetic and, optionally, the k-derivative (the residual
 * of Section 4, and the derivative the refinement's Newton step needs).
 *   arith 0: FP64, as bem_residual.
 *   arith 1: double-FP32 ("float-float": every quantity as a pair of FP32 numbers, about
 *            48 significant bits) for the off-diagonal single-layer entries, each entry to
 *            a relative error of about 1e-13; the self and near-field terms stay FP64. On
 *            this GPU, whose FP64 pipe is ~65x slower than its FP32 pipe, it is over ten
 *            times faster than arith 0. The general operator (bem_set_operator with
 *            c_H != 0) always uses the FP64 kernels.
 *   Rd_dev     optional n x m complex output A'(lam_c) x_c (derivative in k), may be NULL
 * Other arguments as bem_residual. Synchronises the stream.
 */
bem_status bem_residual_arith(bem_ctx* ctx, int m, const double* lam_host, const double* X_dev,
                              int64_t ldx, double* R_dev, double* Rd_dev, double* relres_host,
                              int arith, void* stream);

/*
 * Reduced linearised eigenproblem (Section 3.1, Eq. EVP_red, Eq. sc1_cauchy_red, Eq. sc2 -
 * sc5). Given the weighted projected matrices Bhat_j (N x nu x nu, as bem_project writes
 * them, for the context's current contour), finds eigenpairs of
 *     sum_j Bhat_j y / (lambda - z_j) = 0
 * nearest the shift s by subspace iteration with a block of p vectors on the shifted and
 * inverted linearisation H = (A - s M)^{-1} M (applied through the Schur complement
 * S = sum_j Bhat_j / (z_j - s)), CholeskyQR2 after every application and a Rayleigh-Ritz
 * step every 5 iterations; stops when every Ritz value inside the contour among the p/2
 * with the largest |mu| has reduced residual
 * ||sum_j Bhat_j y / (lambda - z_j)|| / (||y|| sum_j ||Bhat_j|| / |lambda - z_j|) <= tol,
 * or after max_iter iterations. The shift must not be an eigenvalue (S must be regular;
 * a singular S is reported as BEM_EKERNEL). Directions that H annihilates are refilled
 * at random, so p may exceed the number of non-negligible eigenvalues.
 *   lam_host  2*p doubles: the p Ritz values (complex, nearest the shift first is NOT
 *             guaranteed; callers filter by position and residual)
 *   Y_dev     nu x p complex (column-major): y-parts of the Ritz vectors
 *   res_host  p doubles: their reduced residuals
 *   iters_done  iterations performed (may be NULL)
 * 1 <= p <= min(256, N nu). Uses the context's scratch. Synchronises the stream.
 */
bem_status bem_solve_reduced(bem_ctx* ctx, const double* Bhat_dev, int nu, double shift_re,
                             double shift_im, int p, int max_iter, double tol, double* lam_host,
                             double* Y_dev, double* res_host, int* iters_done, void* stream);

/*
 * Ritz vectors x = V y (Section 3: approximate eigenvectors u = U y): X_dev (n x k,
 * leading dimension ldx) = V_dev (n x nu, ldv) Y_dev (nu x k). FP64. Asynchronous.
 */
bem_status bem_ritz_vectors(bem_ctx* ctx, const double* V_dev, int64_t ldv, int nu,
                            const double* Y_dev, int k, double* X_dev, int64_t ldx, void* stream);

/*
 * Node-summed operator of Algorithm 1 (Section 3.3, Eq. linsyssim): with the mesh and the
 * contour of the context,
 *     Y = sum_j c_j A(z_j) X_j        (per_node != 0: a block X_j per node)
 *     Y = (sum_j c_j A(z_j)) X        (per_node == 0: one X; the Schur complement S = sum_j
 *                                      w_j A(z_j) / (z_j - s) is the case c_j = w_j/(z_j - s))
 * evaluated matrix-free by the fused kernel of bem_project's mixed path (FP32 entries, BF16x3
 * tcgen05 contraction, FP32 accumulation; the entries c_j A_il(z_j) are formed in FP32).
 * The operator is the 7-point rule with the self terms (no near-field corrections: it serves
 * the basis construction).
 *   coef_host  2 N doubles (host): c_j as (re, im).
 *   X_dev      n x nu complex, column-major, leading dimension ldx >= n; with per_node, N
 *              such blocks, block j at X_dev + 2 j ldx nu doubles.
 *   Y_dev      n x nu complex, column-major, leading dimension n (output).
 * 1 <= nu <= 256. Uses the context's scratch. Synchronises the stream.
 */
bem_status bem_apply_sum(bem_ctx* ctx, const double* coef_host, const double* X_dev,
                         int64_t ldx, int nu, int per_node, double* Y_dev, void* stream);

/*
 * Matrix-free solve with the same operator (Section 3.3, Eq. wjp1 / Eq. linsyssim: the
 * system S u = b of each inverse power step), never forming S:
 *     (sum_j c_j A(z_j)) X = B
 * by restarted GMRES (restart 40) on every column at once; each Arnoldi step applies the
 * operator to one vector per column with the fused kernel (as bem_apply_sum), the Arnoldi
 * vectors are FP32 and orthogonalised by classical Gram-Schmidt run twice (FP64 dot
 * products), the Hessenberg least-squares problems are solved by Givens rotations on the
 * host (FP64). Stops when every column's true relative residual ||B - S X|| / ||B|| is
 * <= tol (checked at each restart, and when the rotations estimate it below tol / 2), or
 * after max_iter Arnoldi steps in total.
 *   coef_host   2 N doubles (host): c_j as (re, im).
 *   B_dev       n x nu complex, column-major, leading dimension ldb >= n.
 *   X_dev       n x nu complex, column-major, leading dimension ldx >= n (output).
 *   iters       (host, may be NULL): Arnoldi steps taken.
 *   relres_host (host, may be NULL): nu doubles, the final true relative residuals.
 * The operator itself carries the split-precision error of the fused kernel (~3e-5
 * relative), so residuals much below ~1e-5 are not reachable: tol around 1e-4 suits the
 * inexact inverse power steps. 1 <= nu <= 256, tol > 0, max_iter >= 1. Does not fail on
 * slow convergence: the caller reads relres_host. Uses the context's scratch. Synchronises
 * the stream.
 */
bem_status bem_solve_sum(bem_ctx* ctx, const double* coef_host, const double* B_dev,
                         int64_t ldb, int nu, double tol, int max_iter, double* X_dev,
                         int64_t ldx, int* iters, double* relres_host, void* stream);

/*
 * Basis improvement by q steps of the inverse power method for the Cauchy linearisation
 * (Section 3.3, Algorithm 1; Eq. wjp1, Eq. vjp1, Eq. viupd, Eq. linsyssim) with shift s,
 * applied to every column of V (n x nu, leading dimension ldv) at once, starting from
 * v_j = u / (z_j - s):
 *     S u' = sum_j B_j v_j / (z_j - s),  S = sum_j w_j A(z_j) / (z_j - s),
 *     v_j' = (v_j - u') / (z_j - s).
 * (The algebra of (A - sM) w' = M w; the extra u term of the paper's right-hand side
 * vanishes because M has a zero last block.) S is assembled densely in FP32 and LU-
 * factorised once; sum_j B_j v_j / (z_j - s) is applied matrix-free by the node-summed fused
 * kernel (bem_apply_sum). On return V
 * holds the last u (not orthonormalised). Needs n^2 * 8 + N n nu * 8 bytes of scratch.
 * N <= 64, 1 <= nu <= 256. Synchronises the stream.
 */
bem_status bem_inverse_power(bem_ctx* ctx, double* V_dev, int64_t ldv, int nu, int q,
                             double shift_re, double shift_im, void* stream);

/*
 * Basis improvement by q steps of the inverse power method for the Chebyshev interpolant
 * (Section 3.2, Algorithm 2; Eq. reccurenceCheb_odd, Eq. reccurenceCheb_even, Eq. Gmtx,
 * Eq. bodd / beven), for a context whose contour is of kind CHEBYSHEV (N >= 4 points x_k of
 * the interval, degree m = N - 1), the shift at the interval's centre (zeta = 0). The
 * iterate w = [v_0; ..; v_{m-1}] of the colleague linearisation starts from v_i = T_i(0) V;
 * each step solves A w' = M w: the block rows 0..m-2 give the recurrence for v', the last
 * row G u = b with G = sum_i T_i(0) L_i (L_i its blocks, combinations of
 * B_i = sum_k c_ik A(x_k)) assembled densely in FP32 and LU-factorised once, and b from one
 * node-summed application sum_k A(x_k) X_k of the fused kernel; the columns are rescaled.
 * On return V (n x nu, leading dimension ldv) holds the u-part v_0 (not orthonormalised).
 * Scratch: n^2 * 8 + (2 m + N + 1) n nu * 8 bytes. 1 <= nu <= 256. Synchronises the stream.
 */
bem_status bem_inverse_power_chebyshev(bem_ctx* ctx, double* V_dev, int64_t ldv, int nu, int q,
                                       void* stream);

/*
 * bem_inverse_power without forming S (the basis construction at sizes where the dense S,
 * n^2 * 8 bytes, does not fit): the same q steps, each S u' = b solved by bem_solve_sum's
 * GMRES to relative residual tol with at most max_iter Arnoldi steps. Memory: the N n nu
 * iterates, 41 n nu FP32 Arnoldi vectors and the fused kernel's basis planes, no n^2 term.
 * gmres_iters (host, may be NULL): Arnoldi steps over all q solves. Synchronises the stream.
 */
bem_status bem_inverse_power_mf(bem_ctx* ctx, double* V_dev, int64_t ldv, int nu, int q,
                                double shift_re, double shift_im, double tol, int max_iter,
                                int* gmres_iters, void* stream);

/*
 * FP64 refinement of approximate eigenpairs of A(k) x = 0 (the eigenpairs the paper
 * measures by ||T(lambda) u|| / ||u||, Section 4): residual inverse iteration with a
 * frozen FP32 LU of A(sigma) and a Newton step for lambda on
 * e^H A(sigma)^{-1} A(lambda) x = 0 (e = the starting vector); residuals A(lambda) x and
 * A'(lambda) x are FP64 and matrix-free, so the converged pair is an FP64 eigenpair.
 * sigma starts at the given lambda and moves to the current one when the step stalls.
 *   lam_host   2*m doubles: in, starting values; out, refined eigenvalues
 *   X_dev      n x m (ld ldx): in, starting vectors; out, refined vectors (e^H x = 1)
 *   relres_host m doubles: final ||A(lambda) x|| / ||x||
 *   iters_host  optional m ints: iterations used
 * Stops a pair when |dlambda| <= tol |lambda| or after maxit iterations. Synchronises.
 */
bem_status bem_refine(bem_ctx* ctx, int m, double* lam_host, double* X_dev, int64_t ldx,
                      double tol, int maxit, double* relres_host, int* iters_host, void* stream);

/*
 * The whole method (Algorithm 3 with one outer pass) for the context's mesh and contour:
 * basis V0 (n x nu, ld ldv; not modified) -> q inverse power steps about the contour's
 * centre, taken on the circle of radius 2 max(a, b) about that centre (the Cauchy
 * linearisation has eigenvalues clustered at its nodes, which must stay farther from the
 * shift than the wanted eigenvalues) -> CholeskyQR2 -> projection on the contour itself
 * (precision BEM_PREC_FP64 or BEM_PREC_MIXED) ->
 * reduced linearised eigenproblem -> Ritz pairs inside the contour with small reduced
 * residual, nearest the centre first, at most kmax -> FP64 refinement (tolerance tol).
 *   lam_host    2*kmax doubles: eigenvalues found
 *   X_dev       n x kmax (ld ldx): their vectors
 *   k_found     number of pairs returned (several may share an eigenvalue: degenerate
 *               eigenvalues appear once per independent vector)
 *   relres_host kmax doubles: ||A(lambda) x|| / ||x||
 * Synchronises the stream.
 */
bem_status bem_solve(bem_ctx* ctx, const double* V0_dev, int64_t ldv, int nu, int q,
                     int precision, double tol, int kmax, double* lam_host, double* X_dev,
                     int64_t ldx, int* k_found, double* relres_host, void* stream);

/*
 * Synchronise `stream` and report errors that kernels recorded in the context's device
 * status word since the last check (asynchronous calls such as bem_project report device-
 * side failures here): BEM_ETIMEOUT if a bounded wait inside a kernel gave up (the kernel
 * then stopped cleanly and its outputs are invalid), BEM_EKERNEL / BEM_EINVAL for other
 * recorded failures, BEM_ECUDA for a CUDA error. Clears the status word.
 */
bem_status bem_check(bem_ctx* ctx, void* stream);
/*
 * Asynchronous mode (operational; the paper has no counterpart). With on != 0,
 * bem_cholqr2 returns without waiting for its device status word, so that a pipeline of
 * set-up, orthonormalisation and projection runs without a host synchronisation; a Gram
 * matrix that was not positive definite is then reported by the next bem_check (or by the
 * next call that synchronises). Off by default.
 */
bem_status bem_set_async(bem_ctx* ctx, int on);
/*
 * Bound of the pipeline-stage waits of the fused mixed-precision projection kernel
 * (operational; the paper has no counterpart): each wait of a block on its shared-memory
 * pipeline (copies landed, entries evaluated, tensor-core products done) polls an mbarrier
 * at most `polls` times, with 64 ns sleeps after the first 64 (default 1 << 24, about a
 * second), then records BEM_ETIMEOUT in the device status word, raises the block's abort
 * flag and returns. The waits that drain copies and tensor-core products still in flight
 * before a block frees its shared memory and tensor memory keep the default bound whatever
 * this value is, so an aborted block leaves no asynchronous work behind and the context
 * stays usable. polls = 0 makes every stage wait give up at once (a way to exercise the
 * timeout path). Applies to projections planned after the call (bem_project,
 * bem_apply_sum, batches created afterwards).
 */
bem_status bem_set_wait_limit(bem_ctx* ctx, uint32_t polls);
/*
 * Split of the fused mixed-precision kernel's transcendental work between two pipes
 * (tuning; the paper has no counterpart). Each entry of A(z_j) sums 7 quadrature points,
 * each needing e^{i Re(z_j) r}: for the first poly_points of them (0..4) its cosine and
 * sine come from minimax polynomials on the FP32 FMA pipe (phase reduced in half
 * revolutions; error below 2e-7), for the rest from the MUFU sin/cos unit, so that neither
 * pipe idles while the other binds. -1 (the default) selects the measured best split for
 * the unit shape. Applies to later bem_project calls. BEM_EINVAL outside -1..4.
 */
bem_status bem_set_eval_split(bem_ctx* ctx, int poly_points);
/*
 * Arithmetic of the residuals ||A(lambda) x|| / ||x|| that bem_refine and bem_solve report
 * for their eigenpairs (Section 4's accuracy measure): 0 FP64 (default), 1 double-FP32
 * as bem_residual_arith (entries to ~1e-13 relative; over ten times faster on this GPU,
 * for the largest meshes, where an FP64 residual takes seconds per eigenpair). The
 * refinement's own iterations always use double-FP32. BEM_EINVAL for other values.
 */
bem_status bem_set_refine_residual(bem_ctx* ctx, int arith);
/*
 * Twin pairs across thread-block clusters in the fused mixed-precision kernel (scheduling;
 * the paper has no counterpart). When one node's [Re Y | Im Y] accumulator fills a whole
 * SM's tensor memory (bases of more than 128 columns) and the contour has twin nodes (equal
 * real parts, as the conjugate nodes of a contour symmetric about the real axis), on != 0
 * (the default) runs each twin pair on a cluster of two CTAs: each evaluates half of every
 * 128 x 16 block of entries for both nodes, sharing the distance, sine and cosine of each
 * quadrature point, and sends the other node's half to its partner through distributed
 * shared memory. on = 0 keeps one node per CTA. The results agree to the rounding of the
 * FP32 evaluation (the same operations on the same values, so normally bit for bit).
 * Applies to later bem_project calls. BEM_EINVAL for other values than 0 and 1.
 */
bem_status bem_set_twin_clusters(bem_ctx* ctx, int on);
/*
 * Work decomposition of the last mixed-precision bem_project on this context: nodes per
 * work unit (1..4), whether twin pairs ran on two-CTA clusters (0/1), column splits S and
 * CTAs launched. Zeros before the first such projection. Any pointer may be NULL.
 */
bem_status bem_mixed_shape(const bem_ctx* ctx, int* nodes_per_unit, int* paired, int* splits,
                           int64_t* ctas);

/* Number of CUDA kernels this context has launched since creation (diagnostics). */
int64_t bem_kernel_launches(const bem_ctx* ctx);

/*
 * Diagnostics for roofline accounting (no counterpart in the paper).
 * bem_set_timing: when enable != 0, every bem_project records CUDA events on its stream
 *   around its main kernel (the fused evaluation + contraction; with BEM_PREC_HMATRIX the
 *   leaf kernel of every node); resets the record.
 * bem_kernel_times: durations in ms of up to max_out recorded launches (in call order),
 *   synchronising on their stop events; *count receives how many; resets the record.
 *   At most 256 launches are kept between resets.
 * bem_microbench: measured throughput (operations per second over the whole device) of
 *   one pipe: kind 0 FP64 FMA (2 flops each), 1 FP32 FMA (2 flops each), 2 MUFU ex2,
 *   3 MUFU sin, 4 MUFU cos, 5 MUFU rsqrt, 6 paired FP32 FMA (fma.rn.f32x2, 2 flops per
 *   lane), 7 the fused kernel's polynomial sine-and-cosine on the FMA pipe (phases per
 *   second, each giving both). Synchronous; runs on the legacy default stream.
 */
bem_status bem_set_timing(bem_ctx* ctx, int enable);
bem_status bem_kernel_times(bem_ctx* ctx, double* ms_out, int max_out, int* count);
bem_status bem_microbench(bem_ctx* ctx, int kind, double* ops_per_s);

/*
 * Chebyshev variant (Section 2, Eq. Chebyshev; Section 3, Eq. sc1_chebyshev_red; the
 * setting of Algorithm 2), for eigenvalues near a real interval. Requires a contour of kind
 * CHEBYSHEV with N >= 4 points (interpolation degree m = N - 1).
 * bem_chebyshev_coeffs: from P_dev = the unweighted projections V^H A(z_k) V of bem_project
 *   (N x nu x nu, as Bhat), the coefficients of the interpolant in the Chebyshev basis,
 *   B_i = (2 - delta_i0) / N sum_k cos(i pi (k + 1/2) / N) P_k, i = 0..N-1 (B_dev, same
 *   layout). Asynchronous.
 * bem_solve_chebyshev: eigenpairs of sum_i B_i T_i(zeta) y = 0, zeta = (z - c) / a, nearest
 *   the shift (in z units), by subspace iteration of block size p with the shift-and-invert
 *   operator of the colleague linearisation (A - sigma M)^{-1} M, A w = zeta M w,
 *   w = [T_0 y; ..; T_{m-1} y]; each application solves the block system by the three-term
 *   recurrence and one nu x nu system (Algorithm 2 at sigma = 0). Outputs as
 *   bem_solve_reduced: lam_host (2p doubles, z units), Y_dev (nu x p, the y-parts), res_host
 *   (p reduced residuals ||sum_i T_i(zeta) B_i y|| / (||y|| sum_i |T_i(zeta)| ||B_i||_1)).
 *   Stops when the dominant half of the Ritz values contains values with |Re zeta| < 1 and
 *   |Im zeta| < 0.25 and all of them have residuals <= tol, or after max_iter steps.
 *   Synchronises the stream.
 */
bem_status bem_chebyshev_coeffs(bem_ctx* ctx, const double* P_dev, int nu, double* B_dev,
                                void* stream);
/* One application of the shift-and-invert operator of bem_solve_chebyshev to p columns:
 * HW = (A - sigma M)^{-1} M W, sigma = (shift - c) / a; W_dev and HW_dev ((N - 1) nu x p,
 * column-major, leading dimension (N - 1) nu). Synchronises the stream. */
bem_status bem_chebyshev_apply(bem_ctx* ctx, const double* B_dev, int nu, double shift_re,
                               double shift_im, const double* W_dev, int p, double* HW_dev,
                               void* stream);
bem_status bem_solve_chebyshev(bem_ctx* ctx, const double* B_dev, int nu, double shift_re,
                               double shift_im, int p, int max_iter, double tol, double* lam_host,
                               double* Y_dev, double* res_host, int* iters_done, void* stream);

/*
 * Near-field treatment (an operator variant for fine meshes; the paper integrates the
 * regular panel integrals by Gauss quadrature, Section 1, and a fixed low-order rule loses
 * accuracy when the collocation point is close to the panel). A pair (i, l), i != l, is
 * near when the distance between the centroids is below twice the larger panel diameter
 * (longest edge). mode 0: off, every pair i != l takes the 7-point rule; mode 1: near pairs
 * take the 8 x 8 conical-product rule (the triangle as the image of the unit square under
 * y = a + s (b - a) + s t (c - b), Gauss-Legendre in s and t, collapsed at the vertex nearest
 * the collocation point); mode 2: as mode 1, except that the mixed-precision projection takes
 * the near pairs' corrections from the surrogate network (bem_surrogate_*; BEM_ESTATE if
 * none is loaded). The mode applies to bem_project (both precisions), bem_residual,
 * bem_refine and bem_solve (residuals and refinement always use the 8 x 8 rule); the
 * Algorithm 1 operator of bem_inverse_power keeps the 7-point rule. It is kept across
 * bem_set_mesh (the pair list is rebuilt for the new mesh at first use). Building the list
 * synchronises `stream`. Contexts with a near-field mode are not accepted by the batched
 * projection. Precision: the FP64 projection, residuals and refinement evaluate the rule in
 * FP64 with the exact functions; the mixed projection evaluates it in FP32 with the
 * hardware approximations of exp2, sine, cosine and reciprocal square root (pair geometry
 * shared by eight contour nodes; N x nnz FP32 values held in the context's work memory).
 * bem_near_pairs: the pair list of the current mesh (builds it if needed): *nnz pairs;
 *   row_ptr_host (n + 1 int32, nullable) and cols_host (nnz int32, nullable, increasing
 *   within each row). BEM_ESTATE when the mode is 0. Synchronous.
 */
bem_status bem_set_near_field(bem_ctx* ctx, int mode, void* stream);
bem_status bem_near_pairs(bem_ctx* ctx, int64_t* nnz, int32_t* row_ptr_host, int32_t* cols_host,
                          void* stream);

/*
 * Surrogate network of the near-field correction (a learned replacement for the 8 x 8 rule
 * of near pairs in the mixed projection; the paper has no counterpart). A multilayer
 * perceptron 11 -> 64 -> 64 -> 64 -> 2 (tanh) maps a near pair's canonical features to
 * (A_near - A_7) / h, h the panel diameter. Features (11 floats per sample): the triangle's
 * vertices in a frame with origin at the collocation point x, e1 along (b - a), e3 along the
 * normal (b - a) x (c - b) turned so that a lies on its non-negative side, e2 = e3 x e1
 * (a the vertex nearest x, b and c following it), divided by h; then Re(k h), Im(k h).
 * Parameters (bem_surrogate_size() floats): in_shift[11], in_scale[11], W1[64][11], b1[64],
 * W2[64][64], b2[64], W3[64][64], b3[64], W4[2][64], b4[2], out_scale[2]; the output is
 * out_scale * (W4 h3 + b4) on features standardised as (f - in_shift) * in_scale.
 * The context keeps FP32 master weights (trained) and an inference copy with the weights
 * rounded to BF16 (used by bem_surrogate_forward and by the mixed projection in near-field
 * mode 2). In the projection the network runs on the tensor core: tiles of 128 (pair,
 * node) samples, the three 64-wide layers as BF16 tcgen05 MMAs on activations split into
 * BF16 hi + lo (FP32 accumulation), tanh by the MUFU's approximation; a sample whose
 * features leave the training box (widened by 2 % of its width) takes the 8 x 8 rule.
 * Device arrays are row-major: features count x 11, targets and outputs count x 2.
 *
 * bem_surrogate_init: Xavier-uniform weights from `seed`, zero biases, identity scalings.
 * bem_surrogate_set / _get: copy the parameters from / to the host (which: 0 master, 1
 *   inference copy); synchronous.
 * bem_surrogate_samples: `count` training samples from the current mesh's near pairs
 *   (near-field mode >= 1 required): pair and k drawn uniformly (k in [kr_lo, kr_hi] x
 *   [ki_lo, ki_hi], FP32-rounded) by SplitMix64 of `seed`; features, target (A_near - A_7)/h
 *   from the FP64 8 x 8 rule; optionally pairs_dev (count x 2 int32: row, panel) and k_dev
 *   (count complex). Asynchronous.
 * bem_surrogate_forward: outputs of the inference copy. Asynchronous.
 * bem_surrogate_grad: mean over the samples of the squared error in units of out_scale,
 *   summed over the outputs (*loss_host), and its gradient with respect to the master parameters (grad_dev,
 *   bem_surrogate_size() floats; zero for the scalings), FP32 forward and backward kernels
 *   of the library. Synchronous.
 * bem_surrogate_train: `epochs` passes of Adam (betas 0.9 / 0.999; the step size decays
 *   geometrically from lr to lr / 100 over the run) over the samples in
 *   batches of `batch`, each epoch in an affine permutation of the samples; fit_scaling != 0
 *   first sets the standardisation and output scale from the samples' means and standard
 *   deviations. loss_host (nullable, epochs doubles): mean batch loss per epoch. Refreshes
 *   the inference copy. Synchronous.
 * Errors: BEM_EINVAL for bad arguments, BEM_ESTATE without a network (init or set first).
 */
int bem_surrogate_size(void);
/*
 * bem_surrogate_usage: samples (near pair x contour node) whose correction the network gave
 * (*network) and whose features fell outside its training box so that the plain 8 x 8 rule
 * gave it (*rule), summed over the mixed projections with near-field mode 2 since the
 * previous call; the counters are reset. Synchronises the stream. Zeros before the first
 * such projection.
 */
bem_status bem_surrogate_usage(bem_ctx* ctx, int64_t* network, int64_t* rule, void* stream);
bem_status bem_surrogate_init(bem_ctx* ctx, uint64_t seed, void* stream);
bem_status bem_surrogate_set(bem_ctx* ctx, const float* params_host, int64_t count, void* stream);
bem_status bem_surrogate_get(bem_ctx* ctx, int which, float* params_host, int64_t count,
                             void* stream);
bem_status bem_surrogate_samples(bem_ctx* ctx, double kr_lo, double kr_hi, double ki_lo,
                                 double ki_hi, int64_t count, uint64_t seed, float* feat_dev,
                                 float* target_dev, int32_t* pairs_dev, double* k_dev,
                                 void* stream);
bem_status bem_surrogate_forward(bem_ctx* ctx, const float* feat_dev, int64_t count,
                                 float* out_dev, void* stream);
bem_status bem_surrogate_grad(bem_ctx* ctx, const float* feat_dev, const float* target_dev,
                              int64_t count, float* grad_dev, double* loss_host, void* stream);
bem_status bem_surrogate_train(bem_ctx* ctx, const float* feat_dev, const float* target_dev,
                               int64_t count, int epochs, int batch, double lr, int fit_scaling,
                               uint64_t seed, double* loss_host, void* stream);

/*
 * Context statistics and checkpoints (operational support; the paper has no counterpart).
 * bem_stats: the context's sizes and counters: device, panels n, vertices nv, contour nodes N
 *   (0 before bem_set_contour), near-field mode and its pair count (-1 while the list is not
 *   built for the current mesh), kernel launches so far, bytes of device workspace held,
 *   whether a surrogate network is loaded. Host only, no synchronisation.
 * bem_save_state: writes a checkpoint of what defines the operator and the contour (mesh,
 *   contour, near-field mode, surrogate network master parameters) into buf (host). With
 *   buf == NULL it only sets *len to the size needed; with *len too small it fails with
 *   BEM_EINVAL and sets *len. Synchronous. BEM_ESTATE without a mesh.
 * bem_load_state: restores such a checkpoint into a context (any device): sets the mesh,
 *   the network, the contour and the near-field mode as the corresponding calls would.
 *   BEM_EINVAL for a buffer that is not a checkpoint, truncated or inconsistent.
 */
typedef struct {
  int device;
  int64_t n, nv;
  int N;
  int near_mode;
  int64_t near_pairs;
  int64_t launches;
  int64_t workspace_bytes;
  int surrogate_ready;
} bem_stats_t;
bem_status bem_stats(const bem_ctx* ctx, bem_stats_t* out);
bem_status bem_save_state(bem_ctx* ctx, void* buf, size_t* len, void* stream);
bem_status bem_load_state(bem_ctx* ctx, const void* buf, size_t len, void* stream);

/*
 * Batched projection (Section 3's projection for many independent problems at once, as a
 * parameter study or a sweep over geometries needs). Each problem is a context with its
 * mesh and contour already set (bem_set_mesh, bem_set_contour), a basis V_dev[k]
 * (n_k x nu[k] complex128, column-major, leading dimension ldv[k] >= n_k) and an output
 * Bhat_dev[k] (N_k x nu[k] x nu[k] complex128, as bem_project). All contexts must be
 * distinct and on one device; 1 <= nprob <= 4096, 1 <= nu[k] <= min(n_k, 256); only
 * precision BEM_PREC_MIXED is accepted (BEM_EINVAL otherwise).
 *
 * bem_batch_create plans every problem (workspaces of the contexts, FP32 self terms),
 * orders the problems by decreasing work and records one CUDA graph: per problem the basis
 * preparation, then ONE persistent launch of the fused kernel (one block per SM taking the
 * work units of all problems from a shared counter), then per problem the V^H Y reduction
 * and weighting. With autotune != 0 it times whole runs for every work-unit shape in
 * {column splits: per-problem default, 1, 2, 3, 4} x {nodes per unit: up to 4, up to 2}
 * (three runs each, which overwrite Bhat) and keeps the fastest. It synchronises `stream` first (V may
 * still be written there) and runs its work on a private stream; on return the batch is
 * idle. The caller owns V and Bhat and must keep them allocated while the batch exists.
 * bem_batch_run replays the graph on `stream` (asynchronous). It returns BEM_ESTATE if a
 * context's mesh, contour or workspace changed since creation (create a new batch then).
 * Device-side errors are reported per context by bem_check.
 * bem_batch_info: chosen split count and node cap (0 = per-problem default), work units of
 * the persistent launch, and the autotuner's time per run in ms (0 without autotuning).
 * bem_project_batched: create (no autotuning), run, wait for completion, check every
 * context, destroy. Synchronous.
 * Errors are reported through bem_last_error of the first context.
 */
typedef struct bem_batch bem_batch;
bem_status bem_batch_create(bem_ctx* const* ctxs, int nprob, const double* const* V_dev,
                            const int64_t* ldv, const int* nu, double* const* Bhat_dev,
                            int precision, int autotune, bem_batch** out, void* stream);
bem_status bem_batch_run(bem_batch* batch, void* stream);
bem_status bem_batch_info(const bem_batch* batch, int* splits, int* nodes_per_unit,
                          int64_t* units, double* tuned_ms);
void bem_batch_destroy(bem_batch* batch);
bem_status bem_project_batched(bem_ctx* const* ctxs, int nprob, const double* const* V_dev,
                               const int64_t* ldv, const int* nu, double* const* Bhat_dev,
                               int precision, void* stream);

/*
 * Order of the Cauchy approximation (Section 4, Example 3: grow m until the rational
 * approximation is accurate on the circle of radius r/2 inside the contour). For each N of
 * N_list (count entries, each 2..1024) the N-node trapezoid approximation on the contour
 * (kind circle or ellipse, centre c, semi-axes a, b; nodes and weights as bem_set_contour)
 * T~(zeta) X = sum_j w_j T(z_j) X / (z_j - zeta) is compared with T(zeta) X at nsamples
 * (1..64) points of the inner contour (same centre, semi-axes a/2, b/2, angles
 * 2 pi (s + 1/4) / nsamples) for the caller's test vectors X_dev (n x ncols complex,
 * column-major, leading dimension ldx, 1 <= ncols <= 64). err_out[k] receives the largest
 * relative error ||T~ X - T X||_F / ||T X||_F of N_list[k]; *N_chosen the first N whose
 * error is <= tol (or -1). T is the context's operator (near field included when set),
 * applied matrix-free in double-FP32 arithmetic (entries to ~1e-13). Does not change the
 * context's contour. Synchronises the stream.
 */
bem_status bem_select_order(bem_ctx* ctx, int kind, double c_re, double c_im, double a, double b,
                            const int* N_list, int count, int nsamples, const double* X_dev,
                            int64_t ldx, int ncols, double tol, int* N_chosen, double* err_out,
                            void* stream);

/*
 * Allocation-free projection (the paper has no counterpart: this serves callers that
 * cannot call cudaMalloc, such as code running under a locked or externally owned memory
 * pool, or a process whose device footprint must not grow after start-up).
 * Computes the same Bhat_j = w_j V^H A(z_j) V as bem_project with BEM_PREC_FP64, without a
 * context: the caller passes the mesh already on the device (xyz_dev: 3*nv doubles,
 * tri_dev: 3*nt int32), the contour parameters (as bem_set_contour), V_dev (nt x nu,
 * column-major, ldv >= nt) and Bhat_dev (N x nu x nu, as bem_project). Every intermediate
 * lives in one 64 MiB device array inside the library, which each GPU that loads the
 * library holds until the process exits; nothing is allocated or freed by this call.
 * Limit: 372*nt + 16*nt*N + 16*nt*nu + 32*N bytes (plus alignment) must fit in 64 MiB,
 * otherwise BEM_EINVAL (e.g. nt = 3072, N = 32, nu = 64 fits; the nodes are processed in
 * groups that fit). Every call looks up the array's device address on `device` (with that
 * device current; this allocates nothing, and a primary context that was reset and
 * re-created in between is handled); the first call on a device may load the module, so
 * make it before any stream capture. All calls share the array and it keeps the last
 * call's contents: calls that overlap on the GPU (other streams or threads) race and must
 * be serialised by the caller. Returns BEM_EINVAL for a bad argument, a problem beyond the
 * limit or a vertex index out of range, BEM_ECUDA on a CUDA error; the reason is kept per
 * host thread for bem_noalloc_last_error. Synchronises the stream once (after the geometry
 * checks); the rest is asynchronous on `stream`.
 */
bem_status bem_project_fp64_noalloc(int device, int64_t nv, const double* xyz_dev, int64_t nt,
                                    const int32_t* tri_dev, int kind, double c_re, double c_im,
                                    double a, double b, int N, const double* V_dev,
                                    int64_t ldv, int nu, double* Bhat_dev, void* stream);
/*
 * Message of the calling host thread's last failed bem_project_fp64_noalloc call (empty
 * after a successful one). The string stays valid until the thread's next call.
 */
const char* bem_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BEM_GB300_H */
