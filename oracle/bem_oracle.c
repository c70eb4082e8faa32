/*
 * Plain FP64 CPU oracle for the Helmholtz single-layer collocation matrix A(k).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's CPU
 * baseline load this library. It shares no code, header or constant table with the CUDA
 * path; the two sides only read the same mesh arrays.
 *
 * What is computed (the method's matrix T(k) with a = 1, b = 0, i.e. the single-layer part
 * of the boundary integral equation, Section 1, Eq. (HelmBIM) and Eq. (GreenFun)):
 *
 *   A_il(k) = sum_q W_lq g(k, |x_i - y_lq|),   g(k, r) = exp(i k r) / (4 pi r),      i != l
 *   A_ii(k) = integral over triangle i of g(k, |x_i - y|) dA(y)                       i == l
 *
 * with x_i the centroid of triangle i (constant-element collocation), y_lq and W_lq the
 * points and weights of Radon's 7-point degree-5 rule on triangle l (weights times area).
 * The singular self integral is taken in polar coordinates about x_i in the plane of the
 * triangle; the radial integral is exact,
 *
 *   int_0^R exp(i k rho) / (4 pi rho) rho d rho = R h(i k R) / (4 pi),   h(w) = (e^w - 1)/w,
 *
 * and the angular integral over each edge is taken in u = asinh(s / d) (d the distance
 * from x_i to the edge's line, s the signed position along it from the foot of the
 * perpendicular, so R = d cosh(u) and d(phi) = du / cosh(u)): the integrand d h(i k R) is
 * entire in u, and 16-point Gauss-Legendre is used on each side of u = 0. The derivative dA/dk, used by the eigenvalue refinement, is taken term
 * by term: g' = i exp(i k r) / (4 pi) and, for the self term, i R^2 h'(i k R) / (4 pi).
 *
 * Near field (operator variant used for fine meshes): a pair (i, l), i != l, is near when
 * the distance between the centroids is below 2 max(h_i, h_l), h the panel diameter (its
 * longest edge). Its entry is then the 64-point conical-product rule instead of the 7-point
 * rule: the triangle (a, b, c) is the image of the unit square under
 * y = a + s (b - a) + s t (c - b), with Jacobian 2 |T| s, and 8-point Gauss-Legendre is used in
 * s and in t; the collapsed vertex a is the vertex of triangle l nearest x_i (the first of
 * them in the triangle's order on a tie), b and c follow it cyclically.
 *
 * Operator variant (the paper's general T = A H - B G of Eq. HelmBIM, for Neumann and Robin
 * conditions): with coefficients (c_G, c_H) the matrix is c_G G + c_H H, G the single layer
 * above and H = 1/2 I + K the double layer with its jump (the unknown is then the boundary
 * value u, Green's representation taken to the boundary from inside with outward normals):
 *
 *   K_il(k) = sum_q W_lq dg/dn_y(x_i, y_lq),  dg/dn_y = exp(i k r) (i k r - 1) (y - x).n_l
 *                                                        / (4 pi r^3),             i != l
 *   K_ii(k) = 0  (x_i lies in the plane of triangle i, so (y - x).n_i vanishes on it)
 *
 * n_l the unit normal of triangle l in the vertex order (outward for an outward-oriented
 * mesh). Its k-derivative is -k exp(i k r) (y - x).n_l / (4 pi r). Near pairs take the same
 * 64-point conical rule for this kernel. The default (c_G, c_H) = (1, 0) is the single layer.
 *
 * Everything is double / double complex, loops are plain, rows are spread over OpenMP
 * threads (no blocking, no reordering of any sum).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double PI = 3.14159265358979323846264338327950288;

/* ---------------- quadrature rules ---------------- */

/* Radon's 7-point rule (degree 5) in barycentric coordinates; weights sum to 1. */
static void rule7(double bary[7][3], double w[7]) {
    const double s15 = sqrt(15.0);
    const double a1 = (6.0 - s15) / 21.0, b1 = (9.0 + 2.0 * s15) / 21.0;
    const double a2 = (6.0 + s15) / 21.0, b2 = (9.0 - 2.0 * s15) / 21.0;
    const double w0 = 9.0 / 40.0;
    /* the points nearer the vertices (a1) carry the smaller weight */
    const double w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;
    double pts[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3},
                        {a1, a1, b1}, {a1, b1, a1}, {b1, a1, a1},
                        {a2, a2, b2}, {a2, b2, a2}, {b2, a2, a2}};
    double ww[7] = {w0, w1, w1, w1, w2, w2, w2};
    memcpy(bary, pts, sizeof(pts));
    memcpy(w, ww, sizeof(ww));
}

/* n-point Gauss-Legendre on [-1, 1] by Newton's method on P_n (three-term recurrence). */
static void gauss_legendre(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double t = cos(PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
        }
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

/* ---------------- small vector helpers ---------------- */

static void sub3(const double* a, const double* b, double* o) {
    o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
static double dot3(const double* a, const double* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static double norm3(const double* a) { return sqrt(dot3(a, a)); }
static void cross3(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* h(w) = (e^w - 1) / w and h'(w) = (w e^w - e^w + 1) / w^2, by Taylor series near 0. */
static cplx h_fun(cplx w) {
    if (cabs(w) < 0.5) {
        cplx s = 0.0, term = 1.0;           /* term = w^m / (m+1)! */
        for (int m = 0; m < 24; ++m) {
            s += term;
            term *= w / (m + 2.0);
        }
        return s;
    }
    return (cexp(w) - 1.0) / w;
}
static cplx hprime_fun(cplx w) {
    if (cabs(w) < 0.5) {
        cplx s = 0.0, wp = 1.0;              /* sum_{m>=1} m w^{m-1} / (m+1)! */
        double fact = 2.0;                   /* (m+1)! at m = 1 */
        for (int m = 1; m < 26; ++m) {
            s += m * wp / fact;
            wp *= w;
            fact *= (m + 2.0);
        }
        return s;
    }
    return (w * cexp(w) - cexp(w) + 1.0) / (w * w);
}

/* ---------------- geometry ---------------- */

typedef struct {
    double centroid[3];
    double area;
    double nrm[3];     /* unit normal, vertex order */
    double diam;       /* longest edge */
    double v[3][3];    /* vertices */
    double qp[7][3];
    double qw[7];
} panel_t;

static void panel_geometry(const double* xyz, const int32_t* tri, int64_t l, panel_t* P) {
    double bary[7][3], w[7];
    rule7(bary, w);
    const double* v0 = xyz + 3 * (int64_t)tri[3 * l + 0];
    const double* v1 = xyz + 3 * (int64_t)tri[3 * l + 1];
    const double* v2 = xyz + 3 * (int64_t)tri[3 * l + 2];
    double e1[3], e2[3], nrm[3];
    sub3(v1, v0, e1);
    sub3(v2, v0, e2);
    cross3(e1, e2, nrm);
    P->area = 0.5 * norm3(nrm);
    for (int c = 0; c < 3; ++c) P->nrm[c] = nrm[c] / (2.0 * P->area);
    for (int c = 0; c < 3; ++c) P->centroid[c] = (v0[c] + v1[c] + v2[c]) / 3.0;
    double e3[3];
    sub3(v2, v1, e3);
    P->diam = fmax(fmax(norm3(e1), norm3(e2)), norm3(e3));
    for (int c = 0; c < 3; ++c) {
        P->v[0][c] = v0[c];
        P->v[1][c] = v1[c];
        P->v[2][c] = v2[c];
    }
    for (int q = 0; q < 7; ++q) {
        for (int c = 0; c < 3; ++c)
            P->qp[q][c] = bary[q][0] * v0[c] + bary[q][1] * v1[c] + bary[q][2] * v2[c];
        P->qw[q] = w[q] * P->area;
    }
}

/* ---------------- kernels ---------------- */

/* g(k, r) (deriv = 0) or dg/dk (deriv = 1) at distance r. */
static cplx g_kernel(cplx k, double r, int deriv) {
    const cplx e = cexp(I * k * r);
    return deriv ? I * e / (4.0 * PI) : e / (4.0 * PI * r);
}

/* dg/dn_y (deriv = 0) or its k-derivative (deriv = 1) for y - x = d, normal n at y. */
static cplx dl_kernel(cplx k, const double* d, const double* n, int deriv) {
    const double r = norm3(d);
    const double dn = dot3(d, n);
    const cplx e = cexp(I * k * r);
    if (deriv) return -k * e * dn / (4.0 * PI * r);
    return e * (I * k * r - 1.0) * dn / (4.0 * PI * r * r * r);
}

/* ---------------- the self term ---------------- */

/* integral over triangle (v0, v1, v2) of exp(i k |x - y|) / (4 pi |x - y|) dA(y) for x
 * inside the triangle (deriv = 0), or its k-derivative (deriv = 1). */
static cplx self_integral(const double* v0, const double* v1, const double* v2,
                          const double* x, cplx k, int deriv) {
    double gx[16], gw[16];
    gauss_legendre(16, gx, gw);
    const double* v[3] = {v0, v1, v2};
    cplx total = 0.0;
    for (int e = 0; e < 3; ++e) {
        const double* p = v[e];
        const double* q = v[(e + 1) % 3];
        double t[3], px[3], qx[3], perp[3];
        sub3(q, p, t);
        double len = norm3(t);
        for (int c = 0; c < 3; ++c) t[c] /= len;
        sub3(p, x, px);
        sub3(q, x, qx);
        double sp = dot3(px, t), sq = dot3(qx, t);
        for (int c = 0; c < 3; ++c) perp[c] = px[c] - sp * t[c];
        double d = norm3(perp);
        /* u = asinh(s / d) along the edge: R = d cosh(u), d(phi) = du / cosh(u) */
        double u_p = asinh(sp / d), u_q = asinh(sq / d);
        double lo[2], hi[2];
        int pieces = 0;
        if (u_p < 0.0 && u_q > 0.0) {
            lo[0] = u_p; hi[0] = 0.0; lo[1] = 0.0; hi[1] = u_q; pieces = 2;
        } else {
            lo[0] = u_p; hi[0] = u_q; pieces = 1;
        }
        for (int s = 0; s < pieces; ++s) {
            double half = 0.5 * (hi[s] - lo[s]), mid = 0.5 * (hi[s] + lo[s]);
            for (int g = 0; g < 16; ++g) {
                double u = mid + half * gx[g];
                double R = d * cosh(u);
                cplx wv = I * k * R;
                /* value: R h(ikR) dphi = d h(ikR) du; derivative: i R^2 h'(ikR) dphi */
                cplx f = deriv ? I * d * R * hprime_fun(wv) : d * h_fun(wv);
                total += half * gw[g] * f;
            }
        }
    }
    return total / (4.0 * PI);
}

/* ---------------- the near-field rule ---------------- */

/* Conical-product rule of order m (m x m points) for the integral over triangle v of
 * g(k, |x - y|) (deriv = 0) or its k-derivative (deriv = 1); collapsed at the vertex of the
 * triangle nearest x. */
static cplx near_integral(const double v[3][3], const double* x, cplx k, int deriv, int m,
                          int kind) {
    double gx[64], gw[64];
    gauss_legendre(m, gx, gw);
    int a = 0;
    double best = 0.0;
    for (int q = 0; q < 3; ++q) {
        double d[3];
        sub3(v[q], x, d);
        double r = norm3(d);
        if (q == 0 || r < best) {
            best = r;
            a = q;
        }
    }
    const double* A = v[a];
    const double* B = v[(a + 1) % 3];
    const double* C = v[(a + 2) % 3];
    double ab[3], bc[3], nrm[3];
    sub3(B, A, ab);
    sub3(C, B, bc);
    cross3(ab, bc, nrm);
    const double twice_area = norm3(nrm);
    double un[3];
    for (int c = 0; c < 3; ++c) un[c] = nrm[c] / twice_area;
    cplx total = 0.0;
    for (int p = 0; p < m; ++p) {
        const double sp = 0.5 * (gx[p] + 1.0), wp = 0.5 * gw[p];
        for (int q = 0; q < m; ++q) {
            const double tq = 0.5 * (gx[q] + 1.0), wq = 0.5 * gw[q];
            double y[3], d[3];
            for (int c = 0; c < 3; ++c) y[c] = A[c] + sp * ab[c] + sp * tq * bc[c];
            const cplx g = kind ? (sub3(y, x, d), dl_kernel(k, d, un, deriv))
                                : (sub3(x, y, d), g_kernel(k, norm3(d), deriv));
            total += wp * wq * twice_area * sp * g;
        }
    }
    return total;
}

static int is_near(const panel_t* Pi, const panel_t* Pl) {
    double d[3];
    sub3(Pi->centroid, Pl->centroid, d);
    return norm3(d) < 2.0 * fmax(Pi->diam, Pl->diam);
}

typedef struct {
    cplx cG, cH;   /* T = cG G + cH (1/2 I + K) */
} op_t;

static op_t op_from(const double* op4) {
    op_t o;
    o.cG = op4 ? op4[0] + I * op4[1] : 1.0;
    o.cH = op4 ? op4[2] + I * op4[3] : 0.0;
    return o;
}

/* T_il(k) (deriv = 0) or dT_il/dk (deriv = 1); near != 0 selects the near-field variant. */
static cplx entry(const double* xyz, const int32_t* tri, const panel_t* Pi,
                  const panel_t* Pl, int64_t i, int64_t l, cplx k, int deriv, int near,
                  op_t op) {
    cplx s = 0.0;
    if (near && i != l && is_near(Pi, Pl)) {
        if (op.cG != 0.0) s += op.cG * near_integral(Pl->v, Pi->centroid, k, deriv, 8, 0);
        if (op.cH != 0.0) s += op.cH * near_integral(Pl->v, Pi->centroid, k, deriv, 8, 1);
        return s;
    }
    if (i == l) {
        const double* v0 = xyz + 3 * (int64_t)tri[3 * l + 0];
        const double* v1 = xyz + 3 * (int64_t)tri[3 * l + 1];
        const double* v2 = xyz + 3 * (int64_t)tri[3 * l + 2];
        if (op.cG != 0.0) s += op.cG * self_integral(v0, v1, v2, Pi->centroid, k, deriv);
        if (op.cH != 0.0 && !deriv) s += op.cH * 0.5;   /* the jump; K_ii = 0 */
        return s;
    }
    for (int q = 0; q < 7; ++q) {
        double d[3], dy[3];
        sub3(Pi->centroid, Pl->qp[q], d);
        sub3(Pl->qp[q], Pi->centroid, dy);
        cplx t = 0.0;
        if (op.cG != 0.0) t += op.cG * g_kernel(k, norm3(d), deriv);
        if (op.cH != 0.0) t += op.cH * dl_kernel(k, dy, Pl->nrm, deriv);
        s += Pl->qw[q] * t;
    }
    return s;
}

/* ---------------- exported API ---------------- */

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* The 7-point rule (barycentric points row by row, then weights). */
void oracle_rule7(double* bary21, double* w7) {
    double b[7][3], w[7];
    rule7(b, w);
    memcpy(bary21, b, sizeof(b));
    memcpy(w7, w, sizeof(w));
}

void oracle_gauss_legendre(int n, double* x, double* w) { gauss_legendre(n, x, w); }

/* Per panel: centroid (3), area (1), 7 points (21), 7 weights (7). */
void oracle_geometry(const double* xyz, int64_t nt, const int32_t* tri,
                     double* centroid, double* area, double* qp, double* qw) {
    for (int64_t l = 0; l < nt; ++l) {
        panel_t P;
        panel_geometry(xyz, tri, l, &P);
        memcpy(centroid + 3 * l, P.centroid, sizeof(P.centroid));
        area[l] = P.area;
        memcpy(qp + 21 * l, P.qp, sizeof(P.qp));
        memcpy(qw + 7 * l, P.qw, sizeof(P.qw));
    }
}

/* Self integral of triangle (v0,v1,v2) at the point x (complex k); out = (re, im). */
void oracle_self_integral(const double* v0, const double* v1, const double* v2,
                          const double* x, double k_re, double k_im, int deriv,
                          double* out) {
    cplx s = self_integral(v0, v1, v2, x, k_re + I * k_im, deriv);
    out[0] = creal(s);
    out[1] = cimag(s);
}

/* Dense A(k) (or dA/dk) for rows [r0, r1), row-major with row stride nt (complex). */
void oracle_matrix_op(const double* xyz, int64_t nt, const int32_t* tri, double k_re,
                      double k_im, int deriv, int64_t r0, int64_t r1, double* A_out,
                      int nthreads, int near, const double* op4) {
    set_threads(nthreads);
    const op_t op = op_from(op4);
    cplx k = k_re + I * k_im;
    cplx* A = (cplx*)A_out;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = r0; i < r1; ++i) {
        panel_t Pi, Pl;
        panel_geometry(xyz, tri, i, &Pi);
        for (int64_t l = 0; l < nt; ++l) {
            panel_geometry(xyz, tri, l, &Pl);
            A[(i - r0) * nt + l] = entry(xyz, tri, &Pi, &Pl, i, l, k, deriv, near, op);
        }
    }
}

void oracle_matrix(const double* xyz, int64_t nt, const int32_t* tri, double k_re,
                   double k_im, int deriv, int64_t r0, int64_t r1, double* A_out,
                   int nthreads, int near) {
    oracle_matrix_op(xyz, nt, tri, k_re, k_im, deriv, r0, r1, A_out, nthreads, near, 0);
}

/*
 * Y_j = A(z_j) V for every node j, rows [r0, r1) only (row sampling at large n).
 * z: N complex nodes (interleaved); V: n x nu complex, column-major; Y_out: for node j the
 * block Y_out + j * (r1 - r0) * nu, column-major (r1 - r0) x nu.
 */
void oracle_apply_op(const double* xyz, int64_t nt, const int32_t* tri, int N,
                     const double* z, int nu, const double* V_in, int64_t r0, int64_t r1,
                     double* Y_out, int nthreads, int near, const double* op4) {
    set_threads(nthreads);
    const op_t op = op_from(op4);
    const cplx* V = (const cplx*)V_in;
    cplx* Y = (cplx*)Y_out;
    const int64_t rows = r1 - r0;
    for (int64_t t = 0; t < (int64_t)N * rows * nu; ++t) Y[t] = 0.0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = r0; i < r1; ++i) {
        panel_t Pi, Pl;
        panel_geometry(xyz, tri, i, &Pi);
        for (int64_t l = 0; l < nt; ++l) {
            panel_geometry(xyz, tri, l, &Pl);
            for (int j = 0; j < N; ++j) {
                cplx k = z[2 * j] + I * z[2 * j + 1];
                cplx a = entry(xyz, tri, &Pi, &Pl, i, l, k, 0, near, op);
                cplx* Yj = Y + (int64_t)j * rows * nu;
                for (int c = 0; c < nu; ++c)
                    Yj[(int64_t)c * rows + (i - r0)] += a * V[(int64_t)c * nt + l];
            }
        }
    }
}

void oracle_apply(const double* xyz, int64_t nt, const int32_t* tri, int N,
                  const double* z, int nu, const double* V_in, int64_t r0, int64_t r1,
                  double* Y_out, int nthreads, int near) {
    oracle_apply_op(xyz, nt, tri, N, z, nu, V_in, r0, r1, Y_out, nthreads, near, 0);
}

/* The conical-product rule of order m (<= 64) for triangle (v0, v1, v2) at x; out = (re, im). */
void oracle_near_rule_kind(const double* v0, const double* v1, const double* v2,
                           const double* x, double k_re, double k_im, int deriv, int m,
                           int kind, double* out) {
    double v[3][3];
    for (int c = 0; c < 3; ++c) {
        v[0][c] = v0[c];
        v[1][c] = v1[c];
        v[2][c] = v2[c];
    }
    cplx s = near_integral(v, x, k_re + I * k_im, deriv, m, kind);
    out[0] = creal(s);
    out[1] = cimag(s);
}

void oracle_near_rule(const double* v0, const double* v1, const double* v2, const double* x,
                      double k_re, double k_im, int deriv, int m, double* out) {
    oracle_near_rule_kind(v0, v1, v2, x, k_re, k_im, deriv, m, 0, out);
}

/* Entries T_il(k) for count (i, l) pairs (rows[t], cols[t]); out: 2 count doubles. */
void oracle_entries(const double* xyz, int64_t nt, const int32_t* tri, double k_re,
                    double k_im, const int64_t* rows, const int64_t* cols, int64_t count,
                    double* out, int near, const double* op4) {
    const op_t op = op_from(op4);
    const cplx k = k_re + I * k_im;
    cplx* o = (cplx*)out;
    for (int64_t t = 0; t < count; ++t) {
        panel_t Pi, Pl;
        panel_geometry(xyz, tri, rows[t], &Pi);
        panel_geometry(xyz, tri, cols[t], &Pl);
        o[t] = entry(xyz, tri, &Pi, &Pl, rows[t], cols[t], k, 0, near, op);
    }
}

/* Near pairs of rows [r0, r1): counts[i - r0] = number of near panels l of row i; with
 * cols non-null, the panels themselves in increasing l, row after row (row_ptr given by
 * the caller from the counts). */
void oracle_near_pairs(const double* xyz, int64_t nt, const int32_t* tri, int64_t r0,
                       int64_t r1, int64_t* counts, const int64_t* row_ptr, int64_t* cols) {
    for (int64_t i = r0; i < r1; ++i) {
        panel_t Pi, Pl;
        panel_geometry(xyz, tri, i, &Pi);
        int64_t c = 0;
        for (int64_t l = 0; l < nt; ++l) {
            if (l == i) continue;
            panel_geometry(xyz, tri, l, &Pl);
            if (is_near(&Pi, &Pl)) {
                if (cols) cols[row_ptr[i - r0] + c] = l;
                ++c;
            }
        }
        counts[i - r0] = c;
    }
}
