// Dense eigen-decomposition of a small complex matrix (m <= 256), FP64, sequential code
// usable from host and device. Used for the Rayleigh-Ritz step of the reduced linearised
// eigenproblem (the paper solves that problem with dense methods when it is small and
// with subspace iteration / Arnoldi when it is larger; Section 3.1).
//
// Algorithm (textbook, e.g. Golub & Van Loan, Matrix Computations, Ch. 7):
//  1. Householder reduction to upper Hessenberg form, H = Q^H A Q, Q accumulated;
//  2. implicitly shifted QR iteration with single complex Wilkinson shifts (exceptional
//     shifts after 10 and 20 stalled iterations), Givens rotations chased down the
//     active block, deflation when a subdiagonal entry falls below eps times its
//     neighbours; the rotations are accumulated into Z (Schur form A = Z T Z^H);
//  3. eigenvectors of the triangular T by back substitution, mapped back with Z and
//     normalised to unit 2-norm.
#pragma once

#include <math.h>
#include <stdint.h>

#ifdef __CUDACC__
#define BEM_HD __host__ __device__
#else
#define BEM_HD
#endif

namespace bem {
namespace small {

struct zc {
  double re, im;
};

BEM_HD inline zc mk(double r, double i) {
  zc z;
  z.re = r;
  z.im = i;
  return z;
}
BEM_HD inline zc add(zc a, zc b) { return mk(a.re + b.re, a.im + b.im); }
BEM_HD inline zc sub(zc a, zc b) { return mk(a.re - b.re, a.im - b.im); }
BEM_HD inline zc mul(zc a, zc b) { return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
BEM_HD inline zc cj(zc a) { return mk(a.re, -a.im); }
BEM_HD inline zc scl(zc a, double s) { return mk(a.re * s, a.im * s); }
BEM_HD inline double abs2(zc a) { return a.re * a.re + a.im * a.im; }
BEM_HD inline double absz(zc a) { return hypot(a.re, a.im); }
BEM_HD inline double abs1(zc a) { return fabs(a.re) + fabs(a.im); }
BEM_HD inline zc dvd(zc a, zc b) {
  // Smith's algorithm
  if (fabs(b.re) >= fabs(b.im)) {
    const double r = b.im / b.re, d = b.re + b.im * r;
    return mk((a.re + a.im * r) / d, (a.im - a.re * r) / d);
  }
  const double r = b.re / b.im, d = b.im + b.re * r;
  return mk((a.re * r + a.im) / d, (a.im * r - a.re) / d);
}
// principal square root
BEM_HD inline zc csqrt_(zc a) {
  const double r = absz(a);
  if (r == 0.0) return mk(0.0, 0.0);
  if (a.re >= 0.0) {
    const double t = sqrt(0.5 * (r + a.re));
    return mk(t, 0.5 * a.im / t);
  }
  const double t = sqrt(0.5 * (r - a.re));
  return mk(0.5 * fabs(a.im) / t, a.im >= 0.0 ? t : -t);
}

// Column-major access
#define SE_A(M, i, j) (M)[(int64_t)(j) * m + (i)]

// Givens rotation [c s; -conj(s) c] (c real) with [c s; -conj(s) c] [x; y] = [r; 0].
BEM_HD inline void givens(zc x, zc y, double& c, zc& s) {
  const double ax = absz(x), ay = absz(y);
  if (ay == 0.0) {
    c = 1.0;
    s = mk(0.0, 0.0);
    return;
  }
  if (ax == 0.0) {
    c = 0.0;
    s = scl(cj(y), 1.0 / ay);   // maps [0; y] -> [|y|; 0]
    return;
  }
  const double nrm = hypot(ax, ay);
  c = ax / nrm;
  const zc ph = scl(x, 1.0 / ax);              // x / |x|
  s = scl(mul(ph, cj(y)), 1.0 / nrm);          // (x/|x|) conj(y) / nrm
}

// Eigenvalues w[0..m) and (if V != nullptr) unit eigenvectors V (m x m, column-major) of
// the column-major m x m matrix A (destroyed). Work arrays: Z (m x m). Returns 0 on
// success, the index+1 of the block that failed to converge otherwise.
BEM_HD inline int eig(int m, zc* A, zc* w, zc* V, zc* Z) {
  const double eps = 2.220446049250313e-16;
  // identity
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < m; ++i) SE_A(Z, i, j) = mk(i == j ? 1.0 : 0.0, 0.0);
  // 1. Hessenberg reduction: columns k = 0 .. m-3
  for (int k = 0; k + 2 < m; ++k) {
    double nrm2 = 0.0;
    for (int i = k + 1; i < m; ++i) nrm2 += abs2(SE_A(A, i, k));
    const double nrm = sqrt(nrm2);
    if (nrm == 0.0) continue;
    const zc x0 = SE_A(A, k + 1, k);
    const double ax0 = absz(x0);
    const zc ph = ax0 > 0.0 ? scl(x0, 1.0 / ax0) : mk(1.0, 0.0);
    const zc alpha = scl(ph, -nrm);   // new subdiagonal entry
    // v = x - alpha e1 stored in the column below the subdiagonal; v0 kept apart
    zc v0 = sub(x0, alpha);
    double vn2 = abs2(v0);
    for (int i = k + 2; i < m; ++i) vn2 += abs2(SE_A(A, i, k));
    if (vn2 == 0.0) continue;
    const double beta = 2.0 / vn2;    // P = I - beta v v^H
    // left: A[k+1:, k:] -= beta v (v^H A[k+1:, k:])
    for (int j = k; j < m; ++j) {
      zc s = mul(cj(v0), SE_A(A, k + 1, j));
      for (int i = k + 2; i < m; ++i) s = add(s, mul(cj(SE_A(A, i, k)), SE_A(A, i, j)));
      s = scl(s, beta);
      if (j == k) {
        // column k becomes (alpha, 0, ..., 0) below the diagonal; v still stored there
        continue;
      }
      SE_A(A, k + 1, j) = sub(SE_A(A, k + 1, j), mul(v0, s));
      for (int i = k + 2; i < m; ++i) SE_A(A, i, j) = sub(SE_A(A, i, j), mul(SE_A(A, i, k), s));
    }
    // right: A[:, k+1:] -= beta (A[:, k+1:] v) v^H ; Z likewise
    for (int pass = 0; pass < 2; ++pass) {
      zc* M = pass == 0 ? A : Z;
      for (int i = 0; i < m; ++i) {
        zc s = mul(SE_A(M, i, k + 1), v0);
        for (int j = k + 2; j < m; ++j) s = add(s, mul(SE_A(M, i, j), SE_A(A, j, k)));
        s = scl(s, beta);
        SE_A(M, i, k + 1) = sub(SE_A(M, i, k + 1), mul(s, cj(v0)));
        for (int j = k + 2; j < m; ++j)
          SE_A(M, i, j) = sub(SE_A(M, i, j), mul(s, cj(SE_A(A, j, k))));
      }
    }
    SE_A(A, k + 1, k) = alpha;
    for (int i = k + 2; i < m; ++i) SE_A(A, i, k) = mk(0.0, 0.0);
  }
  // 2. shifted QR on the Hessenberg matrix (full Schur form)
  int ihi = m - 1;
  int iter = 0;
  while (ihi >= 0) {
    int l = ihi;
    while (l > 0) {
      const double tst = abs1(SE_A(A, l - 1, l - 1)) + abs1(SE_A(A, l, l));
      if (abs1(SE_A(A, l, l - 1)) <= eps * (tst > 0.0 ? tst : 1.0)) {
        SE_A(A, l, l - 1) = mk(0.0, 0.0);
        break;
      }
      --l;
    }
    if (l == ihi) {   // 1 x 1 block converged
      w[ihi] = SE_A(A, ihi, ihi);
      --ihi;
      iter = 0;
      continue;
    }
    if (++iter > 60 * m) return ihi + 1;
    // shift: eigenvalue of the trailing 2 x 2 closer to its last diagonal entry
    zc mu;
    if (iter % 11 == 10) {
      const double e = abs1(SE_A(A, ihi, ihi - 1));
      mu = add(SE_A(A, ihi, ihi), mk(0.75 * e, -0.4375 * e));   // exceptional shift
    } else {
      const zc a = SE_A(A, ihi - 1, ihi - 1), b = SE_A(A, ihi - 1, ihi);
      const zc c = SE_A(A, ihi, ihi - 1), d = SE_A(A, ihi, ihi);
      const zc tr2 = scl(add(a, d), 0.5);
      const zc hd = scl(sub(a, d), 0.5);
      const zc disc = csqrt_(add(mul(hd, hd), mul(b, c)));
      const zc e1 = add(tr2, disc), e2 = sub(tr2, disc);
      mu = abs2(sub(e1, d)) <= abs2(sub(e2, d)) ? e1 : e2;
    }
    // implicit QR sweep on rows/cols l .. ihi
    zc x = sub(SE_A(A, l, l), mu);
    zc y = SE_A(A, l + 1, l);
    for (int k = l; k < ihi; ++k) {
      double c;
      zc s;
      givens(x, y, c, s);
      // rows k, k+1: columns from max(l, k-1) to m-1
      for (int j = (k > l ? k - 1 : l); j < m; ++j) {
        const zc t1 = SE_A(A, k, j), t2 = SE_A(A, k + 1, j);
        SE_A(A, k, j) = add(scl(t1, c), mul(s, t2));
        SE_A(A, k + 1, j) = sub(scl(t2, c), mul(cj(s), t1));
      }
      // columns k, k+1: rows 0 .. min(k+2, ihi)
      const int rmax = (k + 2 < ihi ? k + 2 : ihi);
      for (int i = 0; i <= rmax; ++i) {
        const zc t1 = SE_A(A, i, k), t2 = SE_A(A, i, k + 1);
        SE_A(A, i, k) = add(scl(t1, c), mul(cj(s), t2));
        SE_A(A, i, k + 1) = sub(scl(t2, c), mul(s, t1));
      }
      for (int i = 0; i < m; ++i) {
        const zc t1 = SE_A(Z, i, k), t2 = SE_A(Z, i, k + 1);
        SE_A(Z, i, k) = add(scl(t1, c), mul(cj(s), t2));
        SE_A(Z, i, k + 1) = sub(scl(t2, c), mul(s, t1));
      }
      if (k + 1 < ihi) {
        x = SE_A(A, k + 1, k);
        y = SE_A(A, k + 2, k);
      }
    }
  }
  if (!V) return 0;
  // 3. eigenvectors of T (upper triangular, in A) by back substitution, then Z y
  double tnorm = 0.0;
  for (int j = 0; j < m; ++j)
    for (int i = 0; i <= j; ++i) tnorm = fmax(tnorm, abs1(SE_A(A, i, j)));
  const double small_pivot = eps * (tnorm > 0.0 ? tnorm : 1.0);
  for (int e = 0; e < m; ++e) {
    zc* y = &SE_A(V, 0, e);
    for (int i = 0; i < m; ++i) y[i] = mk(0.0, 0.0);
    y[e] = mk(1.0, 0.0);
    const zc lam = SE_A(A, e, e);
    for (int i = e - 1; i >= 0; --i) {
      zc s = mk(0.0, 0.0);
      for (int k = i + 1; k <= e; ++k) s = add(s, mul(SE_A(A, i, k), y[k]));
      zc dnm = sub(SE_A(A, i, i), lam);
      if (abs1(dnm) < small_pivot) dnm = mk(small_pivot, 0.0);
      y[i] = dvd(mk(-s.re, -s.im), dnm);
    }
  }
  // T is no longer needed: A <- Z Y (y_e has zeros below row e), then normalise into V
  for (int e = 0; e < m; ++e) {
    const zc* y = &SE_A(V, 0, e);
    for (int i = 0; i < m; ++i) {
      zc s = mk(0.0, 0.0);
      for (int k = 0; k <= e; ++k) s = add(s, mul(SE_A(Z, i, k), y[k]));
      SE_A(A, i, e) = s;
    }
  }
  for (int e = 0; e < m; ++e) {
    double n2 = 0.0;
    for (int i = 0; i < m; ++i) n2 += abs2(SE_A(A, i, e));
    const double inv = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
    for (int i = 0; i < m; ++i) SE_A(V, i, e) = scl(SE_A(A, i, e), inv);
  }
  return 0;
}

#undef SE_A

}  // namespace small
}  // namespace bem
