// The boundary operator T(k) = c_G G(k) + c_H (1/2 I + K(k)) (the general form of Eq. HelmBIM:
// Dirichlet conditions take the single layer G, Neumann the double layer with its jump,
// H = 1/2 I + K, Robin a combination), with the kernels, at y - x = d, r = |d|, n the unit
// normal of the source panel,
//   G: exp(i k r) / (4 pi r),    K: exp(i k r) (i k r - 1) (d . n) / (4 pi r^3),
// and their k-derivatives i exp(i k r) / (4 pi) and -k exp(i k r) (d . n) / (4 pi r).
// K vanishes on the panel's own plane, so the self entry of H is the jump 1/2.
#pragma once

namespace bem {

struct OpCoef {
  double cgr = 1.0, cgi = 0.0;   // c_G
  double chr = 0.0, chi = 0.0;   // c_H
};

__host__ __device__ inline bool op_single(const OpCoef& o) {
  return o.cgr == 1.0 && o.cgi == 0.0 && o.chr == 0.0 && o.chi == 0.0;
}

// Factor F with T's point term = w exp(i k r) / (4 pi r) * F:
//   F = c_G + c_H s (i k r - 1),  s = (d . n) / r^2,  k = kr + i ki, so
//   s (i k r - 1) = -s (1 + ki r) + i s kr r.
template <typename T>
__host__ __device__ inline void op_factor(const OpCoef& o, T s, T kr_r, T ki_r, T& fr, T& fi) {
  const T a = -s * (T(1) + ki_r), b = s * kr_r;
  fr = T(o.cgr) + T(o.chr) * a - T(o.chi) * b;
  fi = T(o.cgi) + T(o.chr) * b + T(o.chi) * a;
}

// Factor D of the k-derivative with the point term w exp(i k r) / (4 pi) * D:
//   D = i c_G - c_H k (d . n) / r = i c_G - c_H k s r.
__host__ __device__ inline void op_dfactor(const OpCoef& o, double s_r, double kr, double ki,
                                           double& dr, double& di) {
  // -c_H k s r with k = kr + i ki
  const double pr = -(o.chr * kr - o.chi * ki) * s_r, pi_ = -(o.chr * ki + o.chi * kr) * s_r;
  dr = -o.cgi + pr;
  di = o.cgr + pi_;
}

#ifdef __CUDACC__
// acc += w * T's point term at d = y - x (FP64): w exp(i k r) / r * F, or for the
// k-derivative w exp(i k r) * D (w the quadrature weight including 1 / (4 pi)); nl the
// source panel's unit normal.
__device__ inline void op_point64(double2& acc, const OpCoef& op, double w, double dx, double dy,
                                  double dz, double nx, double ny, double nz, double kr,
                                  double ki, bool deriv) {
  const double r = sqrt(dx * dx + dy * dy + dz * dz);
  double sn, cs;
  sincos(kr * r, &sn, &cs);
  const double e = w * exp(-ki * r);
  const double dn = dx * nx + dy * ny + dz * nz;
  double fr, fi;
  if (deriv) {
    op_dfactor(op, dn / r, kr, ki, fr, fi);
    const double br = e * cs, bi = e * sn;
    acc.x += br * fr - bi * fi;
    acc.y += br * fi + bi * fr;
  } else {
    op_factor(op, dn / (r * r), kr * r, ki * r, fr, fi);
    const double br = e * cs / r, bi = e * sn / r;
    acc.x += br * fr - bi * fi;
    acc.y += br * fi + bi * fr;
  }
}
#endif

}  // namespace bem
