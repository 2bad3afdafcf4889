// Particle surfaces on the device: ellipsoids and spherical-harmonic coefficient surfaces (Section 3,
// Eqs. 31, 36, 37), shared by the geometry set-up and the magnetostatic coupling.
#pragma once

#include "common.cuh"

namespace rbs {

// Particle surfaces.  An ellipsoid x = D s (D = diag(a, b, c)): J = |cof(D) s| is the area per unit
// solid angle (W / sin(theta) of Eq. 36) and the normal is D^{-1} s normalised.  A coefficient
// surface x = sum c_nm Y_nm (Eq. 31) in the library's basis order (m = 0..p_g, n = m..p_g, cos then
// sin, orthonormal, no Condon-Shortley sign): tangents by spectral differentiation (Eq. 37) with the
// regular forms dPbar_n^m/dtheta = (sqrt((n+m)(n-m+1)) Pbar_n^{m-1} - sqrt((n+m+1)(n-m)) Pbar_n^{m+1})/2,
// dPbar_n^0/dtheta = -sqrt(n(n+1)) Pbar_n^1 and Pbar_n^m / sin(theta) from the n-recurrence started at
// sin^(m-1)(theta), so J = |x_theta x (x_phi / sin(theta))| holds at the poles too.  The body frame of a
// coefficient surface is centred at its area centroid (shift).
constexpr int kMaxShapeDegree = RBS_MAX_SHAPE_DEGREE;

struct ShapeRef {
  int kind;  // 0 ellipsoid, 1 coefficient surface
  double a, b, c;
  const double* coef;
  int pg;
  double ox, oy, oz;  // centroid shift
};

__device__ inline ShapeRef shape_ref(int s, const int* kind, const double* axes, const int* pg, const long long* coef_off,
                              const double* coef, const double* shift) {
  ShapeRef r;
  r.kind = kind[s];
  r.a = axes[3 * s];
  r.b = axes[3 * s + 1];
  r.c = axes[3 * s + 2];
  r.pg = pg[s];
  r.coef = coef + (coef_off[s] >= 0 ? coef_off[s] : 0);
  r.ox = shift[3 * s];
  r.oy = shift[3 * s + 1];
  r.oz = shift[3 * s + 2];
  return r;
}

// One column m of normalised associated Legendre values Pbar_n^m(t), n = m..pg (index n), and of
// Pbar_n^m / sin(theta) (m >= 1); pmm_prev is Pbar_{m-1}^{m-1} on entry, Pbar_m^m on exit.
__device__ inline void legendre_column(int m, int pg, double t, double st, double& pmm, double* P, double* Q) {
  double qmm = 0.0;
  if (m > 0) {
    qmm = sqrt((2.0 * m + 1.0) / (2.0 * m)) * pmm;  // Pbar_m^m / sin
    pmm = qmm * st;
  }
  for (int n = 0; n <= pg; ++n) P[n] = Q[n] = 0.0;
  P[m] = pmm;
  Q[m] = qmm;
  if (m + 1 <= pg) {
    P[m + 1] = sqrt(2.0 * m + 3.0) * t * pmm;
    Q[m + 1] = sqrt(2.0 * m + 3.0) * t * qmm;
  }
  for (int n = m + 2; n <= pg; ++n) {
    const double a = sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
    const double b = sqrt(((n - 1.0) * (n - 1.0) - (double)m * m) / (4.0 * (n - 1.0) * (n - 1.0) - 1.0));
    P[n] = a * (t * P[n - 1] - b * P[n - 2]);
    Q[n] = a * (t * Q[n - 1] - b * Q[n - 2]);
  }
}

// x, J and the unit normal at parameter point s; with xt and xp non-null also the tangents x_theta and
// x_phi / sin(theta) (phi = atan2(s_y, s_x), so phi = 0 at the poles).
__device__ inline void eval_surface(const ShapeRef& S, double sx, double sy, double sz, double* x, double* J, double* nrm,
                                    double* xt_out = nullptr, double* xp_out = nullptr) {
  if (S.kind == 0) {
    x[0] = S.a * sx;
    x[1] = S.b * sy;
    x[2] = S.c * sz;
    const double cx = S.b * S.c * sx, cy = S.a * S.c * sy, cz = S.a * S.b * sz;
    *J = sqrt(cx * cx + cy * cy + cz * cz);
    double gx = sx / S.a, gy = sy / S.b, gz = sz / S.c;
    const double gn = rsqrt(gx * gx + gy * gy + gz * gz);
    nrm[0] = gx * gn;
    nrm[1] = gy * gn;
    nrm[2] = gz * gn;
    if (xt_out) {
      const double st = sqrt(sx * sx + sy * sy);
      const double cp = st > 0.0 ? sx / st : 1.0, sp = st > 0.0 ? sy / st : 0.0;
      xt_out[0] = S.a * sz * cp;
      xt_out[1] = S.b * sz * sp;
      xt_out[2] = -S.c * st;
      xp_out[0] = -S.a * sp;
      xp_out[1] = S.b * cp;
      xp_out[2] = 0.0;
    }
    return;
  }
  const double t = fmin(1.0, fmax(-1.0, sz)), st = sqrt(fmax(0.0, sx * sx + sy * sy));
  const double phi = atan2(sy, sx);
  const int pg = S.pg;
  const int nc = (pg + 1) * (pg + 1);
  double P0[kMaxShapeDegree + 1], P1[kMaxShapeDegree + 1], P2[kMaxShapeDegree + 1];
  double Q0[kMaxShapeDegree + 1], Q1[kMaxShapeDegree + 1], Q2[kMaxShapeDegree + 1];
  double* Pm = P0;  // column m - 1
  double* Pc = P1;  // column m
  double* Pp = P2;  // column m + 1
  double* Qm = Q0;
  double* Qc = Q1;
  double* Qp = Q2;
  double pmm = 0.28209479177387814;  // Pbar_0^0 = 1 / sqrt(4 pi)
  legendre_column(0, pg, t, st, pmm, Pc, Qc);
  double pmm_next = pmm;
  if (pg >= 1) legendre_column(1, pg, t, st, pmm_next, Pp, Qp);
  double xv[3] = {0, 0, 0}, xt[3] = {0, 0, 0}, xp[3] = {0, 0, 0};
  const double r2 = 1.4142135623730951;
  int b = 0;
  for (int m = 0; m <= pg; ++m) {
    double cm = 1.0, sm = 0.0;
    if (m > 0) sincos(m * phi, &sm, &cm);
    for (int n = m; n <= pg; ++n) {
      double dP;
      if (m == 0) {
        dP = (n >= 1) ? -sqrt(n * (n + 1.0)) * Pp[n] : 0.0;
      } else {
        const double up = (m + 1 <= n) ? sqrt((n + m + 1.0) * (n - m)) * Pp[n] : 0.0;
        dP = 0.5 * (sqrt((n + m) * (n - m + 1.0)) * Pm[n] - up);
      }
      if (m == 0) {
        for (int q = 0; q < 3; ++q) {
          const double cf = S.coef[q * nc + b];
          xv[q] += cf * Pc[n];
          xt[q] += cf * dP;
        }
        ++b;
      } else {
        for (int q = 0; q < 3; ++q) {
          const double cc = S.coef[q * nc + b], cs = S.coef[q * nc + b + 1];
          xv[q] += r2 * Pc[n] * (cc * cm + cs * sm);
          xt[q] += r2 * dP * (cc * cm + cs * sm);
          xp[q] += r2 * m * Qc[n] * (-cc * sm + cs * cm);
        }
        b += 2;
      }
    }
    // roll the columns: m -> m + 1
    double* tp = Pm;
    Pm = Pc;
    Pc = Pp;
    Pp = tp;
    tp = Qm;
    Qm = Qc;
    Qc = Qp;
    Qp = tp;
    if (m + 2 <= pg) legendre_column(m + 2, pg, t, st, pmm_next, Pp, Qp);
  }
  x[0] = xv[0] - S.ox;
  x[1] = xv[1] - S.oy;
  x[2] = xv[2] - S.oz;
  const double c0 = xt[1] * xp[2] - xt[2] * xp[1], c1 = xt[2] * xp[0] - xt[0] * xp[2], c2 = xt[0] * xp[1] - xt[1] * xp[0];
  *J = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
  nrm[0] = c0 / *J;
  nrm[1] = c1 / *J;
  nrm[2] = c2 / *J;
  if (xt_out) {
    for (int q = 0; q < 3; ++q) {
      xt_out[q] = xt[q];
      xp_out[q] = xp[q];
    }
  }
}

#define RBS_SHAPE_ARGS const int *sh_kind, const double *sh_axes, const int *sh_pg, const long long *sh_coef_off, \
                       const double *sh_coef, const double *sh_shift
#define RBS_SHAPE_PASS c.d_sh_kind.ptr, c.d_sh_axes.ptr, c.d_sh_pg.ptr, c.d_sh_coef_off.ptr, c.d_sh_coef.ptr, \
                       c.d_sh_shift.ptr
#define RBS_SHAPE_REF(s) shape_ref((s), sh_kind, sh_axes, sh_pg, sh_coef_off, sh_coef, sh_shift)

}  // namespace rbs
