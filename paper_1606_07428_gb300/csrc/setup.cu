// Geometry set-up: grids (Section 3, Eq. 33), surface nodes, normals and weights (Eqs. 35-36),
// moments (Eq. 18), the singular-rule and upsampling interpolation operators, the body-frame self
// blocks of each distinct shape (Section 3.1, Eq. 38), the block-diagonal preconditioner
// (Section 3.2), the near-pair list and the smooth pair-sum work list.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <tuple>
#include <unordered_map>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "surface.cuh"

namespace rbs {

// ------------------------------------------------------------------------------------------
// Host constants: Gauss-Legendre rules by Newton's method on the Legendre three-term recurrence
// (initial guesses cos(pi (i + 3/4) / (n + 1/2))); weights 2 / ((1 - t^2) P_n'(t)^2).

void gauss_legendre_newton(int n, std::vector<double>& t, std::vector<double>& w) {
  t.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double x = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      double pn = (n == 1) ? x : p1, pn1 = (n == 1) ? 1.0 : p0;
      dp = n * (x * pn - pn1) / (x * x - 1.0);
      double dx = pn / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) {
        // one more evaluation of the derivative at the converged node
        p0 = 1.0;
        p1 = x;
        for (int k = 2; k <= n; ++k) {
          double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = pk;
        }
        pn = (n == 1) ? x : p1;
        pn1 = (n == 1) ? 1.0 : p0;
        dp = n * (x * pn - pn1) / (x * x - 1.0);
        break;
      }
    }
    t[n - 1 - i] = x;  // ascending
    w[n - 1 - i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

// ------------------------------------------------------------------------------------------
// Device helpers

// Real orthonormal spherical harmonics (Eq. 32 with cos / sin in place of e^{i m phi}) of degree
// <= p and order <= mmax at (cos_t, sin_t, phi), written to out[b * stride] in the library's own
// basis order: m = 0..mmax, n = m..p, cos variant then (m > 0) sin variant.
__device__ void real_sh_eval(int p, int mmax, double ct, double st, double phi, double* out, long long stride) {
  double pmm = 0.28209479177387814;  // 1 / sqrt(4 pi)
  int b = 0;
  const double sq2 = 1.4142135623730951;
  for (int m = 0; m <= mmax; ++m) {
    if (m > 0) pmm *= sqrt((2.0 * m + 1.0) / (2.0 * m)) * st;
    double cm = 1.0, sm = 0.0;
    if (m > 0) {
      sincos(m * phi, &sm, &cm);
      cm *= sq2;
      sm *= sq2;
    }
    double pnm2 = 0.0, pnm1 = pmm;
    for (int n = m; n <= p; ++n) {
      double pn;
      if (n == m) {
        pn = pmm;
      } else if (n == m + 1) {
        pn = sqrt(2.0 * m + 3.0) * ct * pmm;
      } else {
        double a = sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
        double bb = sqrt(((n - 1.0) * (n - 1.0) - (double)m * m) / (4.0 * (n - 1.0) * (n - 1.0) - 1.0));
        pn = a * (ct * pnm1 - bb * pnm2);
      }
      if (n > m) {
        pnm2 = pnm1;
        pnm1 = pn;
      }
      if (m == 0) {
        out[(long long)(b++) * stride] = pn;
      } else {
        out[(long long)(b++) * stride] = pn * cm;
        out[(long long)(b++) * stride] = pn * sm;
      }
    }
  }
}

// Y at a set of points given as unit vectors (x, y, z, *): Y[pt * nbasis + b].
__global__ void k_sh_at_points(int p, int mmax, int nbasis, const double4* pts, int npts, double* Y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npts) return;
  double4 s = pts[i];
  double ct = s.z, st = sqrt(fmax(0.0, s.x * s.x + s.y * s.y));
  double phi = atan2(s.y, s.x);
  real_sh_eval(p, mmax, ct, st, phi, Y + (long long)i * nbasis, 1);
}

// Grid points of a (p, nphi) grid as unit vectors, w = unit-sphere weight (2 pi / nphi) lambda_j.
__global__ void k_grid_points(int p, int nphi, const double* t, const double* lam, double4* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int np = (p + 1) * nphi;
  if (i >= np) return;
  int j = i / nphi, k = i % nphi;
  double ct = t[j], st = sqrt(fmax(0.0, 1.0 - ct * ct));
  double sp, cp;
  sincospi(2.0 * k / nphi, &sp, &cp);
  out[i] = make_double4(st * cp, st * sp, ct, 2.0 * kPi / nphi * lam[j]);
}

// Analysis matrix An[b * np + node] = Y_b(node) * weight(node), from Yg[node * nbasis + b].
__global__ void k_analysis(int np, int nbasis, const double* Yg, const double4* gp, double* An) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)np * nbasis) return;
  int b = (int)(i / np), node = (int)(i % np);
  An[i] = Yg[(long long)node * nbasis + b] * gp[node].w;
}



// Surface nodes of all particles (lab frame): x = c + R x_b(s), n = R n_b(s) and weight
// (2 pi / nphi) lambda_j J(s) (Eq. 35 with W / sin(theta) = J), s the grid point of Eq. 33.
__global__ void k_nodes(int n, const long long* offset, const int* pvec, const int* nphivec, const int* shape_of,
                        RBS_SHAPE_ARGS, const double* centre, const double* rot, const long long* gtab_off,
                        const double* gtab, double4* x, double4* nrm, int* pid) {
  for (int i = blockIdx.y; i < n; i += gridDim.y) {
    const long long o = offset[i];
    const int nphi = nphivec[i], p = pvec[i];
    const int np = (p + 1) * nphi;
    const double* t = gtab + gtab_off[i];
    const double* lam = t + (p + 1);
    const ShapeRef S = RBS_SHAPE_REF(shape_of[i]);
    const double* R = rot + 9 * i;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < np; l += gridDim.x * blockDim.x) {
      const int j = l / nphi, k = l % nphi;
      const double ct = t[j], st = sqrt(fmax(0.0, 1.0 - ct * ct));
      double sp, cp;
      sincospi(2.0 * k / nphi, &sp, &cp);
      double xb[3], J, nb[3];
      eval_surface(S, st * cp, st * sp, ct, xb, &J, nb);
      const double w = 2.0 * kPi / nphi * lam[j] * J;
      x[o + l] = make_double4(R[0] * xb[0] + R[1] * xb[1] + R[2] * xb[2] + centre[3 * i],
                              R[3] * xb[0] + R[4] * xb[1] + R[5] * xb[2] + centre[3 * i + 1],
                              R[6] * xb[0] + R[7] * xb[1] + R[8] * xb[2] + centre[3 * i + 2], w);
      nrm[o + l] = make_double4(R[0] * nb[0] + R[1] * nb[1] + R[2] * nb[2], R[3] * nb[0] + R[4] * nb[1] + R[5] * nb[2],
                                R[6] * nb[0] + R[7] * nb[1] + R[8] * nb[2], 0.0);
      pid[o + l] = i;
    }
  }
}

// Coefficient surfaces: area centroid on the shape's own grid (the shift), then the largest and
// smallest centroid distance over the nodes of its upsampled grid, the smallest J over both grids and
// the enclosed volume sum w x.n / 3 (negative for an inward parametrisation).  One block per shape.
struct ShapeGrid {
  int s, p, nphi, pup;
  long long t, t_up;  // offsets of (t, lambda) in the grid table
};

__global__ void k_shape_extent(const ShapeGrid* sg, RBS_SHAPE_ARGS, double* shift_out, const double* gtab,
                               double* diag) {
  __shared__ double red[5][256];
  const ShapeGrid G = sg[blockIdx.x];
  const int s = G.s;
  ShapeRef S = RBS_SHAPE_REF(s);
  S.ox = S.oy = S.oz = 0.0;
  const int p = G.p, nphi = G.nphi;
  const double* t = gtab + G.t;
  const double* lam = t + (p + 1);
  double acc[5] = {0, 0, 0, 0, 0};
  double jmin = INFINITY;
  for (int l = threadIdx.x; l < (p + 1) * nphi; l += blockDim.x) {
    const int j = l / nphi, k = l % nphi;
    const double ct = t[j], st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double ssp, scp;
    sincospi(2.0 * k / nphi, &ssp, &scp);
    double xb[3], J, nb[3];
    eval_surface(S, st * scp, st * ssp, ct, xb, &J, nb);
    const double w = 2.0 * kPi / nphi * lam[j] * J;
    acc[0] += w * xb[0];
    acc[1] += w * xb[1];
    acc[2] += w * xb[2];
    acc[3] += w;
    acc[4] += w * (xb[0] * nb[0] + xb[1] * nb[1] + xb[2] * nb[2]) / 3.0;
    jmin = fmin(jmin, J);
  }
  for (int q = 0; q < 5; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int q = 0; q < 5; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
    __syncthreads();
  }
  S.ox = red[0][0] / red[3][0];
  S.oy = red[1][0] / red[3][0];
  S.oz = red[2][0] / red[3][0];
  const double vol = red[4][0];
  __syncthreads();
  if (threadIdx.x == 0) {
    shift_out[3 * s] = S.ox;
    shift_out[3 * s + 1] = S.oy;
    shift_out[3 * s + 2] = S.oz;
  }
  const int pup = G.pup, nphi_up = nphi + 2 * (pup - p);
  const double* tu = gtab + G.t_up;
  double mx = 0.0, mn = INFINITY;
  for (int l = threadIdx.x; l < (pup + 1) * nphi_up; l += blockDim.x) {
    const int j = l / nphi_up, k = l % nphi_up;
    const double ct = tu[j], st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double ssp, scp;
    sincospi(2.0 * k / nphi_up, &ssp, &scp);
    double xb[3], J, nb[3];
    eval_surface(S, st * scp, st * ssp, ct, xb, &J, nb);
    const double d = sqrt(xb[0] * xb[0] + xb[1] * xb[1] + xb[2] * xb[2]);
    mx = fmax(mx, d);
    mn = fmin(mn, d);
    jmin = fmin(jmin, J);
  }
  red[0][threadIdx.x] = mx;
  red[1][threadIdx.x] = mn;
  red[2][threadIdx.x] = jmin;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      red[0][threadIdx.x] = fmax(red[0][threadIdx.x], red[0][threadIdx.x + h]);
      red[1][threadIdx.x] = fmin(red[1][threadIdx.x], red[1][threadIdx.x + h]);
      red[2][threadIdx.x] = fmin(red[2][threadIdx.x], red[2][threadIdx.x + h]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    diag[4 * blockIdx.x] = red[0][0];
    diag[4 * blockIdx.x + 1] = red[1][0];
    diag[4 * blockIdx.x + 2] = red[2][0];
    diag[4 * blockIdx.x + 3] = vol;
  }
}

// Body-frame nodes (x_b, weight) of one shape on its own grid.
__global__ void k_body_nodes(int np, int nphi, const double* t, const double* lam, int shape, RBS_SHAPE_ARGS,
                             double4* out) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= np) return;
  const ShapeRef S = RBS_SHAPE_REF(shape);
  const int j = l / nphi, k = l % nphi;
  const double ct = t[j], st = sqrt(fmax(0.0, 1.0 - ct * ct));
  double sp, cp;
  sincospi(2.0 * k / nphi, &sp, &cp);
  double xb[3], J, nb[3];
  eval_surface(S, st * cp, st * sp, ct, xb, &J, nb);
  out[l] = make_double4(xb[0], xb[1], xb[2], 2.0 * kPi / nphi * lam[j] * J);
}

// Node positions as unevaluated float32 sums hi + lo (hi = the position rounded to float32, lo = the
// rounded remainder), with the particle id in hi.w, and the normals in float32, for the packed
// float32 pair kernels.
// For the double-float pair kernels: positions split exactly into three float32 parts
// (v = hi + mid + lo: each part is the float32 rounding of what the previous ones leave, and 72 bits
// hold the 53 of a float64), and normals as hi + lo pairs.
__global__ void k_split_positions(long long N, const double4* x, const double4* nrm, const int* pid, float4* hi,
                                  float4* lo, float4* n32, float4* x3h, float4* x3m, float4* x3l, float4* nh,
                                  float4* nl) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= N) return;
  const double4 p = x[t], q = nrm[t];
  const float hx = (float)p.x, hy = (float)p.y, hz = (float)p.z;
  const float pw = __int_as_float(pid[t]);
  hi[t] = make_float4(hx, hy, hz, pw);
  lo[t] = make_float4((float)(p.x - (double)hx), (float)(p.y - (double)hy), (float)(p.z - (double)hz), 0.0f);
  n32[t] = make_float4((float)q.x, (float)q.y, (float)q.z, 0.0f);
  const double rx = p.x - (double)hx, ry = p.y - (double)hy, rz = p.z - (double)hz;
  const float mx = (float)rx, my = (float)ry, mz = (float)rz;
  x3h[t] = make_float4(hx, hy, hz, pw);
  x3m[t] = make_float4(mx, my, mz, 0.0f);
  x3l[t] = make_float4((float)(rx - (double)mx), (float)(ry - (double)my), (float)(rz - (double)mz), 0.0f);
  const float ax = (float)q.x, ay = (float)q.y, az = (float)q.z;
  nh[t] = make_float4(ax, ay, az, 0.0f);
  nl[t] = make_float4((float)(q.x - (double)ax), (float)(q.y - (double)ay), (float)(q.z - (double)az), 0.0f);
}

// Per-particle area |Gamma_i| = sum w and inverse moment tensor (Eq. 18), one block per particle.
__global__ void k_moments(int n, const long long* offset, const double4* x, const double* centre, double* area,
                          double* tauinv) {
  int i = blockIdx.x;
  if (i >= n) return;
  __shared__ double red[7][256];
  // sums of w, w rx^2, w ry^2, w rz^2, w rx ry, w rx rz, w ry rz
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  double accyz = 0.0;
  double cx = centre[3 * i], cy = centre[3 * i + 1], cz = centre[3 * i + 2];
  for (long long s = offset[i] + threadIdx.x; s < offset[i + 1]; s += blockDim.x) {
    double4 p = x[s];
    double rx = p.x - cx, ry = p.y - cy, rz = p.z - cz, w = p.w;
    acc[0] += w;
    acc[1] += w * rx * rx;
    acc[2] += w * ry * ry;
    acc[3] += w * rz * rz;
    acc[4] += w * rx * ry;
    acc[5] += w * rx * rz;
    accyz += w * ry * rz;
  }
  acc[6] = accyz;
  for (int q = 0; q < 7; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int q = 0; q < 7; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double W = red[0][0], xx = red[1][0], yy = red[2][0], zz = red[3][0], xy = red[4][0], xz = red[5][0],
           yz = red[6][0];
    double t[9] = {yy + zz, -xy, -xz, -xy, xx + zz, -yz, -xz, -yz, xx + yy};
    double c00 = t[4] * t[8] - t[5] * t[7], c01 = t[5] * t[6] - t[3] * t[8], c02 = t[3] * t[7] - t[4] * t[6];
    double det = t[0] * c00 + t[1] * c01 + t[2] * c02;
    double inv[9] = {c00, t[2] * t[7] - t[1] * t[8], t[1] * t[5] - t[2] * t[4],
                     c01, t[0] * t[8] - t[2] * t[6], t[2] * t[3] - t[0] * t[5],
                     c02, t[1] * t[6] - t[0] * t[7], t[0] * t[4] - t[1] * t[3]};
    area[i] = W;
    for (int q = 0; q < 9; ++q) tauinv[9 * i + q] = inv[q] / det;
  }
}

// Kernel-value matrix of the singular rule for one shape and polar index j, azimuthal k < nkc:
// C[((kind * nkc + k) * 9 + 3 al + be) * nrot + a] = omega_a J(s_a) kernel_{al be}(x_t - x(s_a)),
// target t = (j, k), rotated point s_a = R_z(phi_k) rotpts[j][a]; kind 0 = traction (Eqs. 13, 22),
// kind 1 = Stokeslet (Eq. 10).
__global__ void k_self_kernel_values(int nphi, int nkc, int nrot, double tj, const int* shape_ids, RBS_SHAPE_ARGS,
                                     const double4* rotpts_j, double* Cbase, size_t perC) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  int k = blockIdx.y;
  if (a >= nrot) return;
  const ShapeRef S = RBS_SHAPE_REF(shape_ids[blockIdx.z]);
  double* C = Cbase + perC * blockIdx.z;
  double sp, cp;
  sincospi(2.0 * k / nphi, &sp, &cp);
  const double4 q = rotpts_j[a];
  const double st = sqrt(fmax(0.0, 1.0 - tj * tj));
  double xt[3], Jt, g[3];
  eval_surface(S, st * cp, st * sp, tj, xt, &Jt, g);
  double y[3], J, ny[3];
  eval_surface(S, cp * q.x - sp * q.y, sp * q.x + cp * q.y, q.z, y, &J, ny);
  const double r0 = xt[0] - y[0], r1 = xt[1] - y[1], r2 = xt[2] - y[2];
  const double wJ = q.w * J;
  const double d2 = r0 * r0 + r1 * r1 + r2 * r2;
  const double inv = rsqrt(d2);
  const double inv2 = inv * inv;
  const double rr[3] = {r0, r1, r2};
  const double rn = r0 * g[0] + r1 * g[1] + r2 * g[2];
  const double ck = -3.0 / (4.0 * kPi) * rn * inv2 * inv2 * inv * wJ;
  const double cs = wJ / (8.0 * kPi);
  for (int al = 0; al < 3; ++al)
    for (int be = 0; be < 3; ++be) {
      const double rab = rr[al] * rr[be];
      C[((long long)(0 * nkc + k) * 9 + 3 * al + be) * nrot + a] = ck * rab;
      C[((long long)(1 * nkc + k) * 9 + 3 * al + be) * nrot + a] = cs * ((al == be ? inv : 0.0) + rab * inv2 * inv);
    }
}

// Scatter G[((kind * nkc + k) * 9 + 3 al + be) * np + (j' nphi + k')] into the body blocks:
// stored row 3 r + al, r = j nkc + k (the node (j, k) itself when nkc = nphi, its representative
// index when nkc = nk); column 3 s + be, s = j' nphi + (k' + k) mod nphi.
__global__ void k_self_scatter(int nphi, int nkc, int np, int j, const double* Gbase, size_t perG,
                               const long long* block_off, double* BKbase, double* BSbase) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const double* G = Gbase + perG * blockIdx.y;
  double* BK = BKbase + block_off[blockIdx.y];
  double* BS = BSbase + block_off[blockIdx.y];
  long long total = 2LL * nkc * 9 * np;
  if (i >= total) return;
  int col = (int)(i % np);
  long long row = i / np;
  int ab = (int)(row % 9);
  long long kk = row / 9;
  int k = (int)(kk % nkc), kind = (int)(kk / nkc);
  int al = ab / 3, be = ab % 3;
  int jp = col / nphi, kp = col % nphi;
  int r = j * nkc + k, s = jp * nphi + (kp + k) % nphi;
  double* B = kind == 0 ? BK : BS;
  B[(long long)(3 * r + al) * (3 * np) + 3 * s + be] = G[i];
}

// Preconditioner matrix before inversion: M = 1/2 I + K0 + L0 in the body frame, with
// L0_ts = w_s (I - [r_t]x [r_s]x) (Eq. 26 written as a block; r the body-frame node).
// Stored row 3 r + al belongs to node (r / nk) nphi + r % nk (the node r itself when nk = nphi).
__global__ void k_precond_matrix(int np, int nphi, int nk, int rows, const double4* body, const double* BK, double* M) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long dim = 3LL * np;
  if (i >= (long long)rows * dim) return;
  int row = (int)(i / dim), col = (int)(i % dim);
  int r = row / 3, al = row % 3, sn = col / 3, be = col % 3;
  int tn = (r / nk) * nphi + r % nk;
  const double4 xt = body[tn], xs = body[sn];
  const double rt[3] = {xt.x, xt.y, xt.z}, rs[3] = {xs.x, xs.y, xs.z};
  // ([a]x [b]x)_{al be} = a_be b_al - (a . b) delta_{al be}
  double dot = rt[0] * rs[0] + rt[1] * rs[1] + rt[2] * rs[2];
  double cc = rt[be] * rs[al] - (al == be ? dot : 0.0);
  double Lv = xs.w * ((al == be ? 1.0 : 0.0) - cc);
  M[i] = BK[i] + Lv + (3 * tn + al == col ? 0.5 : 0.0);
}

// The preconditioner of an ellipsoid by symmetry: M = 1/2 I + K0 + L0 commutes with the eight
// reflections of the grid, so in the basis of the irreducible representations it splits into eight
// diagonal blocks.  Block c, entry (a, b), a = (orbit O, beta), b = (orbit O', beta'):
//   sqrt(|O| / |O'|) sum over nodes z of O' of chi_c(g_z) sign_{g_z}(beta') M[3 rep(O) + beta][3 z + beta'],
// g_z the reflection taking rep(O') to z; only representative rows of M are read.  Blocks are padded
// to dmax with the identity.  Grid: (dmax^2 / 256, 8, shapes).
__global__ void k_irrep_blocks(int np, int nrep, int dmax, int d0, int d1, int d2, int d3, int d4, int d5, int d6,
                               int d7, SymTables T, const long long* block_off, const double* Mrows, double* out) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)dmax * dmax) return;
  const int cc = blockIdx.y;
  const int dims[8] = {d0, d1, d2, d3, d4, d5, d6, d7};
  const int d = dims[cc];
  const int a = (int)(e / dmax), b = (int)(e % dmax);
  double* B = out + ((long long)blockIdx.z * 8 + cc) * dmax * dmax;
  if (a >= d || b >= d) {
    B[e] = (a == b) ? 1.0 : 0.0;
    return;
  }
  const int qa = T.irrep_list[cc * 3 * nrep + a], qb = T.irrep_list[cc * 3 * nrep + b];
  const int ra = qa / 3, bea = qa % 3, rb = qb / 3, beb = qb % 3;
  const double* row = Mrows + block_off[blockIdx.z] + (long long)(3 * ra + bea) * (3 * np);
  double acc = 0.0;
  for (int q = 0; q < T.orbit[rb]; ++q) {
    const int z = T.orb_node[8 * rb + q], g = T.orb_g[8 * rb + q];
    const double chi = (__popc(cc & g) & 1) ? -1.0 : 1.0;
    const double sg = ((g >> beb) & 1) ? -1.0 : 1.0;
    acc += chi * sg * row[3 * z + beb];
  }
  B[e] = sqrt((double)T.orbit[ra] / (double)T.orbit[rb]) * acc;
}

// Representative rows of M^{-1} from the inverted irrep blocks: entry (3 r + al, 3 s + be) =
// sum over irreps c holding both (r, al) and (rep(s), be) of
//   Binv_c[(r, al), (rep(s), be)] chi_c(g_s) sign_{g_s}(be) / sqrt(|O_r| |O_rep(s)|).
// Grid: (rows * 3 np / 256, shapes).
__global__ void k_irrep_assemble(int np, int nrep, int dmax, SymTables T, const double* binv,
                                 const long long* block_off, double* Mrows) {
  const long long dim = 3LL * np;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= 3LL * nrep * dim) return;
  const int row = (int)(e / dim), col = (int)(e % dim);
  const int r = row / 3, al = row % 3, sn = col / 3, be = col % 3;
  const int rs = T.rep_of[sn], gs = T.g_of[sn];
  const double sg = ((gs >> be) & 1) ? -1.0 : 1.0;
  const double norm = rsqrt((double)T.orbit[r] * (double)T.orbit[rs]);
  double acc = 0.0;
  for (int cc = 0; cc < 8; ++cc) {
    const int pa = T.irrep_pos[cc * 3 * nrep + 3 * r + al], pb = T.irrep_pos[cc * 3 * nrep + 3 * rs + be];
    if (pa < 0 || pb < 0) continue;
    const double chi = (__popc(cc & gs) & 1) ? -1.0 : 1.0;
    acc += binv[((long long)blockIdx.y * 8 + cc) * dmax * dmax + (long long)pa * dmax + pb] * chi;
  }
  Mrows[block_off[blockIdx.y] + e] = acc * sg * norm;
}

// out (cols x rows) = in (rows x cols)^T
__global__ void k_transpose(const double* in, int rows, int cols, double* out) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)rows * cols) return;
  int r = (int)(i / cols), c = (int)(i % cols);
  out[(long long)c * rows + r] = in[i];
}

__global__ void k_to_float(const double* in, float* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// float64 to the bits of float16 (bf16 = 0) or bfloat16 (bf16 = 1), rounded to nearest.
__global__ void k_to_16bit(const double* in, uint16_t* out, long long n, int bf16) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = bf16 ? __bfloat16_as_ushort(__double2bfloat16(in[i])) : __half_as_ushort(__double2half(in[i]));
}

// Upsampled source nodes of every near-source particle: lab positions and weights on its
// (pup + 1) x nphi_up grid.
__global__ void k_up_nodes(int nu, const int* up_particle, const long long* up_off, const int* pvec, const int* nphivec,
                           const int* pupvec, const int* shape_of, RBS_SHAPE_ARGS, const double* centre,
                           const double* rot, const long long* gtab_up_off, const double* gtab, double4* out) {
  for (int u = blockIdx.y; u < nu; u += gridDim.y) {
    const int i = up_particle[u];
    const int pup = pupvec[i];
    const int nphi_up = nphivec[i] + 2 * (pup - pvec[i]);
    const int nup = (pup + 1) * nphi_up;
    const double* t = gtab + gtab_up_off[i];
    const double* lam = t + (pup + 1);
    const ShapeRef S = RBS_SHAPE_REF(shape_of[i]);
    const double* R = rot + 9 * i;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nup; l += gridDim.x * blockDim.x) {
      const int j = l / nphi_up, k = l % nphi_up;
      const double ct = t[j], st = sqrt(fmax(0.0, 1.0 - ct * ct));
      double sp, cp;
      sincospi(2.0 * k / nphi_up, &sp, &cp);
      double xb[3], J, nb[3];
      eval_surface(S, st * cp, st * sp, ct, xb, &J, nb);
      out[up_off[u] + l] = make_double4(R[0] * xb[0] + R[1] * xb[1] + R[2] * xb[2] + centre[3 * i],
                                        R[3] * xb[0] + R[4] * xb[1] + R[5] * xb[2] + centre[3 * i + 1],
                                        R[6] * xb[0] + R[7] * xb[1] + R[8] * xb[2] + centre[3 * i + 2],
                                        2.0 * kPi / nphi_up * lam[j] * J);
    }
  }
}

// ------------------------------------------------------------------------------------------
// Host orchestration

static void quat_to_rot_host(const double* q, double* R) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double nrm = std::sqrt(w * w + x * x + y * y + z * z);
  w /= nrm;
  x /= nrm;
  y /= nrm;
  z /= nrm;
  R[0] = 1 - 2 * (y * y + z * z);
  R[1] = 2 * (x * y - w * z);
  R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);
  R[4] = 1 - 2 * (x * x + z * z);
  R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);
  R[7] = 2 * (y * z + w * x);
  R[8] = 1 - 2 * (x * x + y * y);
}

template <typename T>
static Status upload(DevBuf<T>& buf, const std::vector<T>& host, cudaStream_t s) {
  RBS_TRY(buf.alloc(host.size()));
  if (!host.empty()) RBS_CUDA_TRY(cudaMemcpyAsync(buf.ptr, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return Status::Ok();
}

static int count_basis(int p, int mmax) {
  int nb = p + 1;
  for (int m = 1; m <= mmax; ++m) nb += 2 * (p - m + 1);
  return nb;
}

// Node (j, k) under the reflection g (bit 0: x -> -x, i.e. phi -> pi - phi; bit 1: y -> -y, phi -> -phi;
// bit 2: z -> -z, theta -> pi - theta).
static int reflect_node(int g, int t, int p, int nphi) {
  int j = t / nphi, k = t % nphi;
  if (g & 4) j = p - j;
  if (g & 2) k = (nphi - k) % nphi;
  if (g & 1) k = (nphi / 2 - k + nphi) % nphi;
  return j * nphi + k;
}

// Orbits of the grid's nodes under the eight reflections, and the bases of the eight irreducible
// representations of the reflection group on surface fields: the basis vector of (orbit O, component
// beta) in irrep c exists when every reflection h fixing O's representative has chi_c(h) sign_h(beta) = 1,
// chi_c(h) = (-1)^popcount(c & h), sign_h(beta) = -1 when h reflects component beta.
static void build_symmetry(Grid& g) {
  g.nj = g.p / 2 + 1;
  g.nk = g.nphi / 4 + 1;
  g.nrep = g.nj * g.nk;
  g.rep_of.assign(g.np, -1);
  g.g_of.assign(g.np, -1);
  g.orbit.assign(g.nrep, 0);
  g.stab.assign(g.nrep, 0);
  g.orb_node.assign(8 * g.nrep, -1);
  g.orb_g.assign(8 * g.nrep, -1);
  for (int r = 0; r < g.nrep; ++r) {
    const int t0 = (r / g.nk) * g.nphi + r % g.nk;
    for (int h = 0; h < 8; ++h) {
      const int t = reflect_node(h, t0, g.p, g.nphi);
      if (t == t0) g.stab[r] |= 1 << h;
      if (g.rep_of[t] < 0) {
        g.rep_of[t] = r;
        g.g_of[t] = h;
        g.orb_node[8 * r + g.orbit[r]] = t;
        g.orb_g[8 * r + g.orbit[r]] = h;
        ++g.orbit[r];
      }
    }
  }
  g.irrep_pos.assign(8 * 3 * g.nrep, -1);
  g.dmax = 0;
  for (int cc = 0; cc < 8; ++cc) {
    int d = 0;
    for (int r = 0; r < g.nrep; ++r)
      for (int be = 0; be < 3; ++be) {
        bool ok = true;
        for (int h = 0; h < 8; ++h)
          if ((g.stab[r] >> h) & 1) {
            const int chi = (__builtin_popcount(cc & h) & 1) ? -1 : 1;
            const int sg = ((h >> be) & 1) ? -1 : 1;
            if (chi * sg != 1) ok = false;
          }
        if (ok) g.irrep_pos[cc * 3 * g.nrep + 3 * r + be] = d++;
      }
    g.irrep_dim[cc] = d;
    g.dmax = std::max(g.dmax, d);
  }
}

// Host only: the symmetry tables of the (p, n_phi) grid (rep_of, g_of per node; irrep dimensions).
Status grid_symmetry_host(int p, int nphi, std::vector<int>& rep_of, std::vector<int>& g_of, int irrep_dim[8],
                          int* nrep) {
  Grid g;
  g.p = p;
  g.nphi = nphi;
  g.np = (p + 1) * nphi;
  build_symmetry(g);
  rep_of = g.rep_of;
  g_of = g.g_of;
  for (int c = 0; c < 8; ++c) irrep_dim[c] = g.irrep_dim[c];
  *nrep = g.nrep;
  return Status::Ok();
}

// Device layout of the symmetry tables: rep_of, g_of (np each), orbit (nrep), orb_node, orb_g
// (8 nrep each), irrep_pos (24 nrep), irrep_list (24 nrep: per irrep, 3 r + beta of each basis vector).
SymTables sym_tables(const Grid& g) {
  const int* b = g.d_sym.ptr;
  SymTables t;
  t.rep_of = b;
  t.g_of = b + g.np;
  t.orbit = t.g_of + g.np;
  t.orb_node = t.orbit + g.nrep;
  t.orb_g = t.orb_node + 8 * g.nrep;
  t.irrep_pos = t.orb_g + 8 * g.nrep;
  t.irrep_list = t.irrep_pos + 24 * g.nrep;
  return t;
}

// Build one grid's tables.
static Status build_grid(Context& c, Grid& g) {
  cudaStream_t s = c.stream;
  g.np = (g.p + 1) * g.nphi;
  g.mmax = (g.nphi - 1) / 2;
  if (g.mmax > g.p) g.mmax = g.p;
  g.nbasis = count_basis(g.p, g.mmax);
  g.ps = c.opt.p_self_factor * g.p;
  g.nrot = (g.ps + 1) * (2 * g.ps + 2);
  g.pup = c.opt.p_up_factor * g.p;
  g.nphi_up = g.nphi + 2 * (g.pup - g.p);
  g.nup = (g.pup + 1) * g.nphi_up;
  gauss_legendre_newton(g.p + 1, g.t, g.lam);
  gauss_legendre_newton(g.pup + 1, g.t_up, g.lam_up);
  RBS_TRY(upload(g.d_t, g.t, s));
  RBS_TRY(upload(g.d_lam, g.lam, s));
  build_symmetry(g);
  {
    std::vector<int> tab;
    tab.insert(tab.end(), g.rep_of.begin(), g.rep_of.end());
    tab.insert(tab.end(), g.g_of.begin(), g.g_of.end());
    tab.insert(tab.end(), g.orbit.begin(), g.orbit.end());
    tab.insert(tab.end(), g.orb_node.begin(), g.orb_node.end());
    tab.insert(tab.end(), g.orb_g.begin(), g.orb_g.end());
    tab.insert(tab.end(), g.irrep_pos.begin(), g.irrep_pos.end());
    std::vector<int> list(24 * g.nrep, -1);
    for (int cc = 0; cc < 8; ++cc)
      for (int q = 0; q < 3 * g.nrep; ++q) {
        const int pos = g.irrep_pos[cc * 3 * g.nrep + q];
        if (pos >= 0) list[cc * 3 * g.nrep + pos] = q;
      }
    tab.insert(tab.end(), list.begin(), list.end());
    RBS_TRY(upload(g.d_sym, tab, s));
  }
  RBS_TRY(upload(g.d_t_up, g.t_up, s));
  RBS_TRY(upload(g.d_lam_up, g.lam_up, s));

  // rotated singular-rule points for targets (theta_j, phi = 0): R_y(theta_j) applied to the rule
  // around the pole; theta' by Gauss-Legendre on [0, pi], phi' uniform (2 ps + 2 points).
  std::vector<double> u, lu;
  gauss_legendre_newton(g.ps + 1, u, lu);
  int nb = 2 * g.ps + 2;
  std::vector<double> rot((size_t)(g.p + 1) * g.nrot * 4);
  for (int j = 0; j <= g.p; ++j) {
    double ct = g.t[j], st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
    for (int a = 0; a <= g.ps; ++a) {
      double th = 0.5 * kPi * (u[a] + 1.0);
      double wth = 0.5 * kPi * lu[a];
      for (int bb = 0; bb < nb; ++bb) {
        double ph = 2.0 * kPi * bb / nb;
        double px = std::sin(th) * std::cos(ph), py = std::sin(th) * std::sin(ph), pz = std::cos(th);
        // R_y(theta) = [[ct, 0, st], [0, 1, 0], [-st, 0, ct]]
        size_t idx = ((size_t)j * g.nrot + (size_t)a * nb + bb) * 4;
        rot[idx + 0] = ct * px + st * pz;
        rot[idx + 1] = py;
        rot[idx + 2] = -st * px + ct * pz;
        rot[idx + 3] = wth * std::sin(th) * (2.0 * kPi / nb);
      }
    }
  }
  RBS_TRY(upload(g.d_rotpts, rot, s));

  // analysis matrix on the grid
  DevBuf<double4> gp;
  RBS_TRY(gp.alloc(g.np));
  k_grid_points<<<cdiv(g.np, 128), 128, 0, s>>>(g.p, g.nphi, g.d_t.ptr, g.d_lam.ptr, gp.ptr);
  DevBuf<double>& Yg = g.d_yg;
  DevBuf<double>& An = g.d_an;
  RBS_TRY(Yg.alloc((size_t)g.np * g.nbasis));
  RBS_TRY(An.alloc((size_t)g.np * g.nbasis));
  k_sh_at_points<<<cdiv(g.np, 128), 128, 0, s>>>(g.p, g.mmax, g.nbasis, gp.ptr, g.np, Yg.ptr);
  k_analysis<<<cdiv((long long)g.np * g.nbasis, 256), 256, 0, s>>>(g.np, g.nbasis, Yg.ptr, gp.ptr, An.ptr);
  RBS_CUDA_TRY(cudaGetLastError());

  // singular-rule interpolation: Interp_j = Y(rotated points of j) x An
  DevBuf<double> Yr;
  long long nrp = (long long)(g.p + 1) * g.nrot;
  RBS_TRY(Yr.alloc((size_t)nrp * g.nbasis));
  k_sh_at_points<<<cdiv(nrp, 128), 128, 0, s>>>(g.p, g.mmax, g.nbasis, (const double4*)g.d_rotpts.ptr, (int)nrp,
                                                Yr.ptr);
  RBS_TRY(g.d_interp.alloc((size_t)nrp * g.np));
  RBS_TRY(dgemm_batched(s, (int)nrp, g.np, g.nbasis, Yr.ptr, g.nbasis, 0, An.ptr, g.np, 0, g.d_interp.ptr, g.np, 0, 1));

  // upsampling interpolation U = Y(upsampled grid) x An
  DevBuf<double4> gup;
  RBS_TRY(gup.alloc(g.nup));
  k_grid_points<<<cdiv(g.nup, 128), 128, 0, s>>>(g.pup, g.nphi_up, g.d_t_up.ptr, g.d_lam_up.ptr, gup.ptr);
  DevBuf<double> Yu;
  RBS_TRY(Yu.alloc((size_t)g.nup * g.nbasis));
  k_sh_at_points<<<cdiv(g.nup, 128), 128, 0, s>>>(g.p, g.mmax, g.nbasis, gup.ptr, g.nup, Yu.ptr);
  // U^T = An^T Y(upsampled)^T, stored N_p x N_up
  {
    DevBuf<double> YuT, AnT;
    RBS_TRY(YuT.alloc((size_t)g.nup * g.nbasis));
    RBS_TRY(AnT.alloc((size_t)g.np * g.nbasis));
    k_transpose<<<cdiv((long long)g.nup * g.nbasis, 256), 256, 0, s>>>(Yu.ptr, g.nup, g.nbasis, YuT.ptr);
    k_transpose<<<cdiv((long long)g.np * g.nbasis, 256), 256, 0, s>>>(An.ptr, g.nbasis, g.np, AnT.ptr);
    RBS_TRY(g.d_up.alloc((size_t)g.nup * g.np));
    RBS_TRY(dgemm_batched(s, g.np, g.nup, g.nbasis, AnT.ptr, g.nbasis, 0, YuT.ptr, g.nup, 0, g.d_up.ptr, g.nup, 0, 1));
    RBS_TRY(g.d_up32.alloc((size_t)g.nup * g.np));
    k_to_float<<<256, 256, 0, s>>>(g.d_up.ptr, g.d_up32.ptr, (long long)g.nup * g.np);
    RBS_CUDA_TRY(cudaStreamSynchronize(s));
  }
  RBS_CUDA_TRY(cudaGetLastError());
  RBS_CUDA_TRY(cudaStreamSynchronize(s));  // temporaries are released on return
  return Status::Ok();
}

// Self blocks of every shape of one grid, in chunks of shapes.  For each chunk and polar index j:
// kernel values C (18 nkc x nrot per shape), one batched GEMM G = C x Interp_j, and the scatter
// into the body-frame blocks with the azimuthal shift.  Shapes stored by representative rows (sym)
// need the targets j <= p / 2, k <= nphi / 4 only.
static Status build_self_blocks(Context& c, int gi, const std::vector<int>& shape_ids, bool sym) {
  cudaStream_t s = c.stream;
  Grid& g = *c.grids[gi];
  const int nkc = sym ? g.nk : g.nphi;
  const int jmax = sym ? g.nj - 1 : g.p;
  long long rowsC = 18LL * nkc;
  size_t perC = (size_t)rowsC * g.nrot, perG = (size_t)rowsC * g.np;
  size_t budget = (size_t)1 << 27;  // doubles, 1 GB
  int per_chunk = (int)std::max<size_t>(1, budget / (perC + perG));
  int nsh = (int)shape_ids.size();
  int chunk = std::min(std::min(per_chunk, nsh), 65535);
  DevBuf<double> C, G;
  RBS_TRY(C.alloc(perC * chunk));
  RBS_TRY(G.alloc(perG * chunk));
  std::vector<long long> off(nsh);
  for (int k = 0; k < nsh; ++k) off[k] = (long long)c.shapes[shape_ids[k]].block_off;
  DevBuf<int> d_ids;
  DevBuf<long long> d_off;
  RBS_TRY(upload(d_ids, shape_ids, s));
  RBS_TRY(upload(d_off, off, s));
  for (int start = 0; start < nsh; start += chunk) {
    int cnt = std::min(chunk, nsh - start);
    for (int j = 0; j <= jmax; ++j) {
      dim3 grd(cdiv(g.nrot, 128), nkc, cnt);
      k_self_kernel_values<<<grd, 128, 0, s>>>(g.nphi, nkc, g.nrot, g.t[j], d_ids.ptr + start, RBS_SHAPE_PASS,
                                               (const double4*)g.d_rotpts.ptr + (size_t)j * g.nrot, C.ptr, perC);
      RBS_CUDA_TRY(cudaGetLastError());
      RBS_TRY(dgemm_batched(s, (int)rowsC, g.np, g.nrot, C.ptr, g.nrot, (long long)perC,
                            g.d_interp.ptr + (size_t)j * g.nrot * g.np, g.np, 0, G.ptr, g.np, (long long)perG, cnt));
      long long tot = 2LL * nkc * 9 * g.np;
      dim3 grs(cdiv(tot, 256), cnt);
      k_self_scatter<<<grs, 256, 0, s>>>(g.nphi, nkc, g.np, j, G.ptr, perG, d_off.ptr + start, c.d_blockK.ptr,
                                         c.d_blockS.ptr);
      RBS_CUDA_TRY(cudaGetLastError());
    }
  }
  RBS_CUDA_TRY(cudaStreamSynchronize(s));
  return Status::Ok();
}

// Lab-frame nodes, normals, weights and moments of every particle from the current centres and
// rotations (Eq. 40 with the body frame as reference; Eq. 18).
Status place_particles(Context& c) {
  cudaStream_t s = c.stream;
  const int n = c.n;
  RBS_TRY(upload(c.d_centre, c.centres, s));
  RBS_TRY(upload(c.d_rot, c.rot, s));
  if (c.d_x.n != (size_t)c.N) {
    RBS_TRY(c.d_x.alloc(c.N));
    RBS_TRY(c.d_nrm.alloc(c.N));
    RBS_TRY(c.d_pid.alloc(c.N));
    RBS_TRY(c.d_area.alloc(n));
    RBS_TRY(c.d_tauinv.alloc((size_t)9 * n));
  }
  int maxnp = 0;
  for (int i = 0; i < n; ++i) maxnp = std::max(maxnp, (int)(c.offset[i + 1] - c.offset[i]));
  dim3 grd(cdiv(maxnp, 128), std::min(n, 65535));
  k_nodes<<<grd, 128, 0, s>>>(n, c.d_offset.ptr, c.d_p.ptr, c.d_nphi.ptr, c.d_shape.ptr, RBS_SHAPE_PASS,
                              c.d_centre.ptr, c.d_rot.ptr, c.d_gtab_off.ptr, c.d_gtab.ptr, c.d_x.ptr, c.d_nrm.ptr, c.d_pid.ptr);
  k_moments<<<n, 256, 0, s>>>(n, c.d_offset.ptr, c.d_x.ptr, c.d_centre.ptr, c.d_area.ptr, c.d_tauinv.ptr);
  RBS_TRY(c.d_xhi.alloc(c.N));
  RBS_TRY(c.d_xlo.alloc(c.N));
  RBS_TRY(c.d_wmu32.alloc(c.N));
  RBS_TRY(c.d_nrm32.alloc(c.N));
  for (DevBuf<float4>* b : {&c.d_x3h, &c.d_x3m, &c.d_x3l, &c.d_nrmh, &c.d_nrml, &c.d_wmuh, &c.d_wmul})
    RBS_TRY(b->alloc(c.N));
  k_split_positions<<<cdiv(c.N, 256), 256, 0, s>>>(c.N, c.d_x.ptr, c.d_nrm.ptr, c.d_pid.ptr, c.d_xhi.ptr, c.d_xlo.ptr,
                                                   c.d_nrm32.ptr, c.d_x3h.ptr, c.d_x3m.ptr, c.d_x3l.ptr, c.d_nrmh.ptr,
                                                   c.d_nrml.ptr);
  RBS_CUDA_TRY(cudaGetLastError());
  return Status::Ok();
}

// Near pairs (Section 3, upsampling for close particles): ordered pairs (i, j), i != j of one
// suspension with |c_i - c_j| < R_i + R_j + delta, found with a cell list; RBS_EOVERLAP when two
// inscribed spheres (radius rmin) intersect.  Host only.
Status plan_near(int n, const double* centres, const double* R, const double* rmin, const int* sid, double delta,
                 std::vector<int2>& out) {
  out.clear();
  double rmax = 0.0;
  for (int i = 0; i < n; ++i) rmax = std::max(rmax, R[i]);
  const double cell = 2.0 * rmax + delta;
  std::unordered_map<long long, std::vector<int>> cells;
  // cells of one suspension only: independent suspensions may occupy the same region
  auto key = [&](long long a, long long b, long long d, long long q) {
    return (a * 73856093LL) ^ (b * 19349663LL) ^ (d * 83492791LL) ^ (q * 2654435761LL);
  };
  std::vector<long long> ci(3 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    for (int d = 0; d < 3; ++d) ci[3 * i + d] = (long long)std::floor(centres[3 * i + d] / cell);
    cells[key(ci[3 * i], ci[3 * i + 1], ci[3 * i + 2], sid[i])].push_back(i);
  }
  for (int i = 0; i < n; ++i) {
    std::vector<int> cand;
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          auto it = cells.find(key(ci[3 * i] + dx, ci[3 * i + 1] + dy, ci[3 * i + 2] + dz, sid[i]));
          if (it == cells.end()) continue;
          for (int j : it->second) cand.push_back(j);
        }
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    for (int j : cand) {
      if (j == i || sid[j] != sid[i]) continue;
      double dx = centres[3 * i] - centres[3 * j], dy = centres[3 * i + 1] - centres[3 * j + 1],
             dz = centres[3 * i + 2] - centres[3 * j + 2];
      double d = std::sqrt(dx * dx + dy * dy + dz * dz);
      if (d < rmin[i] + rmin[j])
        return Status::Err(RBS_EOVERLAP, "particles " + std::to_string(i) + " and " + std::to_string(j) +
                                             " overlap (inscribed spheres intersect)");
      if (d < R[i] + R[j] + delta) out.push_back(make_int2(i, j));
    }
  }
  return Status::Ok();
}

// Near-pair list and the upsampled source nodes.
Status build_near(Context& c) {
  cudaStream_t s = c.stream;
  const int n = c.n;
  ++c.config_version;  // captured GMRES step graphs hold this configuration's lists and pointers
  {
    std::vector<double> R(n), rmin(n);
    for (int i = 0; i < n; ++i) {
      R[i] = c.shapes[c.shape_of[i]].radius;
      rmin[i] = c.shapes[c.shape_of[i]].rmin;
    }
    RBS_TRY(plan_near(n, c.centres.data(), R.data(), rmin.data(), c.sid.data(), c.opt.near_delta, c.near_pairs));
  }
  RBS_TRY(upload(c.d_near, c.near_pairs, s));
  // upsampled sources
  c.up_index.assign(n, -1);
  c.up_particle.clear();
  c.up_offset.clear();
  c.n_up_nodes = 0;
  for (const int2& pr : c.near_pairs) {
    int j = pr.y;
    if (c.up_index[j] < 0) {
      c.up_index[j] = (int)c.up_particle.size();
      c.up_particle.push_back(j);
      c.up_offset.push_back(c.n_up_nodes);
      c.n_up_nodes += c.grids[c.grid_of[j]]->nup;
    }
  }
  c.up_offset.push_back(c.n_up_nodes);
  {
    std::vector<const double*> U;
    std::vector<const float*> U32;
    for (int j : c.up_particle) {
      U.push_back(c.grids[c.grid_of[j]]->d_up.ptr);
      U32.push_back(c.grids[c.grid_of[j]]->d_up32.ptr);
    }
    RBS_TRY(upload(c.d_upU, U, s));
    RBS_TRY(upload(c.d_upU32, U32, s));
  }
  RBS_TRY(upload(c.d_up_particle, c.up_particle, s));
  RBS_TRY(upload(c.d_up_off, c.up_offset, s));
  RBS_TRY(upload(c.d_up_index, c.up_index, s));
  RBS_TRY(c.d_up_x.alloc(c.n_up_nodes));
  RBS_TRY(c.d_up_mu.alloc(3 * c.n_up_nodes));
  if (!c.up_particle.empty()) {
    int maxnup = 0;
    for (Grid* g : c.grids) maxnup = std::max(maxnup, g->nup);
    dim3 grd(cdiv(maxnup, 128), (unsigned)std::min<size_t>(c.up_particle.size(), 65535));
    k_up_nodes<<<grd, 128, 0, s>>>((int)c.up_particle.size(), c.d_up_particle.ptr, c.d_up_off.ptr, c.d_p.ptr, c.d_nphi.ptr,
                                   c.d_pup.ptr, c.d_shape.ptr, RBS_SHAPE_PASS, c.d_centre.ptr, c.d_rot.ptr,
                                   c.d_gtab_up_off.ptr, c.d_gtab.ptr, c.d_up_x.ptr);
    RBS_CUDA_TRY(cudaGetLastError());
  }

  c.near_pair_nodes = 0;
  for (const int2& pr : c.near_pairs)
    c.near_pair_nodes += (double)(c.offset[pr.x + 1] - c.offset[pr.x]) *
                         (c.grids[c.grid_of[pr.y]]->nup + (c.offset[pr.y + 1] - c.offset[pr.y]));
  c.stats.near_pairs = (long long)c.near_pairs.size();
  return build_far_field(c);
}

Status update_configuration(Context& c, const double* centres, const double* quats) {
  for (int i = 0; i < 3 * c.n; ++i) c.centres[i] = centres[i];
  for (int i = 0; i < 4 * c.n; ++i) c.quats[i] = quats[i];
  for (int i = 0; i < c.n; ++i) quat_to_rot_host(&c.quats[4 * i], &c.rot[9 * i]);
  RBS_TRY(place_particles(c));
  return build_near(c);
}

// Device tables of the distinct shapes; for coefficient surfaces, their centroid shift, bounding
// radius and checks (a positive area element everywhere, an outward parametrisation).  Particles on a
// coefficient surface report (R, R, R) as their semi-axes, R the bounding radius.
static Status build_shape_tables(Context& c, const std::vector<long long>& grid_tab_off,
                                 const std::vector<long long>& grid_tab_up_off) {
  cudaStream_t s = c.stream;
  const int ns = (int)c.shapes.size();
  std::vector<int> kind(ns), pg(ns, 0);
  std::vector<double> axes(3 * (size_t)ns, 0.0), shift(3 * (size_t)ns, 0.0);
  std::vector<long long> coef_off(ns, -1);
  std::vector<ShapeGrid> sg;
  c.max_np_shape = 0;
  for (int k = 0; k < ns; ++k) {
    const Shape& sh = c.shapes[k];
    c.max_np_shape = std::max(c.max_np_shape, sh.np);
    kind[k] = sh.kind;
    axes[3 * k] = sh.a;
    axes[3 * k + 1] = sh.b;
    axes[3 * k + 2] = sh.c;
    if (sh.kind == 1) {
      pg[k] = c.cs_pg[sh.cs];
      coef_off[k] = c.cs_off[sh.cs];
      const Grid& g = *c.grids[sh.grid];
      sg.push_back(ShapeGrid{k, g.p, g.nphi, g.pup, grid_tab_off[sh.grid], grid_tab_up_off[sh.grid]});
    }
  }
  std::vector<double> coef = c.cs_coef;
  if (coef.empty()) coef.push_back(0.0);
  RBS_TRY(upload(c.d_sh_kind, kind, s));
  RBS_TRY(upload(c.d_sh_pg, pg, s));
  RBS_TRY(upload(c.d_sh_axes, axes, s));
  RBS_TRY(upload(c.d_sh_shift, shift, s));
  RBS_TRY(upload(c.d_sh_coef_off, coef_off, s));
  RBS_TRY(upload(c.d_sh_coef, coef, s));
  if (sg.empty()) return Status::Ok();
  DevBuf<ShapeGrid> d_sg;
  DevBuf<double> d_diag;
  RBS_TRY(upload(d_sg, sg, s));
  RBS_TRY(d_diag.alloc(4 * sg.size()));
  for (size_t b0 = 0; b0 < sg.size(); b0 += 65535) {
    const int cnt = (int)std::min<size_t>(65535, sg.size() - b0);
    k_shape_extent<<<cnt, 256, 0, s>>>(d_sg.ptr + b0, RBS_SHAPE_PASS, c.d_sh_shift.ptr, c.d_gtab.ptr,
                                      d_diag.ptr + 4 * b0);
  }
  RBS_CUDA_TRY(cudaGetLastError());
  std::vector<double> diag(4 * sg.size());
  RBS_CUDA_TRY(cudaMemcpyAsync(diag.data(), d_diag.ptr, sizeof(double) * diag.size(), cudaMemcpyDeviceToHost, s));
  RBS_CUDA_TRY(cudaStreamSynchronize(s));
  for (size_t q = 0; q < sg.size(); ++q) {
    Shape& sh = c.shapes[sg[q].s];
    const double jmin = diag[4 * q + 2], vol = diag[4 * q + 3];
    if (!(jmin > 0.0) || !std::isfinite(diag[4 * q]))
      return Status::Err(RBS_EINVAL, "coefficient surface " + std::to_string(sh.cs) +
                                         " is singular (area element vanishes on the grid)");
    if (!(vol > 0.0))
      return Status::Err(RBS_EINVAL, "coefficient surface " + std::to_string(sh.cs) +
                                         " is inward-oriented (negative enclosed volume)");
    sh.radius = diag[4 * q];
    sh.rmin = diag[4 * q + 1];
  }
  for (int i = 0; i < c.n; ++i) {
    const Shape& sh = c.shapes[c.shape_of[i]];
    if (sh.kind == 1) c.axes[3 * i] = c.axes[3 * i + 1] = c.axes[3 * i + 2] = sh.radius;
  }
  return Status::Ok();
}

Status build_geometry(Context& c) {
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = c.stream;
  const int n = c.n;
  c.mag.release();  // the magnetostatic blocks belong to the previous shapes
  // rotations
  c.rot.assign((size_t)9 * n, 0.0);
  for (int i = 0; i < n; ++i) quat_to_rot_host(&c.quats[4 * i], &c.rot[9 * i]);
  // node offsets
  c.offset.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) c.offset[i + 1] = c.offset[i] + (long long)(c.p[i] + 1) * c.nphi[i];
  c.N = c.offset[n];

  // grids
  for (Grid* g : c.grids) delete g;
  c.grids.clear();
  std::map<std::pair<int, int>, int> grid_id;
  std::vector<int> grid_of(n);
  for (int i = 0; i < n; ++i) {
    auto key = std::make_pair(c.p[i], c.nphi[i]);
    auto it = grid_id.find(key);
    if (it == grid_id.end()) {
      Grid* g = new Grid();
      g->p = c.p[i];
      g->nphi = c.nphi[i];
      it = grid_id.emplace(key, (int)c.grids.size()).first;
      c.grids.push_back(g);
    }
    grid_of[i] = it->second;
  }
  for (Grid* g : c.grids) RBS_TRY(build_grid(c, *g));

  // shapes: an ellipsoid is keyed by its semi-axes, a coefficient surface by its input index
  c.shapes.clear();
  c.shape_of.assign(n, 0);
  const bool coef_surfaces = !c.cs_of.empty();
  std::map<std::tuple<int, double, double, double, int, int>, int> shape_id;
  c.block_elems = 0;
  for (int i = 0; i < n; ++i) {
    const int cs = coef_surfaces ? c.cs_of[i] : -1;
    auto key = cs >= 0 ? std::make_tuple(cs, 0.0, 0.0, 0.0, c.p[i], c.nphi[i])
                       : std::make_tuple(-1, c.axes[3 * i], c.axes[3 * i + 1], c.axes[3 * i + 2], c.p[i], c.nphi[i]);
    auto it = shape_id.find(key);
    if (it == shape_id.end()) {
      Shape sh;
      sh.kind = cs >= 0 ? 1 : 0;
      sh.cs = cs;
      if (cs < 0) {
        sh.a = c.axes[3 * i];
        sh.b = c.axes[3 * i + 1];
        sh.c = c.axes[3 * i + 2];
        sh.radius = std::max(sh.a, std::max(sh.b, sh.c));
        sh.rmin = std::min(sh.a, std::min(sh.b, sh.c));
      }
      sh.grid = grid_of[i];
      sh.np = c.grids[sh.grid]->np;
      // ellipsoids store representative rows when the eight reflected copies of a float64 surface
      // field fit in shared memory (N_p <= 1066, e.g. p = 16 on a 17 x 32 grid)
      // the float64 block kernel's shared memory (the largest variant) within the 227 KB of a CTA
      sh.sym = (sh.kind == 0) && sym_smem_bytes(sh.np, 8, 8) + 1024 <= 227 * 1024;
      sh.rows = sh.sym ? 3 * c.grids[sh.grid]->nrep : 3 * sh.np;
      sh.block_off = c.block_elems;
      c.block_elems += (size_t)sh.rows * 3 * sh.np;
      it = shape_id.emplace(key, (int)c.shapes.size()).first;
      c.shapes.push_back(sh);
    }
    c.shape_of[i] = it->second;
  }

  // per-particle device arrays
  std::vector<long long> gtab_off(n), gtab_up_off(n);
  std::vector<double> gtab;
  std::vector<long long> grid_tab_off(c.grids.size()), grid_tab_up_off(c.grids.size());
  for (size_t gi = 0; gi < c.grids.size(); ++gi) {
    Grid& g = *c.grids[gi];
    grid_tab_off[gi] = (long long)gtab.size();
    gtab.insert(gtab.end(), g.t.begin(), g.t.end());
    gtab.insert(gtab.end(), g.lam.begin(), g.lam.end());
    grid_tab_up_off[gi] = (long long)gtab.size();
    gtab.insert(gtab.end(), g.t_up.begin(), g.t_up.end());
    gtab.insert(gtab.end(), g.lam_up.begin(), g.lam_up.end());
  }
  std::vector<int> pup(n);
  for (int i = 0; i < n; ++i) {
    gtab_off[i] = grid_tab_off[grid_of[i]];
    gtab_up_off[i] = grid_tab_up_off[grid_of[i]];
    pup[i] = c.grids[grid_of[i]]->pup;
  }
  c.grid_of = grid_of;
  RBS_TRY(upload(c.d_gtab_off, gtab_off, s));
  RBS_TRY(upload(c.d_gtab_up_off, gtab_up_off, s));
  RBS_TRY(upload(c.d_gtab, gtab, s));
  RBS_TRY(build_shape_tables(c, grid_tab_off, grid_tab_up_off));
  RBS_TRY(upload(c.d_axes, c.axes, s));
  RBS_TRY(upload(c.d_p, c.p, s));
  RBS_TRY(upload(c.d_nphi, c.nphi, s));
  RBS_TRY(upload(c.d_pup, pup, s));
  RBS_TRY(upload(c.d_offset, c.offset, s));
  RBS_TRY(upload(c.d_shape, c.shape_of, s));
  std::vector<int> nodes(n);
  for (int i = 0; i < n; ++i) nodes[i] = (int)(c.offset[i + 1] - c.offset[i]);
  RBS_TRY(upload(c.d_nodes, nodes, s));
  RBS_TRY(c.d_x.alloc(c.N));
  RBS_TRY(c.d_nrm.alloc(c.N));
  RBS_TRY(c.d_pid.alloc(c.N));
  RBS_TRY(c.d_area.alloc(n));
  RBS_TRY(c.d_tauinv.alloc((size_t)9 * n));
  RBS_TRY(place_particles(c));

  // self blocks (body frame) of every shape
  RBS_TRY(c.d_blockK.alloc(c.block_elems));
  RBS_TRY(c.d_blockS.alloc(c.block_elems));
  {
    std::vector<std::vector<int>> by_grid(2 * c.grids.size());
    for (size_t k = 0; k < c.shapes.size(); ++k)
      by_grid[2 * c.shapes[k].grid + (c.shapes[k].sym ? 1 : 0)].push_back((int)k);
    for (size_t q = 0; q < by_grid.size(); ++q)
      if (!by_grid[q].empty()) RBS_TRY(build_self_blocks(c, (int)(q / 2), by_grid[q], q % 2 == 1));
  }
  std::vector<long long> boff(c.shapes.size());
  for (size_t k = 0; k < c.shapes.size(); ++k) boff[k] = (long long)c.shapes[k].block_off;
  RBS_TRY(upload(c.d_block_off, boff, s));

  // block-diagonal preconditioner P0 = (1/2 I + K0 + L0)^{-1} per shape (Section 3.2)
  if (c.opt.preconditioner) {
    RBS_TRY(c.d_precond.alloc(c.block_elems));
    DevBuf<double4> body;
    RBS_TRY(body.alloc(c.max_np_shape));
    for (size_t k = 0; k < c.shapes.size(); ++k) {
      const Shape& sh = c.shapes[k];
      Grid& g = *c.grids[sh.grid];
      long long elems = (long long)sh.rows * 3 * sh.np;
      k_body_nodes<<<cdiv(sh.np, 128), 128, 0, s>>>(sh.np, g.nphi, g.d_t.ptr, g.d_lam.ptr, (int)k, RBS_SHAPE_PASS,
                                                    body.ptr);
      k_precond_matrix<<<cdiv(elems, 256), 256, 0, s>>>(sh.np, g.nphi, sh.sym ? g.nk : g.nphi, sh.rows, body.ptr,
                                                        c.d_blockK.ptr + sh.block_off, c.d_precond.ptr + sh.block_off);
    }
    RBS_CUDA_TRY(cudaGetLastError());
    // shapes storing every row: invert runs of consecutive (hence contiguous) shapes of one size
    size_t k = 0;
    while (k < c.shapes.size()) {
      if (c.shapes[k].sym) {
        ++k;
        continue;
      }
      size_t e = k + 1;
      while (e < c.shapes.size() && !c.shapes[e].sym && c.shapes[e].np == c.shapes[k].np) ++e;
      RBS_TRY(invert_batched(c, c.d_precond.ptr + c.shapes[k].block_off, 3 * c.shapes[k].np, (int)(e - k)));
      k = e;
    }
    // ellipsoids: by irreducible representation, per grid, in chunks of shapes
    for (size_t gi = 0; gi < c.grids.size(); ++gi) {
      std::vector<long long> offs;
      for (const Shape& sh : c.shapes)
        if (sh.sym && sh.grid == (int)gi) offs.push_back((long long)sh.block_off);
      if (offs.empty()) continue;
      const Grid& g = *c.grids[gi];
      const SymTables T = sym_tables(g);
      const long long per = 8LL * g.dmax * g.dmax;
      const int chunk = (int)std::max<long long>(1, std::min<long long>((long long)offs.size(), (1LL << 28) / per));
      DevBuf<double> blocks;
      DevBuf<long long> d_offs;
      RBS_TRY(blocks.alloc((size_t)per * chunk));
      RBS_TRY(upload(d_offs, offs, s));
      for (size_t b0 = 0; b0 < offs.size(); b0 += chunk) {
        const int cnt = (int)std::min<size_t>(chunk, offs.size() - b0);
        dim3 gb(cdiv((long long)g.dmax * g.dmax, 256), 8, cnt);
        k_irrep_blocks<<<gb, 256, 0, s>>>(g.np, g.nrep, g.dmax, g.irrep_dim[0], g.irrep_dim[1], g.irrep_dim[2],
                                          g.irrep_dim[3], g.irrep_dim[4], g.irrep_dim[5], g.irrep_dim[6],
                                          g.irrep_dim[7], T, d_offs.ptr + b0, c.d_precond.ptr, blocks.ptr);
        RBS_CUDA_TRY(cudaGetLastError());
        RBS_TRY(invert_batched(c, blocks.ptr, g.dmax, 8 * cnt));
        dim3 ga(cdiv(9LL * g.nrep * g.np, 256), cnt);
        k_irrep_assemble<<<ga, 256, 0, s>>>(g.np, g.nrep, g.dmax, T, blocks.ptr, d_offs.ptr + b0, c.d_precond.ptr);
        RBS_CUDA_TRY(cudaGetLastError());
      }
      RBS_CUDA_TRY(cudaStreamSynchronize(s));
    }
    // the float32 copy serves the inner solves of the mixed path, the float64 one the float64 path;
    // the 16-bit modes keep a float16 or bfloat16 copy for the inner solve as well
    if (prec_f32(c.opt.precision)) {
      RBS_TRY(c.d_precond32.alloc(c.block_elems));
      k_to_float<<<1024, 256, 0, s>>>(c.d_precond.ptr, c.d_precond32.ptr, (long long)c.block_elems);
      if (prec_16(c.opt.precision)) {
        RBS_TRY(c.d_precond16.alloc(c.block_elems));
        k_to_16bit<<<1024, 256, 0, s>>>(c.d_precond.ptr, c.d_precond16.ptr, (long long)c.block_elems,
                                        c.opt.precision == RBS_PREC_MIXED_BF16);
      }
      RBS_CUDA_TRY(cudaStreamSynchronize(s));
      c.d_precond.release();
    } else {
      c.d_precond32.release();
    }
  }
  RBS_TRY(c.d_blockK32.alloc(c.block_elems));
  k_to_float<<<1024, 256, 0, s>>>(c.d_blockK.ptr, c.d_blockK32.ptr, (long long)c.block_elems);
  if (prec_16(c.opt.precision)) {
    RBS_TRY(c.d_blockK16.alloc(c.block_elems));
    k_to_16bit<<<1024, 256, 0, s>>>(c.d_blockK.ptr, c.d_blockK16.ptr, (long long)c.block_elems,
                                    c.opt.precision == RBS_PREC_MIXED_BF16);
  } else {
    c.d_blockK16.release();
    c.d_precond16.release();
  }
  RBS_CUDA_TRY(cudaGetLastError());

  RBS_TRY(build_near(c));

  // smooth pair-sum work list: target tiles of 128 nodes, never straddling a suspension, each
  // paired with source chunks of that suspension; chunks split so the grid covers the GPU.
  c.work.clear();
  {
    std::vector<std::pair<long long, long long>> susp;
    int i = 0;
    while (i < n) {
      int e = i + 1;
      while (e < n && c.sid[e] == c.sid[i]) ++e;
      susp.emplace_back(c.offset[i], c.offset[e]);
      i = e;
    }
    const long long TT = 128;
    long long tiles = 0;
    for (auto& sp : susp) tiles += (sp.second - sp.first + TT - 1) / TT;
    // about 96 items per SM, so a persistent grid of ~12 resident blocks per SM runs ~8 rounds and
    // its last round is nearly full; source chunks stay >= 2048 nodes
    long long want = 96LL * std::max(1, c.sm_count);
    int splits = (int)std::max(1LL, (want + tiles - 1) / std::max(1LL, tiles));
    for (auto& sp : susp) {
      long long ns = sp.second - sp.first;
      int sc = (int)std::min<long long>(splits, std::max(1LL, ns / 2048));
      long long chunk = (ns + sc - 1) / sc;
      for (long long tb = sp.first; tb < sp.second; tb += TT)
        for (long long sb = sp.first; sb < sp.second; sb += chunk) {
          longlong4 w;
          w.x = tb;
          w.y = std::min(tb + TT, sp.second);
          w.z = sb;
          w.w = std::min(sb + chunk, sp.second);
          c.work.push_back(w);
        }
    }
  }
  RBS_TRY(upload(c.d_work, c.work, s));

  // particle-block work list
  c.bwork.clear();
  c.sym_list.clear();
  c.max_np = 0;
  c.max_np_sym = 0;
  for (int i = 0; i < n; ++i) {
    c.max_np = std::max(c.max_np, nodes[i]);
    if (c.shapes[c.shape_of[i]].sym) {
      c.sym_list.push_back(i);
      c.max_np_sym = std::max(c.max_np_sym, nodes[i]);
      continue;
    }
    for (int b = 0; b < nodes[i]; b += 24) c.bwork.push_back(make_int4(i, b, std::min(b + 24, nodes[i]), 0));
  }
  RBS_TRY(upload(c.d_bwork, c.bwork, s));
  RBS_TRY(upload(c.d_sym_list, c.sym_list, s));

  // workspace; the suspensions (contiguous runs of equal ids) as segments of the 3N unknowns
  for (auto& v : c.d_vec) RBS_TRY(v.alloc(3 * c.N));
  RBS_TRY(c.d_partials.alloc(64));
  {
    std::vector<long long> so(1, 0);
    for (int i = 1; i <= n; ++i)
      if (i == n || c.sid[i] != c.sid[i - 1]) so.push_back(3 * c.offset[i]);
    RBS_TRY(c.seg3.build(so, s));
  }
  ++c.config_version;
  RBS_TRY(c.d_FT.alloc((size_t)6 * n));
  RBS_TRY(c.d_vo.alloc((size_t)6 * n));
  RBS_CUDA_TRY(cudaStreamSynchronize(s));

  // stats
  c.stats.total_nodes = c.N;
  c.stats.n_particles = n;
  c.stats.n_shapes = (int)c.shapes.size();

  long long fp = 0;
  {
    int i = 0;
    while (i < n) {
      int e = i + 1;
      while (e < n && c.sid[e] == c.sid[i]) ++e;
      long long ns = c.offset[e] - c.offset[i];
      fp += ns * ns;
      for (int k = i; k < e; ++k) fp -= (long long)nodes[k] * nodes[k];
      i = e;
    }
  }
  c.stats.far_pairs = fp;
  c.particle_block_entries = 0;
  for (int k = 0; k < n; ++k) c.particle_block_entries += (double)c.shapes[c.shape_of[k]].rows * 3.0 * nodes[k];

  RBS_TRY(build_self_gemm(c));
  c.stats.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  c.have_geometry = true;
  return Status::Ok();
}

}  // namespace rbs
