// Magnetostatic coupling of paramagnetic particles (Section 4.1.3, magnetorheological flow).
//
// The field outside the particles is H = -grad phi, phi = -H0 . x + S^L[q], with S^L the Laplace single
// layer (G = 1 / (4 pi |x - y|)); the jump conditions give the second-kind equation
// (1/2 I + eta K^L) q = eta H0 . n, eta = (mu - mu0) / (mu + mu0), K^L the target normal derivative of
// S^L (kernel -(r . n_x) / (4 pi |r|^3), r = x - y).  It is discretised like the mobility operators:
// the smooth rule over distinct particles, upsampled sources for near pairs, and the rotated-pole
// singular rule on each particle's own surface (scalar blocks, invariant under the particle's rotation,
// stored per shape with every row).  The smooth pair sums run in double-float arithmetic (about 1e-12),
// the near corrections and blocks in float64; the solve is float64 GMRES, right-preconditioned by the
// inverse of each particle's own 1/2 I + eta K^L block.
//
// On the fluid side of each surface the field is H = -grad_s phi + H_n n, the tangential gradient by
// spectral differentiation of phi on the particle's grid (Eq. 37) and H_n = H0 . n + q / 2 - K^L[q];
// the Maxwell traction mu0 [(H . n) H - |H|^2 n / 2] (mu0 = 1) integrates to each particle's magnetic
// force and torque, which enter the mobility problem like applied ones.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "dfloat.cuh"
#include "surface.cuh"

namespace rbs {

namespace {

constexpr double kInv4Pi = 1.0 / (4.0 * kPi);
constexpr int kMaxGridOrder = 32;  // the largest p that rbs_set_geometry accepts

// Kernel values of the scalar singular rule for one polar index j and all azimuthal k:
// C[(kind * nphi + k) * nrot + a] = omega_a J(s_a) kernel(x_t - x(s_a)), target t = (j, k), rotated
// point s_a = R_z(phi_k) rotpts[j][a]; kind 0 = K^L, kind 1 = S^L.  Grid (nrot / 128, nphi, shapes).
__global__ void k_lap_kernel_values(int nphi, int nrot, double tj, const int* shape_ids, RBS_SHAPE_ARGS,
                                    const double4* rotpts_j, double* Cbase, size_t perC) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
  if (a >= nrot) return;
  const ShapeRef S = RBS_SHAPE_REF(shape_ids[blockIdx.z]);
  double* C = Cbase + perC * blockIdx.z;
  double sp, cp;
  sincospi(2.0 * k / nphi, &sp, &cp);
  const double4 q = rotpts_j[a];
  const double st = sqrt(fmax(0.0, 1.0 - tj * tj));
  double xt[3], Jt, nt[3];
  eval_surface(S, st * cp, st * sp, tj, xt, &Jt, nt);
  double y[3], J, ny[3];
  eval_surface(S, cp * q.x - sp * q.y, sp * q.x + cp * q.y, q.z, y, &J, ny);
  const double r0 = xt[0] - y[0], r1 = xt[1] - y[1], r2 = xt[2] - y[2];
  const double inv = rsqrt(r0 * r0 + r1 * r1 + r2 * r2);
  const double wJ = q.w * J * kInv4Pi;
  C[(long long)(0 * nphi + k) * nrot + a] = -(r0 * nt[0] + r1 * nt[1] + r2 * nt[2]) * inv * inv * inv * wJ;
  C[(long long)(1 * nphi + k) * nrot + a] = inv * wJ;
}

// Scatter G[(kind * nphi + k) * np + (j' nphi + k')] into the scalar blocks: row t = j nphi + k,
// column s = j' nphi + (k' + k) mod nphi.  Grid (2 nphi np / 256, shapes).
__global__ void k_lap_scatter(int nphi, int np, int j, const double* Gbase, size_t perG, const long long* off,
                              double* BK, double* BS) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= 2LL * nphi * np) return;
  const double* G = Gbase + perG * blockIdx.y;
  const int col = (int)(i % np);
  const int row = (int)(i / np);
  const int k = row % nphi, kind = row / nphi;
  const int jp = col / nphi, kp = col % nphi;
  const int t = j * nphi + k, s = jp * nphi + (kp + k) % nphi;
  double* B = (kind == 0 ? BK : BS) + off[blockIdx.y];
  B[(long long)t * np + s] = G[i];
}

// M = 1/2 I + eta K^L_0 for every shape of a run (np x np each, contiguous).
__global__ void k_lap_precond_matrix(long long total, int np, double eta, const double* BK, double* M) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= total) return;
  const long long e = i % ((long long)np * np);
  M[i] = eta * BK[i] + ((e / np) == (e % np) ? 0.5 : 0.0);
}

// Basis values at the grid nodes for spectral differentiation: for retained harmonics (n <= p,
// m <= mmax, in the order m = 0..mmax, n = m..p, cos then sin), Yw[b][l] = Y_b(l) qw_l (quadrature
// weight of the unit sphere), Yt[l][b] = dY_b/dtheta(l), Yp[l][b] = (dY_b/dphi)(l) / sin(theta_l).
// One thread per node.
__global__ void k_basis_derivs(int p, int mmax, int nphi, int nb, const double* t, const double* lam, double* Yw,
                               double* Yt, double* Yp) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  const int np = (p + 1) * nphi;
  if (l >= np) return;
  const int j = l / nphi, k = l % nphi;
  const double ct = t[j], st = sqrt(fmax(0.0, 1.0 - ct * ct));
  const double phi = 2.0 * kPi * k / nphi;
  const double qw = 2.0 * kPi / nphi * lam[j];
  double P0[kMaxGridOrder + 1], P1[kMaxGridOrder + 1], P2[kMaxGridOrder + 1];
  double Q0[kMaxGridOrder + 1], Q1[kMaxGridOrder + 1], Q2[kMaxGridOrder + 1];
  double *Pm = P0, *Pc = P1, *Pp = P2, *Qm = Q0, *Qc = Q1, *Qp = Q2;
  double pmm = 0.28209479177387814;  // Pbar_0^0 = 1 / sqrt(4 pi)
  legendre_column(0, p, ct, st, pmm, Pc, Qc);
  double pmm_next = pmm;
  if (p >= 1) legendre_column(1, p, ct, st, pmm_next, Pp, Qp);
  const double r2 = 1.4142135623730951;
  int b = 0;
  for (int m = 0; m <= mmax; ++m) {
    double cm = 1.0, sm = 0.0;
    if (m > 0) sincos(m * phi, &sm, &cm);
    for (int n = m; n <= p; ++n) {
      double dP;
      if (m == 0) {
        dP = (n >= 1) ? -sqrt(n * (n + 1.0)) * Pp[n] : 0.0;
      } else {
        const double up = (m + 1 <= n) ? sqrt((n + m + 1.0) * (n - m)) * Pp[n] : 0.0;
        dP = 0.5 * (sqrt((n + m) * (n - m + 1.0)) * Pm[n] - up);
      }
      if (m == 0) {
        Yw[(long long)b * np + l] = Pc[n] * qw;
        Yt[(long long)l * nb + b] = dP;
        Yp[(long long)l * nb + b] = 0.0;
        ++b;
      } else {
        Yw[(long long)b * np + l] = r2 * Pc[n] * cm * qw;
        Yt[(long long)l * nb + b] = r2 * dP * cm;
        Yp[(long long)l * nb + b] = -r2 * m * Qc[n] * sm;
        Yw[(long long)(b + 1) * np + l] = r2 * Pc[n] * sm * qw;
        Yt[(long long)l * nb + b + 1] = r2 * dP * sm;
        Yp[(long long)l * nb + b + 1] = r2 * m * Qc[n] * cm;
        b += 2;
      }
    }
    double* tp = Pm;
    Pm = Pc;
    Pc = Pp;
    Pp = tp;
    tp = Qm;
    Qm = Qc;
    Qc = Qp;
    Qp = tp;
    if (m + 2 <= p) legendre_column(m + 2, p, ct, st, pmm_next, Pp, Qp);
  }
}

// Weighted scalar density w q as a double-float pair per node.
__global__ void k_weight_df1(long long N, const double4* __restrict__ x, const double* __restrict__ q,
                             float2* __restrict__ wq) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= N) return;
  const dflt a = df_split(x[t].w * q[t]);
  wq[t] = make_float2(a.h, a.l);
}

// The smooth scalar pair sums in double-float arithmetic (about 1e-12 relative, like float64 here, on
// the float32 pipes): positions staged from exact three-float splits relative to the item's first
// target, the weighted density as double-float pairs, tiles accumulated in double-float.
template <int KIND>
__global__ void __launch_bounds__(128, 8) k_lap_df(int nitems, const longlong4* __restrict__ work,
                                                   const float4* __restrict__ x3h, const float4* __restrict__ x3m,
                                                   const float4* __restrict__ x3l, const float4* __restrict__ nh,
                                                   const float4* __restrict__ nl, const float2* __restrict__ wq,
                                                   double scale, double* __restrict__ y) {
  constexpr int TS = 128;
  __shared__ float4 sph[TS], spl[TS];
  __shared__ float2 sq[TS];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const longlong4 w = work[it];
    const float4 oh = x3h[w.x], om = x3m[w.x], ol = x3l[w.x];
    const long long t = w.x + threadIdx.x;
    const bool valid = t < w.y;
    float4 ah = oh, am = om, al = ol, bh = make_float4(0, 0, 0, 0), bl = make_float4(0, 0, 0, 0);
    int pt = -1;
    if (valid) {
      ah = x3h[t];
      am = x3m[t];
      al = x3l[t];
      bh = nh[t];
      bl = nl[t];
      pt = __float_as_int(ah.w);
    }
    const dflt xt[3] = {df_diff3(ah.x, am.x, al.x, oh.x, om.x, ol.x), df_diff3(ah.y, am.y, al.y, oh.y, om.y, ol.y),
                        df_diff3(ah.z, am.z, al.z, oh.z, om.z, ol.z)};
    const dflt nt[3] = {{bh.x, bl.x}, {bh.y, bl.y}, {bh.z, bl.z}};
    dflt a = {0.0f, 0.0f};
    for (long long s0 = w.z; s0 < w.w; s0 += TS) {
      const int cnt = (int)min((long long)TS, w.w - s0);
      __syncthreads();
      if ((int)threadIdx.x < cnt) {
        const long long s = s0 + threadIdx.x;
        const float4 ph = x3h[s], pm = x3m[s], pl = x3l[s];
        const dflt px = df_diff3(ph.x, pm.x, pl.x, oh.x, om.x, ol.x);
        const dflt py = df_diff3(ph.y, pm.y, pl.y, oh.y, om.y, ol.y);
        const dflt pz = df_diff3(ph.z, pm.z, pl.z, oh.z, om.z, ol.z);
        sph[threadIdx.x] = make_float4(px.h, py.h, pz.h, ph.w);
        spl[threadIdx.x] = make_float4(px.l, py.l, pz.l, 0.0f);
        sq[threadIdx.x] = wq[s];
      }
      __syncthreads();
      dflt acc = {0.0f, 0.0f};
      for (int l = 0; l < cnt; ++l) {
        const float4 yh = sph[l], yl = spl[l];
        const float2 qq = sq[l];
        dflt d[3];
        d[0] = df_two_sum(xt[0].h, -yh.x);
        d[0].l += xt[0].l - yl.x;
        d[1] = df_two_sum(xt[1].h, -yh.y);
        d[1].l += xt[1].l - yl.y;
        d[2] = df_two_sum(xt[2].h, -yh.z);
        d[2].l += xt[2].l - yl.z;
        float p[3], e[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          p[c] = d[c].h * d[c].h;
          e[c] = fmaf(d[c].h, d[c].h, -p[c]);
          e[c] = fmaf(d[c].h + d[c].h, d[c].l, e[c]);
        }
        const dflt s1 = df_two_sum(p[0], p[1]);
        const dflt s2 = df_two_sum(s1.h, p[2]);
        const float r2l = s1.l + s2.l + e[0] + e[1] + e[2];
        const float r2h = s2.h;
        const float y0 = rsqrt_hw(r2h);
        const float q0 = y0 * y0;
        const float qe = fmaf(y0, y0, -q0);
        float tt = fmaf(r2h, q0, -1.0f);
        tt = fmaf(r2h, qe, tt);
        tt = fmaf(r2l, q0, tt);
        dflt inv = {y0, -0.5f * tt * y0};
        if (__float_as_int(yh.w) == pt) inv = {0.0f, 0.0f};
        const dflt wqv = {qq.x, qq.y};
        if (KIND == 0) {
          const dflt rn = df_dot3(d[0], nt[0], d[1], nt[1], d[2], nt[2]);
          const dflt inv3 = df_mul(df_mul(inv, inv), inv);
          df_acc(acc, df_mul(df_mul(rn, inv3), wqv));
        } else {
          df_acc(acc, df_mul(inv, wqv));
        }
      }
      a = df_add_accurate(a, acc);
    }
    if (valid) atomicAdd(y + t, (KIND == 0 ? -scale : scale) * kInv4Pi * ((double)a.h + (double)a.l));
  }
}

// Upsampled scalar densities of the near-source particles: q_up = U q_j (U stored N_p x N_up).
__global__ void k_lap_upsample(int n_up, const int* __restrict__ up_particle, const long long* __restrict__ up_off,
                               const long long* __restrict__ offset, const int* __restrict__ nodes,
                               const double* const* __restrict__ Umats, const double* __restrict__ q,
                               double* __restrict__ qup) {
  for (int u = blockIdx.y; u < n_up; u += gridDim.y) {
    const int j = up_particle[u];
    const int np = nodes[j];
    const long long o = offset[j], base = up_off[u];
    const int nup = (int)(up_off[u + 1] - base);
    const double* Ut = Umats[u];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nup; r += gridDim.x * blockDim.x) {
      double a = 0.0;
      for (int s = 0; s < np; ++s) a = fma(Ut[(long long)s * nup + r], q[o + s], a);
      qup[base + r] = a;
    }
  }
}

// Near correction for one ordered near pair (i, j) per block: for targets of i, add the upsampled
// contribution of j and remove the smooth-rule one.
template <int KIND>
__global__ void __launch_bounds__(128) k_lap_near(const int2* __restrict__ near, const long long* __restrict__ offset,
                                                  const int* __restrict__ nodes, const int* __restrict__ up_index,
                                                  const long long* __restrict__ up_off, const double4* __restrict__ x,
                                                  const double4* __restrict__ nrm, const double* __restrict__ q,
                                                  const double4* __restrict__ up_x, const double* __restrict__ qup,
                                                  double scale, double* __restrict__ y) {
  const int2 pr = near[blockIdx.x];
  const long long oi = offset[pr.x], oj = offset[pr.y];
  const int ni = nodes[pr.x], nj = nodes[pr.y];
  const int u = up_index[pr.y];
  const long long ou = up_off[u];
  const int nu = (int)(up_off[u + 1] - ou);
  for (int tt = threadIdx.x; tt < ni; tt += blockDim.x) {
    const double4 xt = x[oi + tt], nt = nrm[oi + tt];
    double acc = 0.0;
    for (int a = 0; a < nu; ++a) {
      const double4 ps = up_x[ou + a];
      const double dx = xt.x - ps.x, dy = xt.y - ps.y, dz = xt.z - ps.z;
      const double inv = rsqrt(dx * dx + dy * dy + dz * dz);
      const double kv = KIND == 0 ? -(dx * nt.x + dy * nt.y + dz * nt.z) * inv * inv * inv : inv;
      acc = fma(kv, ps.w * qup[ou + a], acc);
    }
    for (int s = 0; s < nj; ++s) {
      const double4 ps = x[oj + s];
      const double dx = xt.x - ps.x, dy = xt.y - ps.y, dz = xt.z - ps.z;
      const double inv = rsqrt(dx * dx + dy * dy + dz * dz);
      const double kv = KIND == 0 ? -(dx * nt.x + dy * nt.y + dz * nt.z) * inv * inv * inv : inv;
      acc = fma(-kv, ps.w * q[oj + s], acc);
    }
    atomicAdd(y + oi + tt, scale * kInv4Pi * acc);
  }
}

// Scalar particle blocks: y_i = beta y_i + alpha B_shape(i) x_i + half x_i, one block per particle,
// a warp per row.
__global__ void __launch_bounds__(256) k_lap_blocks(const long long* __restrict__ offset, const int* __restrict__ nodes,
                                                    const int* __restrict__ shape_of,
                                                    const long long* __restrict__ block_off,
                                                    const double* __restrict__ B, const double* __restrict__ xin,
                                                    double alpha, double half, double* __restrict__ yout) {
  const int i = blockIdx.x;
  const int np = nodes[i];
  const long long o = offset[i];
  const double* A = B + block_off[shape_of[i]];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = warp; t < np; t += (int)(blockDim.x >> 5)) {
    double acc = 0.0;
    for (int s = lane; s < np; s += 32) acc = fma(A[(long long)t * np + s], xin[o + s], acc);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if (lane == 0) yout[o + t] = alpha * acc + half * xin[o + t];
  }
}

// Fluid-side field and Maxwell traction at every node of one particle per block: grad_s phi from the
// grid's differentiation matrices Dt, Dp (N_p x N_p each: d/dtheta and (d/dphi) / sin(theta)) and
// the lab-frame tangents; H = -grad_s phi + H_n n; f = (H . n) H - |H|^2 n / 2.
__global__ void __launch_bounds__(256) k_maxwell(const long long* __restrict__ offset, const int* __restrict__ pvec,
                                                 const int* __restrict__ nphivec, const int* __restrict__ shape_of,
                                                 RBS_SHAPE_ARGS, const double* __restrict__ rot,
                                                 const long long* __restrict__ gtab_off, const double* __restrict__ gtab,
                                                 const int* __restrict__ grid_of, const double* const* __restrict__ Dt,
                                                 const double* const* __restrict__ Dp,
                                                 const double4* __restrict__ nrm, const double* __restrict__ phi,
                                                 const double* __restrict__ Hn, double* __restrict__ f) {
  extern __shared__ double sphi[];
  const int i = blockIdx.x;
  const int p = pvec[i], nphi = nphivec[i], np = (p + 1) * nphi;
  const long long o = offset[i];
  for (int s = threadIdx.x; s < np; s += blockDim.x) sphi[s] = phi[o + s];
  __syncthreads();
  const ShapeRef S = RBS_SHAPE_REF(shape_of[i]);
  const double* R = rot + 9 * i;
  const double* t = gtab + gtab_off[i];
  const double* DT = Dt[grid_of[i]];
  const double* DP = Dp[grid_of[i]];
  for (int l = threadIdx.x; l < np; l += blockDim.x) {
    double ft = 0.0, fp = 0.0;
    for (int s = 0; s < np; ++s) {
      ft = fma(DT[(long long)l * np + s], sphi[s], ft);
      fp = fma(DP[(long long)l * np + s], sphi[s], fp);
    }
    const int j = l / nphi, k = l % nphi;
    const double ct = t[j], st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double sp, cp;
    sincospi(2.0 * k / nphi, &sp, &cp);
    double xb[3], J, nb[3], ab[3], bb[3];
    eval_surface(S, st * cp, st * sp, ct, xb, &J, nb, ab, bb);
    double a[3], b[3];
    for (int r = 0; r < 3; ++r) {
      a[r] = R[3 * r] * ab[0] + R[3 * r + 1] * ab[1] + R[3 * r + 2] * ab[2];
      b[r] = R[3 * r] * bb[0] + R[3 * r + 1] * bb[1] + R[3 * r + 2] * bb[2];
    }
    const double aa = a[0] * a[0] + a[1] * a[1] + a[2] * a[2], bq = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    const double abd = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    const double det = aa * bq - abd * abd;
    const double ca = (bq * ft - abd * fp) / det, cb = (aa * fp - abd * ft) / det;
    const double4 n = nrm[o + l];
    const double hn = Hn[o + l];
    const double H[3] = {-(ca * a[0] + cb * b[0]) + hn * n.x, -(ca * a[1] + cb * b[1]) + hn * n.y,
                         -(ca * a[2] + cb * b[2]) + hn * n.z};
    const double Hdn = H[0] * n.x + H[1] * n.y + H[2] * n.z, HH = H[0] * H[0] + H[1] * H[1] + H[2] * H[2];
    f[3 * (o + l) + 0] = Hdn * H[0] - 0.5 * HH * n.x;
    f[3 * (o + l) + 1] = Hdn * H[1] - 0.5 * HH * n.y;
    f[3 * (o + l) + 2] = Hdn * H[2] - 0.5 * HH * n.z;
  }
}

// F_i = sum w f, T_i = sum w (x - c_i) x f; one block (256 threads) per particle.
__global__ void __launch_bounds__(256) k_force_torque(const long long* __restrict__ offset,
                                                      const double4* __restrict__ x, const double* __restrict__ centre,
                                                      const double* __restrict__ f, double* __restrict__ FT) {
  __shared__ double red[8][6];
  const int i = blockIdx.x;
  const long long o = offset[i], e = offset[i + 1];
  double m[6] = {0, 0, 0, 0, 0, 0};
  for (long long t = o + threadIdx.x; t < e; t += blockDim.x) {
    const double4 p = x[t];
    const double rx = p.x - centre[3 * i], ry = p.y - centre[3 * i + 1], rz = p.z - centre[3 * i + 2];
    const double a = p.w * f[3 * t], b = p.w * f[3 * t + 1], c = p.w * f[3 * t + 2];
    m[0] += a;
    m[1] += b;
    m[2] += c;
    m[3] += ry * c - rz * b;
    m[4] += rz * a - rx * c;
    m[5] += rx * b - ry * a;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) m[q] += __shfl_xor_sync(0xffffffffu, m[q], d);
  }
  if (lane == 0)
    for (int q = 0; q < 6; ++q) red[warp][q] = m[q];
  __syncthreads();
  if (threadIdx.x < 6) {
    double acc = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) acc += red[w][threadIdx.x];
    FT[6 * i + threadIdx.x] = acc;
  }
}

__global__ void k_h0_dot_n(long long N, const double4* __restrict__ nrm, double hx, double hy, double hz, double scale,
                           double* __restrict__ out) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= N) return;
  const double4 n = nrm[t];
  out[t] = scale * (hx * n.x + hy * n.y + hz * n.z);
}

__global__ void k_lin(long long N, double* __restrict__ y, double a, const double* __restrict__ x, double b) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < N) y[t] = a * x[t] + b * y[t];
}

__global__ void k_potential_base(long long N, const double4* __restrict__ x, double hx, double hy, double hz,
                                 double* __restrict__ out) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= N) return;
  const double4 p = x[t];
  out[t] = -(hx * p.x + hy * p.y + hz * p.z);
}

}  // namespace

// ------------------------------------------------------------------------------------------
// Host side.

// Scalar self blocks of every shape (np x np each, all rows) and the differentiation matrices of
// every grid; built once per geometry, on first use.
static Status build_laplace(Context& c) {
  MagState& M = c.mag;
  if (M.built) return Status::Ok();
  cudaStream_t s = c.stream;
  const int ns = (int)c.shapes.size();
  std::vector<long long> off(ns);
  long long total = 0;
  for (int k = 0; k < ns; ++k) {
    off[k] = total;
    total += (long long)c.shapes[k].np * c.shapes[k].np;
  }
  RBS_TRY(M.d_blockK.alloc(total));
  RBS_TRY(M.d_blockS.alloc(total));
  RBS_TRY(M.d_precond.alloc(total));
  M.block_off = off;
  RBS_TRY(M.d_block_off.alloc(ns));
  RBS_CUDA_TRY(cudaMemcpyAsync(M.d_block_off.ptr, off.data(), sizeof(long long) * ns, cudaMemcpyHostToDevice, s));
  for (size_t gi = 0; gi < c.grids.size(); ++gi) {
    Grid& g = *c.grids[gi];
    std::vector<int> ids;
    std::vector<long long> goff;
    for (int k = 0; k < ns; ++k)
      if (c.shapes[k].grid == (int)gi) {
        ids.push_back(k);
        goff.push_back(off[k]);
      }
    if (ids.empty()) continue;
    const long long rowsC = 2LL * g.nphi;
    const size_t perC = (size_t)rowsC * g.nrot, perG = (size_t)rowsC * g.np;
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>(ids.size(), ((size_t)1 << 27) / (perC + perG)));
    DevBuf<double> C, G;
    DevBuf<int> d_ids;
    DevBuf<long long> d_off;
    RBS_TRY(C.alloc(perC * chunk));
    RBS_TRY(G.alloc(perG * chunk));
    RBS_TRY(d_ids.alloc(ids.size()));
    RBS_TRY(d_off.alloc(goff.size()));
    RBS_CUDA_TRY(cudaMemcpyAsync(d_ids.ptr, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice, s));
    RBS_CUDA_TRY(cudaMemcpyAsync(d_off.ptr, goff.data(), sizeof(long long) * goff.size(), cudaMemcpyHostToDevice, s));
    for (size_t st = 0; st < ids.size(); st += chunk) {
      const int cnt = (int)std::min<size_t>(chunk, ids.size() - st);
      for (int j = 0; j <= g.p; ++j) {
        dim3 grd(cdiv(g.nrot, 128), g.nphi, cnt);
        k_lap_kernel_values<<<grd, 128, 0, s>>>(g.nphi, g.nrot, g.t[j], d_ids.ptr + st, RBS_SHAPE_PASS,
                                                (const double4*)g.d_rotpts.ptr + (size_t)j * g.nrot, C.ptr, perC);
        RBS_CUDA_TRY(cudaGetLastError());
        RBS_TRY(dgemm_batched(s, (int)rowsC, g.np, g.nrot, C.ptr, g.nrot, (long long)perC,
                              g.d_interp.ptr + (size_t)j * g.nrot * g.np, g.np, 0, G.ptr, g.np, (long long)perG, cnt));
        dim3 grs(cdiv(2LL * g.nphi * g.np, 256), cnt);
        k_lap_scatter<<<grs, 256, 0, s>>>(g.nphi, g.np, j, G.ptr, perG, d_off.ptr + st, M.d_blockK.ptr,
                                          M.d_blockS.ptr);
        RBS_CUDA_TRY(cudaGetLastError());
      }
    }
    RBS_CUDA_TRY(cudaStreamSynchronize(s));
  }
  // differentiation matrices per grid: Dt = Yt Yw, Dp = Yp Yw (N_p x N_p)
  M.d_Dt.resize(c.grids.size());
  M.d_Dp.resize(c.grids.size());
  std::vector<const double*> pt(c.grids.size()), pp(c.grids.size());
  for (size_t gi = 0; gi < c.grids.size(); ++gi) {
    Grid& g = *c.grids[gi];
    const int mmax = std::min(g.p, (g.nphi - 1) / 2);
    int nb = 0;
    for (int m = 0; m <= mmax; ++m) nb += (g.p - m + 1) * (m == 0 ? 1 : 2);
    DevBuf<double> Yw, Yt, Yp;
    RBS_TRY(Yw.alloc((size_t)nb * g.np));
    RBS_TRY(Yt.alloc((size_t)nb * g.np));
    RBS_TRY(Yp.alloc((size_t)nb * g.np));
    k_basis_derivs<<<cdiv(g.np, 128), 128, 0, s>>>(g.p, mmax, g.nphi, nb, g.d_t.ptr, g.d_lam.ptr, Yw.ptr, Yt.ptr, Yp.ptr);
    RBS_CUDA_TRY(cudaGetLastError());
    M.d_Dt[gi] = new DevBuf<double>();
    M.d_Dp[gi] = new DevBuf<double>();
    RBS_TRY(M.d_Dt[gi]->alloc((size_t)g.np * g.np));
    RBS_TRY(M.d_Dp[gi]->alloc((size_t)g.np * g.np));
    RBS_TRY(dgemm_batched(s, g.np, g.np, nb, Yt.ptr, nb, 0, Yw.ptr, g.np, 0, M.d_Dt[gi]->ptr, g.np, 0, 1));
    RBS_TRY(dgemm_batched(s, g.np, g.np, nb, Yp.ptr, nb, 0, Yw.ptr, g.np, 0, M.d_Dp[gi]->ptr, g.np, 0, 1));
    RBS_CUDA_TRY(cudaStreamSynchronize(s));
    pt[gi] = M.d_Dt[gi]->ptr;
    pp[gi] = M.d_Dp[gi]->ptr;
  }
  RBS_TRY(M.d_Dt_ptr.alloc(pt.size()));
  RBS_TRY(M.d_Dp_ptr.alloc(pp.size()));
  RBS_CUDA_TRY(cudaMemcpyAsync(M.d_Dt_ptr.ptr, pt.data(), sizeof(double*) * pt.size(), cudaMemcpyHostToDevice, s));
  RBS_CUDA_TRY(cudaMemcpyAsync(M.d_Dp_ptr.ptr, pp.data(), sizeof(double*) * pp.size(), cudaMemcpyHostToDevice, s));
  std::vector<int> grid_of(c.grid_of.begin(), c.grid_of.end());
  RBS_TRY(M.d_grid_of.alloc(grid_of.size()));
  RBS_CUDA_TRY(cudaMemcpyAsync(M.d_grid_of.ptr, grid_of.data(), sizeof(int) * grid_of.size(), cudaMemcpyHostToDevice, s));
  RBS_CUDA_TRY(cudaStreamSynchronize(s));
  M.eta = NAN;
  M.built = true;
  return Status::Ok();
}

// Interpolation matrices of the current near-source particles (the near list changes as particles
// move).
static Status refresh_near_sources(Context& c) {
  std::vector<const double*> U;
  for (int j : c.up_particle) U.push_back(c.grids[c.grid_of[j]]->d_up.ptr);
  RBS_TRY(c.mag.d_upU.alloc(std::max<size_t>(1, U.size())));
  if (!U.empty())
    RBS_CUDA_TRY(cudaMemcpyAsync(c.mag.d_upU.ptr, U.data(), sizeof(double*) * U.size(), cudaMemcpyHostToDevice, c.stream));
  return Status::Ok();
}

// The preconditioner (1/2 I + eta K^L_0)^{-1} of every shape, for this eta.
static Status laplace_precond(Context& c, double eta) {
  MagState& M = c.mag;
  if (M.eta == eta) return Status::Ok();
  const int ns = (int)c.shapes.size();
  int k = 0;
  while (k < ns) {
    int e = k + 1;
    while (e < ns && c.shapes[e].np == c.shapes[k].np) ++e;
    const int np = c.shapes[k].np;
    const long long total = (long long)(e - k) * np * np;
    k_lap_precond_matrix<<<cdiv(total, 256), 256, 0, c.stream>>>(total, np, eta, M.d_blockK.ptr + M.block_off[k],
                                                                 M.d_precond.ptr + M.block_off[k]);
    RBS_CUDA_TRY(cudaGetLastError());
    RBS_TRY(invert_batched(c, M.d_precond.ptr + M.block_off[k], np, e - k));
    k = e;
  }
  M.eta = eta;
  return Status::Ok();
}

// y = half x + scale (self + far + near)[kind] x for the scalar operators (kind 0 = K^L, 1 = S^L).
static Status apply_laplace(Context& c, int kind, double half, double scale, const double* x, double* y) {
  MagState& M = c.mag;
  cudaStream_t s = c.stream;
  const double* B = kind == 0 ? M.d_blockK.ptr : M.d_blockS.ptr;
  c.stats.launches++;
  k_lap_blocks<<<c.n, 256, 0, s>>>(c.d_offset.ptr, c.d_nodes.ptr, c.d_shape.ptr, M.d_block_off.ptr, B, x, scale, half, y);
  const int nw = (int)c.work.size();
  if (nw > 0) {
    RBS_TRY(M.d_wq.alloc(c.N));
    c.stats.launches += 2;
    k_weight_df1<<<cdiv(c.N, 256), 256, 0, s>>>(c.N, c.d_x.ptr, x, M.d_wq.ptr);
    const int grid = std::min(nw, 8 * std::max(1, c.sm_count));
#define RBS_LAP_ARGS nw, c.d_work.ptr, c.d_x3h.ptr, c.d_x3m.ptr, c.d_x3l.ptr, c.d_nrmh.ptr, c.d_nrml.ptr, M.d_wq.ptr, scale, y
    if (kind == 0)
      k_lap_df<0><<<grid, 128, 0, s>>>(RBS_LAP_ARGS);
    else
      k_lap_df<1><<<grid, 128, 0, s>>>(RBS_LAP_ARGS);
#undef RBS_LAP_ARGS
  }
  const int nn = (int)c.near_pairs.size();
  if (nn > 0) {
    RBS_TRY(M.d_qup.alloc(std::max<long long>(1, c.n_up_nodes)));
    int maxup = 0;
    for (Grid* g : c.grids) maxup = std::max(maxup, g->nup);
    const int nup_p = (int)c.up_particle.size();
    dim3 gu(cdiv(maxup, 128), (unsigned)std::min(nup_p, 65535));
    c.stats.launches += 2;
    k_lap_upsample<<<gu, 128, 0, s>>>(nup_p, c.d_up_particle.ptr, c.d_up_off.ptr, c.d_offset.ptr, c.d_nodes.ptr,
                                     M.d_upU.ptr, x, M.d_qup.ptr);
    if (kind == 0)
      k_lap_near<0><<<nn, 128, 0, s>>>(c.d_near.ptr, c.d_offset.ptr, c.d_nodes.ptr, c.d_up_index.ptr, c.d_up_off.ptr,
                                       c.d_x.ptr, c.d_nrm.ptr, x, c.d_up_x.ptr, M.d_qup.ptr, scale, y);
    else
      k_lap_near<1><<<nn, 128, 0, s>>>(c.d_near.ptr, c.d_offset.ptr, c.d_nodes.ptr, c.d_up_index.ptr, c.d_up_off.ptr,
                                       c.d_x.ptr, c.d_nrm.ptr, x, c.d_up_x.ptr, M.d_qup.ptr, scale, y);
  }
  RBS_CUDA_TRY(cudaGetLastError());
  return Status::Ok();
}

Status laplace_operator(Context& c, int kind, const double* x, double* y) {
  RBS_TRY(build_laplace(c));
  RBS_TRY(refresh_near_sources(c));
  return apply_laplace(c, kind, 0.0, 1.0, x, y);
}

Status magnetic_forces(Context& c, const double H0[3], double mu_ratio, double tol, double* FT_dev, double* q_out,
                       int* iters_out) {
  RBS_TRY(build_laplace(c));
  RBS_TRY(refresh_near_sources(c));
  MagState& M = c.mag;
  cudaStream_t s = c.stream;
  const long long N = c.N;
  const double eta = (mu_ratio - 1.0) / (mu_ratio + 1.0);
  RBS_TRY(M.d_q.alloc(N));
  RBS_TRY(M.d_b.alloc(N));
  RBS_TRY(M.d_phi.alloc(N));
  RBS_TRY(M.d_hn.alloc(N));
  RBS_TRY(M.d_f.alloc(3 * N));
  *iters_out = 0;
  if (eta == 0.0) {
    RBS_CUDA_TRY(cudaMemsetAsync(FT_dev, 0, sizeof(double) * 6 * c.n, s));
    RBS_CUDA_TRY(cudaMemsetAsync(M.d_q.ptr, 0, sizeof(double) * N, s));
    if (q_out) RBS_CUDA_TRY(cudaMemcpyAsync(q_out, M.d_q.ptr, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
    RBS_CUDA_TRY(cudaStreamSynchronize(s));
    return Status::Ok();
  }
  RBS_TRY(laplace_precond(c, eta));
  // (1/2 I + eta K^L) q = eta H0 . n
  c.stats.launches++;
  k_h0_dot_n<<<cdiv(N, 256), 256, 0, s>>>(N, c.d_nrm.ptr, H0[0], H0[1], H0[2], eta, M.d_b.ptr);
  double bn2 = 0.0;
  {
    std::vector<double> hb(N);
    RBS_CUDA_TRY(cudaMemcpyAsync(hb.data(), M.d_b.ptr, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
    RBS_CUDA_TRY(cudaStreamSynchronize(s));
    for (double v : hb) bn2 += v * v;
  }
  LinOp op;
  op.n = N;
  op.apply_A = [&c, eta](const double* x, double* y) { return apply_laplace(c, 0, 0.5, eta, x, y); };
  op.apply_P = [&c](const double* v, double* z, double*) {
    c.stats.launches++;
    k_lap_blocks<<<c.n, 256, 0, c.stream>>>(c.d_offset.ptr, c.d_nodes.ptr, c.d_shape.ptr, c.mag.d_block_off.ptr,
                                            c.mag.d_precond.ptr, v, 1.0, 0.0, z);
    RBS_CUDA_TRY(cudaGetLastError());
    return Status::Ok();
  };
  op.apply_AP = [&c, eta, &op](const double* v, double* w, double* z) {
    RBS_TRY(op.apply_P(v, z, nullptr));
    return apply_laplace(c, 0, 0.5, eta, z, w);
  };
  double res = 0.0;
  bool conv = false;
  RBS_TRY(gmres_op(c, op, M.d_b.ptr, M.d_q.ptr, true, tol * std::sqrt(bn2), c.opt.max_iters, iters_out, &res, &conv));
  if (!conv) return Status::Err(RBS_ENOTCONV, "magnetostatic GMRES did not converge");
  // phi = -H0 . x + S^L[q];  H_n = H0 . n + q / 2 - K^L[q]
  c.stats.launches += 3;
  k_potential_base<<<cdiv(N, 256), 256, 0, s>>>(N, c.d_x.ptr, H0[0], H0[1], H0[2], M.d_b.ptr);
  RBS_TRY(apply_laplace(c, 1, 0.0, 1.0, M.d_q.ptr, M.d_phi.ptr));
  k_lin<<<cdiv(N, 256), 256, 0, s>>>(N, M.d_phi.ptr, 1.0, M.d_b.ptr, 1.0);
  RBS_TRY(apply_laplace(c, 0, 0.5, -1.0, M.d_q.ptr, M.d_hn.ptr));
  k_h0_dot_n<<<cdiv(N, 256), 256, 0, s>>>(N, c.d_nrm.ptr, H0[0], H0[1], H0[2], 1.0, M.d_b.ptr);
  k_lin<<<cdiv(N, 256), 256, 0, s>>>(N, M.d_hn.ptr, 1.0, M.d_b.ptr, 1.0);
  // traction and its moments
  int maxnp = 0;
  for (Grid* g : c.grids) maxnp = std::max(maxnp, g->np);
  const size_t smem = sizeof(double) * maxnp;
  if (smem > 48 * 1024) RBS_CUDA_TRY(cudaFuncSetAttribute(k_maxwell, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  c.stats.launches += 2;
  k_maxwell<<<c.n, 256, smem, s>>>(c.d_offset.ptr, c.d_p.ptr, c.d_nphi.ptr, c.d_shape.ptr, RBS_SHAPE_PASS, c.d_rot.ptr,
                                   c.d_gtab_off.ptr, c.d_gtab.ptr, M.d_grid_of.ptr, M.d_Dt_ptr.ptr, M.d_Dp_ptr.ptr,
                                   c.d_nrm.ptr, M.d_phi.ptr, M.d_hn.ptr, M.d_f.ptr);
  k_force_torque<<<c.n, 256, 0, s>>>(c.d_offset.ptr, c.d_x.ptr, c.d_centre.ptr, M.d_f.ptr, FT_dev);
  RBS_CUDA_TRY(cudaGetLastError());
  if (q_out) RBS_CUDA_TRY(cudaMemcpyAsync(q_out, M.d_q.ptr, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  RBS_CUDA_TRY(cudaStreamSynchronize(s));
  return Status::Ok();
}

MagState::~MagState() { release(); }

void MagState::release() {
  for (DevBuf<double>* b : d_Dt) delete b;
  for (DevBuf<double>* b : d_Dp) delete b;
  d_Dt.clear();
  d_Dp.clear();
  built = false;
}

}  // namespace rbs
