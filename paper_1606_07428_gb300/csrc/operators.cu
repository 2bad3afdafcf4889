// The pieces of the discrete operators (Sections 2.1-2.3, 3, 3.1):
//  * particle-block kernel: each particle's own surface, y = R A0 R^T x with A0 its body-frame
//    singular-rule block (Eq. 38), fused with 1/2 x and the projection L of Eq. 26, or the
//    block-diagonal preconditioner of Section 3.2;
//  * smooth pair sums over node pairs of distinct particles (traction kernel of Eqs. 13 and 22 in
//    the GMRES matvec, Stokeslet of Eq. 10 for the velocity), float64 and float32 with compensated
//    accumulation;
//  * near correction: for near particle pairs, the base-grid contribution is replaced by the one
//    from the source's upsampled grid (Section 3: upsampling for close targets).
#include <algorithm>

#include "common.cuh"

namespace rbs {

namespace {

constexpr double kTractionScale = -3.0 / (4.0 * kPi);
constexpr double kStokesletScale = 1.0 / (8.0 * kPi);

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double rsq(double v) { return rsqrt(v); }
__device__ __forceinline__ float rsq(float v) { return rsqrtf(v); }
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------------------------------
// Particle-block kernel.  Block = (particle i, node range); 256 threads.  The body-frame input
// z = R_i^T x_i is staged in shared memory; each warp produces the three rows of one node at a
// time as dot products over the 3 N_p columns, then rotates back and adds 1/2 x and L x as the mode
// asks.  TB is the storage type of the blocks (float64 or float32).
template <typename TB>
__global__ void __launch_bounds__(256) k_blocks(int mode, const int4* __restrict__ bwork,
                                                const long long* __restrict__ offset, const int* __restrict__ nodes,
                                                const double* __restrict__ rot, const double* __restrict__ centre,
                                                const int* __restrict__ shape_of, const long long* __restrict__ block_off,
                                                const TB* __restrict__ blocks, const double4* __restrict__ x,
                                                const double* __restrict__ in, double* __restrict__ out,
                                                double* __restrict__ aux, double scale) {
  extern __shared__ double zs[];  // 3 N_p
  __shared__ double red[8][6];
  __shared__ double mom[6];
  const int4 wk = bwork[blockIdx.x];
  const int i = wk.x, np = nodes[i];
  const long long o = offset[i];
  const double* R = rot + 9 * i;
  const double R0 = R[0], R1 = R[1], R2 = R[2], R3 = R[3], R4 = R[4], R5 = R[5], R6 = R[6], R7 = R[7], R8 = R[8];
  const double cx = centre[3 * i], cy = centre[3 * i + 1], cz = centre[3 * i + 2];
  const bool has_block = (mode != kModeL);
  const bool has_L = (mode == kModeSelfK || mode == kModeL);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double m[6] = {0, 0, 0, 0, 0, 0};
  for (int s = threadIdx.x; s < np; s += blockDim.x) {
    const double* xs = in + 3 * (o + s);
    double a = xs[0], b = xs[1], cc = xs[2];
    if (has_block) {
      zs[3 * s + 0] = R0 * a + R3 * b + R6 * cc;
      zs[3 * s + 1] = R1 * a + R4 * b + R7 * cc;
      zs[3 * s + 2] = R2 * a + R5 * b + R8 * cc;
    }
    if (has_L) {
      double4 p = x[o + s];
      double rx = p.x - cx, ry = p.y - cy, rz = p.z - cz, w = p.w;
      m[0] += w * a;
      m[1] += w * b;
      m[2] += w * cc;
      m[3] += w * (ry * cc - rz * b);
      m[4] += w * (rz * a - rx * cc);
      m[5] += w * (rx * b - ry * a);
    }
  }
  if (has_L) {
#pragma unroll
    for (int q = 0; q < 6; ++q) m[q] = warp_sum(m[q]);
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < 6; ++q) red[warp][q] = m[q];
  }
  __syncthreads();
  if (has_L && threadIdx.x < 6) {
    double acc = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) acc += red[w][threadIdx.x];
    mom[threadIdx.x] = acc;
  }
  __syncthreads();
  const int dim = 3 * np;
  const TB* A = blocks + (has_block ? block_off[shape_of[i]] : 0);
  for (int t = wk.y + warp; t < wk.z; t += (blockDim.x >> 5)) {
    double y0 = 0.0, y1 = 0.0, y2 = 0.0;
    if (has_block) {
      const TB* r0 = A + (long long)(3 * t) * dim;
      const TB* r1 = r0 + dim;
      const TB* r2 = r1 + dim;
      for (int col = lane; col < dim; col += 32) {
        double z = zs[col];
        y0 = fma((double)r0[col], z, y0);
        y1 = fma((double)r1[col], z, y1);
        y2 = fma((double)r2[col], z, y2);
      }
      y0 = warp_sum(y0);
      y1 = warp_sum(y1);
      y2 = warp_sum(y2);
    }
    if (lane == 0) {
      const long long g = o + t;
      double l0 = R0 * y0 + R1 * y1 + R2 * y2;
      double l1 = R3 * y0 + R4 * y1 + R5 * y2;
      double l2 = R6 * y0 + R7 * y1 + R8 * y2;
      const double* xt = in + 3 * g;
      if (mode == kModeSelfK || mode == kModeSelfKNoL) {
        l0 += 0.5 * xt[0];
        l1 += 0.5 * xt[1];
        l2 += 0.5 * xt[2];
      }
      if (has_L) {
        double4 p = x[g];
        double rx = p.x - cx, ry = p.y - cy, rz = p.z - cz;
        // a + b x r
        l0 += mom[0] + (mom[4] * rz - mom[5] * ry);
        l1 += mom[1] + (mom[5] * rx - mom[3] * rz);
        l2 += mom[2] + (mom[3] * ry - mom[4] * rx);
      }
      if (mode == kModePrecond) {
        aux[3 * g + 0] = xt[0];
        aux[3 * g + 1] = xt[1];
        aux[3 * g + 2] = xt[2];
      }
      out[3 * g + 0] = scale * l0;
      out[3 * g + 1] = scale * l1;
      out[3 * g + 2] = scale * l2;
    }
  }
}

// ------------------------------------------------------------------------------------------
// Smooth pair sums in float64.  One block per work item (128 targets x a source range); each
// thread owns one target; sources are staged 128 at a time in shared memory with their weighted
// density w_s mu_s.  Pairs on the same particle are excluded (their contribution is the singular
// rule's); the select also removes the r = 0 self pair before it is used.
template <int KIND>
__global__ void __launch_bounds__(128) k_pairs64(const longlong4* __restrict__ work, const double4* __restrict__ x,
                                                 const double4* __restrict__ nrm, const int* __restrict__ pid,
                                                 const double* __restrict__ dens, double* __restrict__ y) {
  constexpr int TS = 128;
  __shared__ double4 sp[TS];
  __shared__ double4 sd[TS];
  __shared__ int spid[TS];
  const longlong4 w = work[blockIdx.x];
  const long long t = w.x + threadIdx.x;
  const bool valid = t < w.y;
  double4 xt = make_double4(0, 0, 0, 0), nt = make_double4(0, 0, 0, 0);
  int pt = -1;
  if (valid) {
    xt = x[t];
    nt = nrm[t];
    pt = pid[t];
  }
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (long long s0 = w.z; s0 < w.w; s0 += TS) {
    const int cnt = (int)min((long long)TS, w.w - s0);
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
      const long long s = s0 + threadIdx.x;
      double4 ps = x[s];
      const double* d = dens + 3 * s;
      sp[threadIdx.x] = ps;
      spid[threadIdx.x] = pid[s];
      sd[threadIdx.x] = make_double4(ps.w * d[0], ps.w * d[1], ps.w * d[2], 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int l = 0; l < cnt; ++l) {
      const double4 ps = sp[l];
      const double4 ds = sd[l];
      const double dx = xt.x - ps.x, dy = xt.y - ps.y, dz = xt.z - ps.z;
      const double r2 = dx * dx + dy * dy + dz * dz;
      double inv = rsqrt(r2);
      if (spid[l] == pt) inv = 0.0;
      const double rr = dx * ds.x + dy * ds.y + dz * ds.z;
      if (KIND == 0) {
        const double inv2 = inv * inv;
        const double rn = dx * nt.x + dy * nt.y + dz * nt.z;
        const double c = rn * rr * (inv2 * inv2 * inv);
        a0 = fma(c, dx, a0);
        a1 = fma(c, dy, a1);
        a2 = fma(c, dz, a2);
      } else {
        const double c = rr * (inv * inv * inv);
        a0 = fma(c, dx, fma(ds.x, inv, a0));
        a1 = fma(c, dy, fma(ds.y, inv, a1));
        a2 = fma(c, dz, fma(ds.z, inv, a2));
      }
    }
  }
  if (valid) {
    const double sc = KIND == 0 ? kTractionScale : kStokesletScale;
    atomicAdd(y + 3 * t + 0, sc * a0);
    atomicAdd(y + 3 * t + 1, sc * a1);
    atomicAdd(y + 3 * t + 2, sc * a2);
  }
}

// ------------------------------------------------------------------------------------------
// Smooth pair sums in float32.  Coordinates are taken relative to the first target of the block in
// float64 before rounding, so a float32 difference keeps the relative accuracy of the separation
// rather than of the absolute position.  Each 256-source tile is summed in float32 and added into
// a compensated (two-sum) float32 accumulator.  Tiles whose particles cannot meet the block's
// targets skip the same-particle test.
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float v) {
  float t = s + v;
  float bp = t - s;
  e += (s - (t - bp)) + (v - bp);
  s = t;
}

template <int KIND, bool MASK>
__device__ __forceinline__ void pair_tile32(const float4* __restrict__ sp, const float4* __restrict__ sd, int cnt,
                                            float xx, float xy, float xz, float nx, float ny, float nz, int pt,
                                            float& p0, float& p1, float& p2) {
#pragma unroll 8
  for (int l = 0; l < cnt; ++l) {
    const float4 ps = sp[l];
    const float4 ds = sd[l];
    const float dx = xx - ps.x, dy = xy - ps.y, dz = xz - ps.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float inv = rsqrtf(r2);
    if (MASK && __float_as_int(ps.w) == pt) inv = 0.0f;
    const float rr = fmaf(dx, ds.x, fmaf(dy, ds.y, dz * ds.z));
    if (KIND == 0) {
      const float inv2 = inv * inv;
      const float rn = fmaf(dx, nx, fmaf(dy, ny, dz * nz));
      const float c = (rn * rr) * (inv2 * inv2 * inv);
      p0 = fmaf(c, dx, p0);
      p1 = fmaf(c, dy, p1);
      p2 = fmaf(c, dz, p2);
    } else {
      const float c = rr * (inv * inv * inv);
      p0 = fmaf(c, dx, fmaf(ds.x, inv, p0));
      p1 = fmaf(c, dy, fmaf(ds.y, inv, p1));
      p2 = fmaf(c, dz, fmaf(ds.z, inv, p2));
    }
  }
}

template <int KIND>
__global__ void __launch_bounds__(128) k_pairs32(const longlong4* __restrict__ work, const double4* __restrict__ x,
                                                 const double4* __restrict__ nrm, const int* __restrict__ pid,
                                                 const double* __restrict__ dens, double* __restrict__ y) {
  constexpr int TS = 256;
  __shared__ float4 sp[TS];
  __shared__ float4 sd[TS];
  const longlong4 w = work[blockIdx.x];
  const long long t = w.x + threadIdx.x;
  const bool valid = t < w.y;
  const double4 org = x[w.x];
  float xx = 0, xy = 0, xz = 0, nx = 0, ny = 0, nz = 0;
  int pt = -1;
  if (valid) {
    double4 xt = x[t];
    double4 nt = nrm[t];
    xx = (float)(xt.x - org.x);
    xy = (float)(xt.y - org.y);
    xz = (float)(xt.z - org.z);
    nx = (float)nt.x;
    ny = (float)nt.y;
    nz = (float)nt.z;
    pt = pid[t];
  }
  const int pid_lo = pid[w.x], pid_hi = pid[w.y - 1];
  float s0a = 0, s1a = 0, s2a = 0, e0 = 0, e1 = 0, e2 = 0;
  for (long long s0 = w.z; s0 < w.w; s0 += TS) {
    const int cnt = (int)min((long long)TS, w.w - s0);
    __syncthreads();
    for (int l = threadIdx.x; l < cnt; l += blockDim.x) {
      const long long s = s0 + l;
      double4 ps = x[s];
      const double* d = dens + 3 * s;
      sp[l] = make_float4((float)(ps.x - org.x), (float)(ps.y - org.y), (float)(ps.z - org.z), __int_as_float(pid[s]));
      sd[l] = make_float4((float)(ps.w * d[0]), (float)(ps.w * d[1]), (float)(ps.w * d[2]), 0.0f);
    }
    __syncthreads();
    const int tlo = pid[s0], thi = pid[s0 + cnt - 1];
    float p0 = 0, p1 = 0, p2 = 0;
    if (thi < pid_lo || tlo > pid_hi)
      pair_tile32<KIND, false>(sp, sd, cnt, xx, xy, xz, nx, ny, nz, pt, p0, p1, p2);
    else
      pair_tile32<KIND, true>(sp, sd, cnt, xx, xy, xz, nx, ny, nz, pt, p0, p1, p2);
    two_sum_acc(s0a, e0, p0);
    two_sum_acc(s1a, e1, p1);
    two_sum_acc(s2a, e2, p2);
  }
  if (valid) {
    const double sc = KIND == 0 ? kTractionScale : kStokesletScale;
    atomicAdd(y + 3 * t + 0, sc * ((double)s0a + (double)e0));
    atomicAdd(y + 3 * t + 1, sc * ((double)s1a + (double)e1));
    atomicAdd(y + 3 * t + 2, sc * ((double)s2a + (double)e2));
  }
}

// ------------------------------------------------------------------------------------------
// Smooth pair sums in double-float arithmetic: each value is an unevaluated sum hi + lo of two
// float32 numbers (Dekker's and Knuth's error-free transformations with fused multiply-add), so the
// float32 pipes deliver about 44 bits per operation.  The reciprocal square root is one Newton step
// from rsqrtf, with the residual 1 - r^2 y0^2 formed by fused multiply-adds.  Each 128-source tile
// is summed in double-float and added into a float64 accumulator, so the sum keeps ~1e-12 relative
// accuracy.  Coordinates are relative to the block's first target as in the float32 kernel.
struct dflt {
  float h, l;
};
__device__ __forceinline__ dflt df_split(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ dflt df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dflt df_mul(dflt a, dflt b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return {p, e};
}
__device__ __forceinline__ dflt df_add(dflt a, dflt b) {
  dflt s = df_two_sum(a.h, b.h);
  s.l += a.l + b.l;
  const float h = s.h + s.l;
  return {h, s.l - (h - s.h)};
}
// acc += v with the low parts carried unnormalised (renormalised when the tile is flushed)
__device__ __forceinline__ void df_acc(dflt& acc, dflt v) {
  const dflt s = df_two_sum(acc.h, v.h);
  acc.h = s.h;
  acc.l += s.l + v.l;
}

template <int KIND, bool MASK>
__device__ __forceinline__ void pair_tile_df(const float4* __restrict__ sph, const float4* __restrict__ spl,
                                             const float4* __restrict__ sdh, const float4* __restrict__ sdl, int cnt,
                                             const dflt* xt, const dflt* nt, int pt, dflt* acc) {
  for (int l = 0; l < cnt; ++l) {
    const float4 yh = sph[l], yl = spl[l], dh = sdh[l], dl = sdl[l];
    dflt d[3];
    d[0] = df_two_sum(xt[0].h, -yh.x);
    d[0].l += xt[0].l - yl.x;
    d[1] = df_two_sum(xt[1].h, -yh.y);
    d[1].l += xt[1].l - yl.y;
    d[2] = df_two_sum(xt[2].h, -yh.z);
    d[2].l += xt[2].l - yl.z;
    // r^2 = sum of d_c^2
    float p[3], e[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      p[c] = d[c].h * d[c].h;
      e[c] = fmaf(d[c].h, d[c].h, -p[c]);
      e[c] = fmaf(d[c].h + d[c].h, d[c].l, e[c]);
    }
    dflt s1 = df_two_sum(p[0], p[1]);
    dflt s2 = df_two_sum(s1.h, p[2]);
    const float r2l = s1.l + s2.l + e[0] + e[1] + e[2];
    const float r2h = s2.h;
    // 1 / sqrt(r^2): y0 = rsqrtf, one Newton step
    const float y0 = rsqrtf(r2h);
    const float q = y0 * y0;
    const float qe = fmaf(y0, y0, -q);
    float t = fmaf(r2h, q, -1.0f);
    t = fmaf(r2h, qe, t);
    t = fmaf(r2l, q, t);
    dflt inv = {y0, -0.5f * t * y0};
    if (MASK && __float_as_int(yh.w) == pt) inv = {0.0f, 0.0f};
    const dflt den[3] = {{dh.x, dl.x}, {dh.y, dl.y}, {dh.z, dl.z}};
    dflt rr = df_mul(d[0], den[0]);
    rr = df_add(rr, df_mul(d[1], den[1]));
    rr = df_add(rr, df_mul(d[2], den[2]));
    const dflt inv2 = df_mul(inv, inv);
    const dflt inv3 = df_mul(inv2, inv);
    if (KIND == 0) {
      const dflt inv5 = df_mul(inv3, inv2);
      dflt rn = df_mul(d[0], nt[0]);
      rn = df_add(rn, df_mul(d[1], nt[1]));
      rn = df_add(rn, df_mul(d[2], nt[2]));
      const dflt cc = df_mul(df_mul(rn, rr), inv5);
#pragma unroll
      for (int c = 0; c < 3; ++c) df_acc(acc[c], df_mul(cc, d[c]));
    } else {
      const dflt cc = df_mul(rr, inv3);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        df_acc(acc[c], df_mul(den[c], inv));
        df_acc(acc[c], df_mul(cc, d[c]));
      }
    }
  }
}

template <int KIND>
__global__ void __launch_bounds__(128) k_pairs_df(const longlong4* __restrict__ work, const double4* __restrict__ x,
                                                  const double4* __restrict__ nrm, const int* __restrict__ pid,
                                                  const double* __restrict__ dens, double* __restrict__ y) {
  constexpr int TS = 128;
  __shared__ float4 sph[TS], spl[TS], sdh[TS], sdl[TS];
  const longlong4 w = work[blockIdx.x];
  const long long t = w.x + threadIdx.x;
  const bool valid = t < w.y;
  const double4 org = x[w.x];
  dflt xt[3] = {{0, 0}, {0, 0}, {0, 0}}, nt[3] = {{0, 0}, {0, 0}, {0, 0}};
  int pt = -1;
  if (valid) {
    const double4 a = x[t], nn = nrm[t];
    xt[0] = df_split(a.x - org.x);
    xt[1] = df_split(a.y - org.y);
    xt[2] = df_split(a.z - org.z);
    nt[0] = df_split(nn.x);
    nt[1] = df_split(nn.y);
    nt[2] = df_split(nn.z);
    pt = pid[t];
  }
  const int pid_lo = pid[w.x], pid_hi = pid[w.y - 1];
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (long long s0 = w.z; s0 < w.w; s0 += TS) {
    const int cnt = (int)min((long long)TS, w.w - s0);
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
      const long long s = s0 + threadIdx.x;
      const double4 ps = x[s];
      const double* dd = dens + 3 * s;
      const dflt px = df_split(ps.x - org.x), py = df_split(ps.y - org.y), pz = df_split(ps.z - org.z);
      const dflt d0 = df_split(ps.w * dd[0]), d1 = df_split(ps.w * dd[1]), d2 = df_split(ps.w * dd[2]);
      sph[threadIdx.x] = make_float4(px.h, py.h, pz.h, __int_as_float(pid[s]));
      spl[threadIdx.x] = make_float4(px.l, py.l, pz.l, 0.0f);
      sdh[threadIdx.x] = make_float4(d0.h, d1.h, d2.h, 0.0f);
      sdl[threadIdx.x] = make_float4(d0.l, d1.l, d2.l, 0.0f);
    }
    __syncthreads();
    const int tlo = pid[s0], thi = pid[s0 + cnt - 1];
    dflt acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    if (thi < pid_lo || tlo > pid_hi)
      pair_tile_df<KIND, false>(sph, spl, sdh, sdl, cnt, xt, nt, pt, acc);
    else
      pair_tile_df<KIND, true>(sph, spl, sdh, sdl, cnt, xt, nt, pt, acc);
    a0 += (double)acc[0].h + (double)acc[0].l;
    a1 += (double)acc[1].h + (double)acc[1].l;
    a2 += (double)acc[2].h + (double)acc[2].l;
  }
  if (valid) {
    const double sc = KIND == 0 ? kTractionScale : kStokesletScale;
    atomicAdd(y + 3 * t + 0, sc * a0);
    atomicAdd(y + 3 * t + 1, sc * a1);
    atomicAdd(y + 3 * t + 2, sc * a2);
  }
}

// ------------------------------------------------------------------------------------------
// Upsampled densities of the near-source particles: mu_up = U mu_j, one warp per upsampled node.
template <typename TU>
__global__ void __launch_bounds__(256) k_upsample(int n_up, const int* __restrict__ up_particle, const long long* __restrict__ up_off,
                                                  const long long* __restrict__ offset, const int* __restrict__ nodes,
                                                  const TU* const* __restrict__ Umats, const double* __restrict__ dens,
                                                  double* __restrict__ upmu) {
  extern __shared__ double mus[];  // 3 N_p
  for (int u = blockIdx.y; u < n_up; u += gridDim.y) {
  const int j = up_particle[u];
  const int np = nodes[j];
  const long long o = offset[j];
  __syncthreads();
  for (int l = threadIdx.x; l < 3 * np; l += blockDim.x) mus[l] = dens[3 * o + l];
  __syncthreads();
  const long long base = up_off[u];
  const int nup = (int)(up_off[u + 1] - base);
  const TU* U = Umats[u];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = blockIdx.x * 8 + warp; r < nup; r += gridDim.x * 8) {
    const TU* row = U + (long long)r * np;
    double a0 = 0, a1 = 0, a2 = 0;
    for (int s = lane; s < np; s += 32) {
      double uv = (double)row[s];
      a0 = fma(uv, mus[3 * s], a0);
      a1 = fma(uv, mus[3 * s + 1], a1);
      a2 = fma(uv, mus[3 * s + 2], a2);
    }
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    a2 = warp_sum(a2);
    if (lane == 0) {
      upmu[3 * (base + r) + 0] = a0;
      upmu[3 * (base + r) + 1] = a1;
      upmu[3 * (base + r) + 2] = a2;
    }
  }
  __syncthreads();
  }
}

// Near correction for one near pair (target particle i, source particle j): add the contribution
// of j's upsampled nodes and subtract that of j's base nodes (already in the smooth sum).  T is the
// arithmetic type; coordinates are relative to the target particle's centre.
template <int KIND, typename T>
__global__ void __launch_bounds__(256) k_near(const int2* __restrict__ near, const long long* __restrict__ offset,
                                              const int* __restrict__ nodes, const double* __restrict__ centre,
                                              const int* __restrict__ up_index, const long long* __restrict__ up_off,
                                              const double4* __restrict__ x, const double4* __restrict__ nrm,
                                              const double* __restrict__ dens, const double4* __restrict__ upx,
                                              const double* __restrict__ upmu, double* __restrict__ y) {
  constexpr int TS = 256;
  __shared__ T sx[TS][3];
  __shared__ T sd[TS][3];
  const int2 pr = near[blockIdx.x];
  const int i = pr.x, j = pr.y;
  const double cx = centre[3 * i], cy = centre[3 * i + 1], cz = centre[3 * i + 2];
  const long long oi = offset[i], oj = offset[j];
  const int npi = nodes[i], npj = nodes[j];
  const int u = up_index[j];
  const long long ub = up_off[u];
  const int nup = (int)(up_off[u + 1] - ub);
  const int total = nup + npj;
  for (int tb = 0; tb < npi; tb += blockDim.x) {
    const int tl = tb + threadIdx.x;
    const bool valid = tl < npi;
    T xx = 0, xy = 0, xz = 0, nx = 0, ny = 0, nz = 0;
    if (valid) {
      double4 xt = x[oi + tl], nt = nrm[oi + tl];
      xx = (T)(xt.x - cx);
      xy = (T)(xt.y - cy);
      xz = (T)(xt.z - cz);
      nx = (T)nt.x;
      ny = (T)nt.y;
      nz = (T)nt.z;
    }
    T a0 = 0, a1 = 0, a2 = 0;
    for (int s0 = 0; s0 < total; s0 += TS) {
      const int cnt = min(TS, total - s0);
      __syncthreads();
      for (int l = threadIdx.x; l < cnt; l += blockDim.x) {
        const int s = s0 + l;
        double4 ps;
        double d0, d1, d2, wgt;
        if (s < nup) {
          ps = upx[ub + s];
          wgt = ps.w;
          d0 = upmu[3 * (ub + s)];
          d1 = upmu[3 * (ub + s) + 1];
          d2 = upmu[3 * (ub + s) + 2];
        } else {
          ps = x[oj + (s - nup)];
          wgt = -ps.w;
          const double* d = dens + 3 * (oj + (s - nup));
          d0 = d[0];
          d1 = d[1];
          d2 = d[2];
        }
        sx[l][0] = (T)(ps.x - cx);
        sx[l][1] = (T)(ps.y - cy);
        sx[l][2] = (T)(ps.z - cz);
        sd[l][0] = (T)(wgt * d0);
        sd[l][1] = (T)(wgt * d1);
        sd[l][2] = (T)(wgt * d2);
      }
      __syncthreads();
      for (int l = 0; l < cnt; ++l) {
        const T dx = xx - sx[l][0], dy = xy - sx[l][1], dz = xz - sx[l][2];
        const T r2 = dx * dx + dy * dy + dz * dz;
        const T inv = rsq(r2);
        const T rr = dx * sd[l][0] + dy * sd[l][1] + dz * sd[l][2];
        if (KIND == 0) {
          const T inv2 = inv * inv;
          const T rn = dx * nx + dy * ny + dz * nz;
          const T c = rn * rr * (inv2 * inv2 * inv);
          a0 += c * dx;
          a1 += c * dy;
          a2 += c * dz;
        } else {
          const T c = rr * (inv * inv * inv);
          a0 += sd[l][0] * inv + c * dx;
          a1 += sd[l][1] * inv + c * dy;
          a2 += sd[l][2] * inv + c * dz;
        }
      }
    }
    if (valid) {
      const double sc = KIND == 0 ? kTractionScale : kStokesletScale;
      atomicAdd(y + 3 * (oi + tl) + 0, sc * (double)a0);
      atomicAdd(y + 3 * (oi + tl) + 1, sc * (double)a1);
      atomicAdd(y + 3 * (oi + tl) + 2, sc * (double)a2);
    }
  }
}

}  // namespace

// ------------------------------------------------------------------------------------------

Status apply_blocks(Context& c, int mode, int prec, const double* x, double* y, double* aux, double scale) {
  if (mode == kModeZero) {
    c.stats.launches += 1;
    RBS_CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(double) * 3 * c.N, c.stream));
    return Status::Ok();
  }
  size_t smem = sizeof(double) * 3 * (size_t)c.max_np;
  const int nb = (int)c.bwork.size();
  bool use32 = (prec == RBS_PREC_MIXED) && (mode == kModeSelfK || mode == kModeSelfKNoL || mode == kModeKOnlySelf ||
                                             mode == kModePrecond);
  const double bytes = (mode == kModeL) ? 0.0 : (double)c.particle_block_entries * (use32 ? 4.0 : 8.0);
  KernelTimer timer(c, RBS_KC_BLOCKS);
  if (use32) {
    const float* B = (mode == kModePrecond) ? c.d_precond32.ptr : c.d_blockK32.ptr;
    if (smem > 48 * 1024)
      RBS_CUDA_TRY(cudaFuncSetAttribute(k_blocks<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_blocks<float><<<nb, 256, smem, c.stream>>>(mode, c.d_bwork.ptr, c.d_offset.ptr, c.d_nodes.ptr, c.d_rot.ptr,
                                                 c.d_centre.ptr, c.d_shape.ptr, c.d_block_off.ptr, B, c.d_x.ptr, x, y,
                                                 aux, scale);
  } else {
    const double* B = (mode == kModePrecond) ? c.d_precond.ptr : (mode == kModeSelfS ? c.d_blockS.ptr : c.d_blockK.ptr);
    if (smem > 48 * 1024)
      RBS_CUDA_TRY(cudaFuncSetAttribute(k_blocks<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_blocks<double><<<nb, 256, smem, c.stream>>>(mode, c.d_bwork.ptr, c.d_offset.ptr, c.d_nodes.ptr, c.d_rot.ptr,
                                                  c.d_centre.ptr, c.d_shape.ptr, c.d_block_off.ptr, B, c.d_x.ptr, x, y,
                                                  aux, scale);
  }
  RBS_CUDA_TRY(cudaGetLastError());
  timer.done(bytes);
  return Status::Ok();
}

Status apply_pairs(Context& c, int kind, int prec, const double* x, double* y) {
  const int nw = (int)c.work.size();
  const bool f32 = (prec == RBS_PREC_MIXED);
  if (nw > 0) {
    int cls = f32 ? (kind == 0 ? RBS_KC_PAIR_K32 : RBS_KC_PAIR_S32) : (kind == 0 ? RBS_KC_PAIR_K64 : RBS_KC_PAIR_S64);
    if (prec == RBS_PREC_DF) cls = kind == 0 ? RBS_KC_PAIR_KDF : RBS_KC_PAIR_SDF;
    KernelTimer timer(c, cls);
    if (prec == RBS_PREC_DF) {
      if (kind == 0)
        k_pairs_df<0><<<nw, 128, 0, c.stream>>>(c.d_work.ptr, c.d_x.ptr, c.d_nrm.ptr, c.d_pid.ptr, x, y);
      else
        k_pairs_df<1><<<nw, 128, 0, c.stream>>>(c.d_work.ptr, c.d_x.ptr, c.d_nrm.ptr, c.d_pid.ptr, x, y);
    } else if (f32) {
      if (kind == 0)
        k_pairs32<0><<<nw, 128, 0, c.stream>>>(c.d_work.ptr, c.d_x.ptr, c.d_nrm.ptr, c.d_pid.ptr, x, y);
      else
        k_pairs32<1><<<nw, 128, 0, c.stream>>>(c.d_work.ptr, c.d_x.ptr, c.d_nrm.ptr, c.d_pid.ptr, x, y);
    } else {
      if (kind == 0)
        k_pairs64<0><<<nw, 128, 0, c.stream>>>(c.d_work.ptr, c.d_x.ptr, c.d_nrm.ptr, c.d_pid.ptr, x, y);
      else
        k_pairs64<1><<<nw, 128, 0, c.stream>>>(c.d_work.ptr, c.d_x.ptr, c.d_nrm.ptr, c.d_pid.ptr, x, y);
    }
    RBS_CUDA_TRY(cudaGetLastError());
    timer.done((double)c.stats.far_pairs);
  }
  const int nn = (int)c.near_pairs.size();
  if (nn > 0) {
    KernelTimer timer(c, RBS_KC_NEAR);
    size_t smem = sizeof(double) * 3 * (size_t)c.max_np;
    if (smem > 48 * 1024) {
      RBS_CUDA_TRY(cudaFuncSetAttribute(k_upsample<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      RBS_CUDA_TRY(cudaFuncSetAttribute(k_upsample<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    int maxup = 0;
    for (Grid* g : c.grids) maxup = std::max(maxup, g->nup);
    const int nup_p = (int)c.up_particle.size();
    dim3 gu(cdiv(maxup, 8), (unsigned)std::min(nup_p, 65535));
    if (f32)
      k_upsample<float><<<gu, 256, smem, c.stream>>>(nup_p, c.d_up_particle.ptr, c.d_up_off.ptr, c.d_offset.ptr, c.d_nodes.ptr,
                                                     c.d_upU32.ptr, x, c.d_up_mu.ptr);
    else
      k_upsample<double><<<gu, 256, smem, c.stream>>>(nup_p, c.d_up_particle.ptr, c.d_up_off.ptr, c.d_offset.ptr,
                                                      c.d_nodes.ptr, c.d_upU.ptr, x, c.d_up_mu.ptr);
    RBS_CUDA_TRY(cudaGetLastError());
#define RBS_NEAR_ARGS                                                                                            \
  c.d_near.ptr, c.d_offset.ptr, c.d_nodes.ptr, c.d_centre.ptr, c.d_up_index.ptr, c.d_up_off.ptr, c.d_x.ptr, \
      c.d_nrm.ptr, x, c.d_up_x.ptr, c.d_up_mu.ptr, y
    if (kind == 0) {
      if (f32)
        k_near<0, float><<<nn, 256, 0, c.stream>>>(RBS_NEAR_ARGS);
      else
        k_near<0, double><<<nn, 256, 0, c.stream>>>(RBS_NEAR_ARGS);
    } else {
      if (f32)
        k_near<1, float><<<nn, 256, 0, c.stream>>>(RBS_NEAR_ARGS);
      else
        k_near<1, double><<<nn, 256, 0, c.stream>>>(RBS_NEAR_ARGS);
    }
#undef RBS_NEAR_ARGS
    RBS_CUDA_TRY(cudaGetLastError());
    timer.done((double)c.near_pair_nodes, 2);
  }
  return Status::Ok();
}

Status apply_operator(Context& c, int op, int prec, const double* x, double* y) {
  switch (op) {
    case RBS_OP_A:
      RBS_TRY(apply_blocks(c, kModeSelfK, prec, x, y, nullptr, 1.0));
      return apply_pairs(c, 0, prec, x, y);
    case RBS_OP_HALF_K:
      RBS_TRY(apply_blocks(c, kModeSelfKNoL, prec, x, y, nullptr, 1.0));
      return apply_pairs(c, 0, prec, x, y);
    case RBS_OP_S:
      RBS_TRY(apply_blocks(c, kModeSelfS, prec, x, y, nullptr, 1.0));
      return apply_pairs(c, 1, prec, x, y);
    case RBS_OP_K_OFF:
      RBS_TRY(apply_blocks(c, kModeZero, prec, x, y, nullptr, 1.0));
      return apply_pairs(c, 0, prec, x, y);
    case RBS_OP_K_SELF:
      return apply_blocks(c, kModeKOnlySelf, prec, x, y, nullptr, 1.0);
    case RBS_OP_S_OFF:
      RBS_TRY(apply_blocks(c, kModeZero, prec, x, y, nullptr, 1.0));
      return apply_pairs(c, 1, prec, x, y);
    case RBS_OP_S_SELF:
      return apply_blocks(c, kModeSelfS, prec, x, y, nullptr, 1.0);
    case RBS_OP_L:
      return apply_blocks(c, kModeL, prec, x, y, nullptr, 1.0);
    default:
      return Status::Err(RBS_EINVAL, "unknown operator id " + std::to_string(op));
  }
}

}  // namespace rbs
