// Hierarchical far field for the smooth pair sums: barycentric Lagrange treecodes (Wang, Krasny and
// Tlupova, 2020) in place of the fast multipole method of Section 3.1, one for the float32 applies of
// the inner solve and, optionally, one at higher degree for the double-float passes.
//
// Per suspension, an octree over the particle centres (a cell with more than one particle splits at
// the midpoint of its centres' bounding box; children in octant order, particles ascending).  Each
// cell has the box of its particles' nodes, the box midpoint as centre, a radius
// r = max_j (|c_j - centre| + R_j) bounding its nodes, and a node count.  The targets of each particle
// form one batch (its leaf cell); a depth-first traversal accepts a cell C for approximation when
//   r_B + r_C < theta d,  d >= r_B + r_C + near_delta  and  (n + 1)^3 < nodes(C),
// else descends, and evaluates the particles of unaccepted leaves directly.  An accepted cell
// carries (n + 1)^3 proxy points on the tensor Chebyshev grid of its box and charges
//   q_abc = sum_s L_a(y_s,x) L_b(y_s,y) L_c(y_s,z) w_s mu_s     (barycentric Lagrange basis L),
// recomputed for every apply; the pair kernels then treat proxy points as ordinary sources.
//
// Layout: one source array holds the N nodes followed by the proxy points of every accepted cell
// (float32: hi + lo positions and weighted density; double-float: three-float positions and float32
// pairs of weighted density, with float64 cluster charges); each target particle has a list of
// (first, count) segments into it: its own particle first (masked by particle id), then the directly
// evaluated particles, then its accepted cells.  Work items pair the targets of one particle (or a
// near-equal part of it, at most 512) with a run of those segments.  The host plan (plan_treecode)
// does no device work, so it also serves the host-only entry point rbs_treecode_plan.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "pairs32.cuh"
#include "pairsdf.cuh"

namespace rbs {

namespace {

constexpr int kTreeMaxQ = 11;        // degree <= 10
constexpr int kTreeMaxTargets = 512; // targets per work item at most
constexpr int kTreeTile32 = 128;     // sources per warp tile of the float32 treecode sum
constexpr int kTreeTileDf = 64;      // and of the double-float one
constexpr int kProxyPid = -3;        // particle id carried by proxy points (never a target's)

// Bounding box of each particle's nodes: lo (3) then hi (3) per particle.
__global__ void __launch_bounds__(128) k_particle_boxes(int n, const long long* __restrict__ offset,
                                                        const double4* __restrict__ x, double* __restrict__ out) {
  __shared__ double red[6][4];
  const int i = blockIdx.x;
  if (i >= n) return;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (long long t = offset[i] + threadIdx.x; t < offset[i + 1]; t += blockDim.x) {
    const double4 p = x[t];
    lo[0] = fmin(lo[0], p.x);
    lo[1] = fmin(lo[1], p.y);
    lo[2] = fmin(lo[2], p.z);
    hi[0] = fmax(hi[0], p.x);
    hi[1] = fmax(hi[1], p.y);
    hi[2] = fmax(hi[2], p.z);
  }
  for (int o = 16; o > 0; o >>= 1)
    for (int d = 0; d < 3; ++d) {
      lo[d] = fmin(lo[d], __shfl_down_sync(0xffffffffu, lo[d], o));
      hi[d] = fmax(hi[d], __shfl_down_sync(0xffffffffu, hi[d], o));
    }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    for (int d = 0; d < 3; ++d) {
      red[d][warp] = lo[d];
      red[3 + d][warp] = hi[d];
    }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int d = threadIdx.x;
    double v = red[d][0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = d < 3 ? fmin(v, red[d][w]) : fmax(v, red[d][w]);
    out[6 * (size_t)i + d] = v;
  }
}

// Float32 weighted density of the nodes, the sources' charges: q[t] = (w_t mu_t, 0).
__global__ void k_tree_node_charges(long long N, const double4* __restrict__ x, const double* __restrict__ dens,
                                    float4* __restrict__ q) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= N) return;
  const double w = x[t].w;
  q[t] = make_float4((float)(w * dens[3 * t]), (float)(w * dens[3 * t + 1]), (float)(w * dens[3 * t + 2]), 0.0f);
}

// Barycentric Lagrange basis of the nq Chebyshev points s (weights bw) at u in [-1, 1]; a point on a
// node gets that node's unit vector.
__device__ __forceinline__ void lagrange_row(float u, const float* s, const float* bw, int nq, float* L) {
  float t[kTreeMaxQ];
  float sum = 0.0f;
  int hit = -1;
#pragma unroll
  for (int k = 0; k < kTreeMaxQ; ++k) {
    t[k] = 0.0f;
    if (k < nq) {
      const float d = u - s[k];
      if (d == 0.0f)
        hit = k;
      else
        t[k] = bw[k] / d;
      sum += t[k];
    }
  }
#pragma unroll
  for (int k = 0; k < kTreeMaxQ; ++k)
    if (k < nq) L[k] = hit >= 0 ? (k == hit ? 1.0f : 0.0f) : t[k] / sum;
}

// Cluster charges: one block per (cluster, run of its particles); each thread owns up to
// kProxyPerThread proxy points and sums L_a L_b L_c q over the run's nodes, staged 256 at a time with
// their Lagrange rows; the partial charges are added atomically (the charges are zeroed first).
constexpr int kChargeThreads = 256;
constexpr int kProxyPerThread = (kTreeMaxQ * kTreeMaxQ * kTreeMaxQ + kChargeThreads - 1) / kChargeThreads;

__global__ void __launch_bounds__(kChargeThreads) k_tree_charges(const int4* __restrict__ items,
                                                                 const int* __restrict__ order,
                                                                 const long long* __restrict__ offset,
                                                                 const double4* __restrict__ x,
                                                                 const float4* __restrict__ qnode,
                                                                 const double* __restrict__ box,
                                                                 const float* __restrict__ cheb, int nq,
                                                                 float4* __restrict__ qproxy) {
  constexpr int TS = kChargeThreads;
  __shared__ float sL[3][TS][kTreeMaxQ];
  __shared__ float4 sq[TS];
  __shared__ float s_pts[kTreeMaxQ], s_bw[kTreeMaxQ];
  const int npx = nq * nq * nq;
  if (threadIdx.x < nq) {
    s_pts[threadIdx.x] = cheb[threadIdx.x];
    s_bw[threadIdx.x] = cheb[nq + threadIdx.x];
  }
  const int4 it = items[blockIdx.x];
  const int u = it.x;
  const double m0 = box[6 * (size_t)u], m1 = box[6 * (size_t)u + 1], m2 = box[6 * (size_t)u + 2];
  const double h0 = box[6 * (size_t)u + 3], h1 = box[6 * (size_t)u + 4], h2 = box[6 * (size_t)u + 5];
  int ka[kProxyPerThread], kb[kProxyPerThread], kc[kProxyPerThread];
  float acc[kProxyPerThread][3];
#pragma unroll
  for (int m = 0; m < kProxyPerThread; ++m) {
    const int k = threadIdx.x + kChargeThreads * m;
    ka[m] = k / (nq * nq);
    kb[m] = (k / nq) % nq;
    kc[m] = k % nq;
    acc[m][0] = acc[m][1] = acc[m][2] = 0.0f;
  }
  for (int pi = it.y; pi < it.z; ++pi) {
    const int j = order[pi];
    const long long o = offset[j], e = offset[j + 1];
    for (long long s0 = o; s0 < e; s0 += TS) {
      const int cnt = (int)min((long long)TS, e - s0);
      __syncthreads();
      if ((int)threadIdx.x < cnt) {
        const double4 p = x[s0 + threadIdx.x];
        lagrange_row((float)((p.x - m0) * h0), s_pts, s_bw, nq, sL[0][threadIdx.x]);
        lagrange_row((float)((p.y - m1) * h1), s_pts, s_bw, nq, sL[1][threadIdx.x]);
        lagrange_row((float)((p.z - m2) * h2), s_pts, s_bw, nq, sL[2][threadIdx.x]);
        sq[threadIdx.x] = qnode[s0 + threadIdx.x];
      }
      __syncthreads();
      for (int l = 0; l < cnt; ++l) {
        const float4 q = sq[l];
#pragma unroll
        for (int m = 0; m < kProxyPerThread; ++m) {
          if (threadIdx.x + kChargeThreads * m < npx) {
            const float f = sL[0][l][ka[m]] * sL[1][l][kb[m]] * sL[2][l][kc[m]];
            acc[m][0] = fmaf(f, q.x, acc[m][0]);
            acc[m][1] = fmaf(f, q.y, acc[m][1]);
            acc[m][2] = fmaf(f, q.z, acc[m][2]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int m = 0; m < kProxyPerThread; ++m) {
    const int k = threadIdx.x + kChargeThreads * m;
    if (k < npx) {
      float4* dst = qproxy + (size_t)u * npx + k;
      atomicAdd(&dst->x, acc[m][0]);
      atomicAdd(&dst->y, acc[m][1]);
      atomicAdd(&dst->z, acc[m][2]);
    }
  }
}

// The float32 treecode pair sum: the packed tile loop of the direct kernel (pairs32.cuh) over source
// tiles filled from the item's segments.  Coordinates are relative to the item's first target; tiles
// that may hold nodes of the targets' own particle (the first nmask sources) mask them by particle id.
// The block size is chosen at launch so that blockDim.x * NT covers the largest item (a whole particle
// where it fits).  Each warp stages its own tiles of 128 sources and never waits for the other warps
// of its block: a block of an odd warp count (five warps for a 144-node particle) spreads unevenly over
// the SM's four schedulers, so block-wide tiles left the warps of the lighter schedulers waiting at
// every tile barrier.  Registers are capped (64 at one target per thread: six 160-thread blocks per SM).
template <int KIND, int NT>
__global__ void __maxnreg__(NT == 1 ? 64 : (NT == 2 ? 128 : 168))
    k_tree32x2(int nitems, const TreeItem* __restrict__ items, const int2* __restrict__ segs,
               const float4* __restrict__ xhi, const float4* __restrict__ xlo, const float4* __restrict__ nrm32,
               const float4* __restrict__ shi, const float4* __restrict__ slo, const float4* __restrict__ sq,
               double* __restrict__ y) {
  constexpr int TW = kTreeTile32, SL = TW / 32;
  const int lane = threadIdx.x & 31;
  const int wbase = (threadIdx.x >> 5) * 32 * NT;  // the warp's targets: wbase + 32 u + lane of the item
  extern __shared__ __align__(16) float tree_smem32[];
  float* const ssx = tree_smem32 + (threadIdx.x >> 5) * (7 * TW);
  float* const ssy = ssx + TW;
  float* const ssz = ssx + 2 * TW;
  float* const srx = ssx + 3 * TW;
  float* const sry = ssx + 4 * TW;
  float* const srz = ssx + 5 * TW;
  int* const spid = reinterpret_cast<int*>(ssx + 6 * TW);
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const TreeItem w = items[it];
    // target slots of this warp that hold a target: u < nu (a warp owns 32 NT consecutive targets, so
    // only the item's last warp has empty slots; they are skipped, and a warp without targets skips
    // the item)
    const int nu = min(NT, max(0, (w.t1 - w.t0 - wbase + 31) / 32));
    if (nu == 0) continue;
    const float4 oh = xhi[w.t0], ol = xlo[w.t0];
    float2 xt[NT][3], nt[NT][3];
    int pt[NT];
    bool valid[NT];
#pragma unroll
    for (int u = 0; u < NT; ++u) {
      const int t = w.t0 + wbase + 32 * u + lane;
      valid[u] = t < w.t1;
      float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, n0 = 0.0f, n1 = 0.0f, n2 = 0.0f;
      pt[u] = -1;
      if (valid[u]) {
        const float4 ah = xhi[t], al = xlo[t], nn = nrm32[t];
        a0 = (ah.x - oh.x) + (al.x - ol.x);
        a1 = (ah.y - oh.y) + (al.y - ol.y);
        a2 = (ah.z - oh.z) + (al.z - ol.z);
        n0 = nn.x;
        n1 = nn.y;
        n2 = nn.z;
        pt[u] = __float_as_int(ah.w);
      }
      xt[u][0] = f2(a0, a0);
      xt[u][1] = f2(a1, a1);
      xt[u][2] = f2(a2, a2);
      nt[u][0] = f2(n0, n0);
      nt[u][1] = f2(n1, n1);
      nt[u][2] = f2(n2, n2);
    }
    float sa[NT][3], ea[NT][3];
#pragma unroll
    for (int u = 0; u < NT; ++u) sa[u][0] = sa[u][1] = sa[u][2] = ea[u][0] = ea[u][1] = ea[u][2] = 0.0f;
    int seg = w.s0, off = 0, done = 0;
    while (seg < w.s1) {
      // the source of each of this lane's slots (lane + 32 k) from a walk over consecutive segments
      // that every lane of the warp takes in step, then all of its loads at once
      int sidx[SL];
#pragma unroll
      for (int k = 0; k < SL; ++k) sidx[k] = 0;
      int filled = 0;
      while (filled < TW && seg < w.s1) {
        const int2 sg = segs[seg];
        const int take = min(sg.y - off, TW - filled);
#pragma unroll
        for (int k = 0; k < SL; ++k) {
          const int l = lane + 32 * k;
          if (l >= filled && l < filled + take) sidx[k] = sg.x + off + (l - filled);
        }
        filled += take;
        off += take;
        if (off >= sg.y) {
          ++seg;
          off = 0;
        }
      }
      const int cnt4 = (filled + 3) & ~3;
      __syncwarp();  // the warp's reads of the previous tile are done
#pragma unroll 2
      for (int k = 0; k < SL; ++k) {
        const int l = lane + 32 * k;
        if (l < filled) {
          const int s = sidx[k];
          const float4 ph = shi[s], pl = slo[s], q = sq[s];
          ssx[l] = (oh.x - ph.x) + (ol.x - pl.x);
          ssy[l] = (oh.y - ph.y) + (ol.y - pl.y);
          ssz[l] = (oh.z - ph.z) + (ol.z - pl.z);
          srx[l] = q.x;
          sry[l] = q.y;
          srz[l] = q.z;
          spid[l] = __float_as_int(ph.w);
        } else if (l < cnt4) {
          ssx[l] = ssy[l] = ssz[l] = 1.0e4f;
          srx[l] = sry[l] = srz[l] = 0.0f;
          spid[l] = -2;
        }
      }
      __syncwarp();
      float2 p[NT][3];
#pragma unroll
      for (int u = 0; u < NT; ++u) p[u][0] = p[u][1] = p[u][2] = f2(0.0f, 0.0f);
#define RBS_TILE(NUV)                                                                              \
  do {                                                                                             \
    if (done < w.nmask)                                                                            \
      pair_tile32x2<KIND, true, NT, NUV>(ssx, ssy, ssz, srx, sry, srz, spid, cnt4, xt, nt, pt, p);  \
    else                                                                                           \
      pair_tile32x2<KIND, false, NT, NUV>(ssx, ssy, ssz, srx, sry, srz, spid, cnt4, xt, nt, pt, p); \
  } while (0)
      if (nu == NT) {
        RBS_TILE(NT);
      } else if constexpr (NT > 1) {
        if (nu == 1) RBS_TILE(1);
        if constexpr (NT > 2) {
          if (nu == 2) RBS_TILE(2);
          if (nu == 3) RBS_TILE(3);
        }
      }
#undef RBS_TILE
      done += filled;
#pragma unroll
      for (int u = 0; u < NT; ++u)
#pragma unroll
        for (int c = 0; c < 3; ++c) two_sum_acc(sa[u][c], ea[u][c], p[u][c].x + p[u][c].y);
    }
    const double sc = KIND == 0 ? kTractionScale : kStokesletScale;
#pragma unroll
    for (int u = 0; u < NT; ++u) {
      if (!valid[u]) continue;
      const long long t = w.t0 + wbase + 32 * u + lane;
#pragma unroll
      for (int c = 0; c < 3; ++c) atomicAdd(y + 3 * t + c, sc * ((double)sa[u][c] + (double)ea[u][c]));
    }
  }
}

// ---- double-float layout (the treecode of the double-float passes)

constexpr int kTreeMaxQ64 = 13;  // degree <= 12
constexpr int kChargeTile64 = 128;
constexpr int kProxyPerThread64 = (kTreeMaxQ64 * kTreeMaxQ64 * kTreeMaxQ64 + kChargeThreads - 1) / kChargeThreads;

// Weighted density of the nodes as float32 pairs: (qh, ql)[t] = split(w_t mu_t).
__global__ void k_tree_df_node_charges(long long N, const double4* __restrict__ x, const double* __restrict__ dens,
                                       float4* __restrict__ qh, float4* __restrict__ ql) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= N) return;
  const double w = x[t].w;
  const dflt a = df_split(w * dens[3 * t]), b = df_split(w * dens[3 * t + 1]), e = df_split(w * dens[3 * t + 2]);
  qh[t] = make_float4(a.h, b.h, e.h, 0.0f);
  ql[t] = make_float4(a.l, b.l, e.l, 0.0f);
}

// Barycentric Lagrange basis in float64 (as lagrange_row).
__device__ __forceinline__ void lagrange_row64(double u, const double* s, const double* bw, int nq, double* L) {
  double t[kTreeMaxQ64];
  double sum = 0.0;
  int hit = -1;
#pragma unroll
  for (int k = 0; k < kTreeMaxQ64; ++k) {
    t[k] = 0.0;
    if (k < nq) {
      const double d = u - s[k];
      if (d == 0.0)
        hit = k;
      else
        t[k] = bw[k] / d;
      sum += t[k];
    }
  }
#pragma unroll
  for (int k = 0; k < kTreeMaxQ64; ++k)
    if (k < nq) L[k] = hit >= 0 ? (k == hit ? 1.0 : 0.0) : t[k] / sum;
}

// Cluster charges in float64 (as k_tree_charges, from the float64 density): q64[3 (u npx + k) + c].
__global__ void __launch_bounds__(kChargeThreads) k_tree_charges64(const int4* __restrict__ items,
                                                                   const int* __restrict__ order,
                                                                   const long long* __restrict__ offset,
                                                                   const double4* __restrict__ x,
                                                                   const double* __restrict__ dens,
                                                                   const double* __restrict__ box,
                                                                   const double* __restrict__ cheb, int nq,
                                                                   double* __restrict__ q64) {
  constexpr int TS = kChargeTile64;
  __shared__ double sL[3][TS][kTreeMaxQ64];
  __shared__ double sq[TS][3];
  __shared__ double s_pts[kTreeMaxQ64], s_bw[kTreeMaxQ64];
  const int npx = nq * nq * nq;
  if (threadIdx.x < nq) {
    s_pts[threadIdx.x] = cheb[threadIdx.x];
    s_bw[threadIdx.x] = cheb[nq + threadIdx.x];
  }
  const int4 it = items[blockIdx.x];
  const int u = it.x;
  const double m0 = box[6 * (size_t)u], m1 = box[6 * (size_t)u + 1], m2 = box[6 * (size_t)u + 2];
  const double h0 = box[6 * (size_t)u + 3], h1 = box[6 * (size_t)u + 4], h2 = box[6 * (size_t)u + 5];
  int ka[kProxyPerThread64], kb[kProxyPerThread64], kc[kProxyPerThread64];
  double acc[kProxyPerThread64][3];
#pragma unroll
  for (int m = 0; m < kProxyPerThread64; ++m) {
    const int k = threadIdx.x + kChargeThreads * m;
    ka[m] = k / (nq * nq);
    kb[m] = (k / nq) % nq;
    kc[m] = k % nq;
    acc[m][0] = acc[m][1] = acc[m][2] = 0.0;
  }
  for (int pi = it.y; pi < it.z; ++pi) {
    const int j = order[pi];
    const long long o = offset[j], e = offset[j + 1];
    for (long long s0 = o; s0 < e; s0 += TS) {
      const int cnt = (int)min((long long)TS, e - s0);
      __syncthreads();
      if ((int)threadIdx.x < cnt) {
        const long long t = s0 + threadIdx.x;
        const double4 p = x[t];
        lagrange_row64((p.x - m0) * h0, s_pts, s_bw, nq, sL[0][threadIdx.x]);
        lagrange_row64((p.y - m1) * h1, s_pts, s_bw, nq, sL[1][threadIdx.x]);
        lagrange_row64((p.z - m2) * h2, s_pts, s_bw, nq, sL[2][threadIdx.x]);
        sq[threadIdx.x][0] = p.w * dens[3 * t];
        sq[threadIdx.x][1] = p.w * dens[3 * t + 1];
        sq[threadIdx.x][2] = p.w * dens[3 * t + 2];
      }
      __syncthreads();
      for (int l = 0; l < cnt; ++l) {
        const double q0 = sq[l][0], q1 = sq[l][1], q2 = sq[l][2];
#pragma unroll
        for (int m = 0; m < kProxyPerThread64; ++m) {
          if (threadIdx.x + kChargeThreads * m < npx) {
            const double f = sL[0][l][ka[m]] * sL[1][l][kb[m]] * sL[2][l][kc[m]];
            acc[m][0] = fma(f, q0, acc[m][0]);
            acc[m][1] = fma(f, q1, acc[m][1]);
            acc[m][2] = fma(f, q2, acc[m][2]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int m = 0; m < kProxyPerThread64; ++m) {
    const int k = threadIdx.x + kChargeThreads * m;
    if (k < npx)
      for (int c = 0; c < 3; ++c) atomicAdd(q64 + 3 * ((size_t)u * npx + k) + c, acc[m][c]);
  }
}

// Float64 cluster charges to the float32 pairs the double-float kernel reads.
__global__ void k_tree_q64_split(long long count, const double* __restrict__ q64, float4* __restrict__ qh,
                                 float4* __restrict__ ql) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= count) return;
  const dflt a = df_split(q64[3 * k]), b = df_split(q64[3 * k + 1]), e = df_split(q64[3 * k + 2]);
  qh[k] = make_float4(a.h, b.h, e.h, 0.0f);
  ql[k] = make_float4(a.l, b.l, e.l, 0.0f);
}

// The double-float treecode pair sum: the packed double-float pair of the direct kernel (pairsdf.cuh)
// over source tiles filled from the item's segments (as k_tree32x2).  KIND 0 traction into y, 1
// Stokeslet into y, 2 traction into y and Stokeslet into y2.
// The double-float treecode pair sum: the packed double-float pair of the direct kernel (pairsdf.cuh)
// over source tiles filled from the item's segments (as k_tree32x2: each warp stages its own tiles, of
// 64 sources here, and never waits for the rest of its block).  KIND 0 traction into y, 1 Stokeslet
// into y, 2 traction into y and Stokeslet into y2.  Registers are capped (96 for one target per
// thread) so that four 160-thread blocks, the size a p = 8 particle's targets take, are resident per
// SM: the double-float pair is a long dependent chain, and with the uncapped 126 registers only three
// blocks (or, at two targets per thread, 238 registers and two 96-thread blocks: under five warps per
// SM) hid its latency.
template <int KIND, int NT>
__global__ void __maxnreg__(NT == 1 ? 96 : 168)
    k_tree_df2(int nitems, const TreeItem* __restrict__ items, const int2* __restrict__ segs,
               const float4* __restrict__ x3h, const float4* __restrict__ x3m, const float4* __restrict__ x3l,
               const float4* __restrict__ nh, const float4* __restrict__ nl, const float4* __restrict__ shi,
               const float4* __restrict__ smid, const float4* __restrict__ slo, const float4* __restrict__ sqh,
               const float4* __restrict__ sql, double* __restrict__ y, double* __restrict__ y2) {
  constexpr int TW = kTreeTileDf, SL = TW / 32;
  const int lane = threadIdx.x & 31;
  const int wbase = (threadIdx.x >> 5) * 32 * NT;  // the warp's targets: wbase + 32 u + lane of the item
  extern __shared__ __align__(16) float tree_smem_df[];
  // per warp: the tile (12 float rows and the particle ids), then the item's origin (three float4)
  float(*sa)[TW] = reinterpret_cast<float(*)[TW]>(tree_smem_df + (threadIdx.x >> 5) * (13 * TW + 12));
  int* const spid = reinterpret_cast<int*>(&sa[12][0]);
  float4* const org = reinterpret_cast<float4*>(&sa[13][0]);
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const TreeItem w = items[it];
    // target slots of this warp that hold a target (as k_tree32x2); a warp without targets skips
    const int nu = min(NT, max(0, (w.t1 - w.t0 - wbase + 31) / 32));
    if (nu == 0) continue;
    __syncwarp();  // the warp's reads of the previous item's origin are done
    if (lane == 0) {
      org[0] = x3h[w.t0];
      org[1] = x3m[w.t0];
      org[2] = x3l[w.t0];
    }
    __syncwarp();
    df2 xt[NT][3], nt[NT][3];
    int pt[NT];
    bool valid[NT];
#pragma unroll
    for (int u = 0; u < NT; ++u) {
      const int t = w.t0 + wbase + 32 * u + lane;
      valid[u] = t < w.t1;
      const float4 oh = org[0], om = org[1], ol = org[2];
      float4 ah = oh, am = om, al = ol, bh = make_float4(0, 0, 0, 0), bl = make_float4(0, 0, 0, 0);
      pt[u] = -1;
      if (valid[u]) {
        ah = x3h[t];
        am = x3m[t];
        al = x3l[t];
        bh = nh[t];
        bl = nl[t];
        pt[u] = __float_as_int(ah.w);
      }
      const dflt dx = df_diff3(ah.x, am.x, al.x, oh.x, om.x, ol.x), dy = df_diff3(ah.y, am.y, al.y, oh.y, om.y, ol.y),
                 dz = df_diff3(ah.z, am.z, al.z, oh.z, om.z, ol.z);
      xt[u][0] = {dup2(dx.h), dup2(dx.l)};
      xt[u][1] = {dup2(dy.h), dup2(dy.l)};
      xt[u][2] = {dup2(dz.h), dup2(dz.l)};
      nt[u][0] = {dup2(bh.x), dup2(bl.x)};
      nt[u][1] = {dup2(bh.y), dup2(bl.y)};
      nt[u][2] = {dup2(bh.z), dup2(bl.z)};
    }
    dflt a[NT][3], a2[NT][3];
#pragma unroll
    for (int u = 0; u < NT; ++u)
#pragma unroll
      for (int c = 0; c < 3; ++c) a[u][c] = a2[u][c] = dflt{0.0f, 0.0f};
    int seg = w.s0, off = 0, done = 0;
    while (seg < w.s1) {
      int sidx[SL];
#pragma unroll
      for (int k = 0; k < SL; ++k) sidx[k] = 0;
      int filled = 0;
      while (filled < TW && seg < w.s1) {
        const int2 sg = segs[seg];
        const int take = min(sg.y - off, TW - filled);
#pragma unroll
        for (int k = 0; k < SL; ++k) {
          const int l = lane + 32 * k;
          if (l >= filled && l < filled + take) sidx[k] = sg.x + off + (l - filled);
        }
        filled += take;
        off += take;
        if (off >= sg.y) {
          ++seg;
          off = 0;
        }
      }
      const int cnt2 = (filled + 1) & ~1;
      __syncwarp();  // the warp's reads of the previous tile are done
#pragma unroll 1
      for (int k = 0; k < SL; ++k) {
        const int l = lane + 32 * k;
        if (l < filled) {
          const int s = sidx[k];
          const float4 ph = shi[s], pm = smid[s], pl = slo[s], qh = sqh[s], ql = sql[s];
          const float4 oh = org[0], om = org[1], ol = org[2];
          const dflt px = df_diff3(ph.x, pm.x, pl.x, oh.x, om.x, ol.x);
          const dflt py = df_diff3(ph.y, pm.y, pl.y, oh.y, om.y, ol.y);
          const dflt pz = df_diff3(ph.z, pm.z, pl.z, oh.z, om.z, ol.z);
          sa[0][l] = px.h;
          sa[1][l] = px.l;
          sa[2][l] = py.h;
          sa[3][l] = py.l;
          sa[4][l] = pz.h;
          sa[5][l] = pz.l;
          sa[6][l] = qh.x;
          sa[7][l] = ql.x;
          sa[8][l] = qh.y;
          sa[9][l] = ql.y;
          sa[10][l] = qh.z;
          sa[11][l] = ql.z;
          spid[l] = __float_as_int(ph.w);
        } else if (l < cnt2) {
          sa[0][l] = sa[2][l] = sa[4][l] = 1.0e4f;
          sa[1][l] = sa[3][l] = sa[5][l] = 0.0f;
          for (int q = 6; q < 12; ++q) sa[q][l] = 0.0f;
          spid[l] = -2;
        }
      }
      __syncwarp();
      const bool masked = done < w.nmask;
      df2 acc[NT][3], acc2[NT][3];
#pragma unroll
      for (int u = 0; u < NT; ++u)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[u][c] = acc2[u][c] = df2{dup2(0.0f), dup2(0.0f)};
      for (int l = 0; l < cnt2; l += 2) {
        df2 ys[3], den[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          ys[c] = {*reinterpret_cast<const float2*>(&sa[2 * c][l]), *reinterpret_cast<const float2*>(&sa[2 * c + 1][l])};
          den[c] = {*reinterpret_cast<const float2*>(&sa[6 + 2 * c][l]),
                    *reinterpret_cast<const float2*>(&sa[7 + 2 * c][l])};
        }
        const int2 pp = *reinterpret_cast<const int2*>(&spid[l]);
#pragma unroll
        for (int u = 0; u < NT; ++u) {
          if (u < nu) {
            if (masked)
              pair2_df<KIND, true>(ys, den, pp, xt[u], nt[u], pt[u], acc[u], acc2[u]);
            else
              pair2_df<KIND, false>(ys, den, pp, xt[u], nt[u], pt[u], acc[u], acc2[u]);
          }
        }
      }
      done += filled;
#pragma unroll
      for (int u = 0; u < NT; ++u)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          a[u][c] = df_add_accurate(a[u][c], fold2(acc[u][c]));
          if (KIND == 2) a2[u][c] = df_add_accurate(a2[u][c], fold2(acc2[u][c]));
        }
    }
    const double sc = KIND == 1 ? kStokesletScale : kTractionScale;
#pragma unroll
    for (int u = 0; u < NT; ++u) {
      if (!valid[u]) continue;
      const long long t = w.t0 + wbase + 32 * u + lane;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        atomicAdd(y + 3 * t + c, sc * ((double)a[u][c].h + (double)a[u][c].l));
        if (KIND == 2) atomicAdd(y2 + 3 * t + c, kStokesletScale * ((double)a2[u][c].h + (double)a2[u][c].l));
      }
    }
  }
}

template <typename T>
Status upload_vec(DevBuf<T>& buf, const std::vector<T>& host, cudaStream_t s) {
  RBS_TRY(buf.alloc(std::max<size_t>(1, host.size())));
  if (!host.empty())
    RBS_CUDA_TRY(cudaMemcpyAsync(buf.ptr, host.data(), sizeof(T) * host.size(), cudaMemcpyHostToDevice, s));
  return Status::Ok();
}

// Host octree cell.
struct HCell {
  int pb = 0, pe = 0;          // particles order[pb, pe)
  double lo[3], hi[3], cen[3];
  double r = 0.0;
  long long nodes = 0;
  int kid[8];
  int nkid = 0;
  int used = -1;               // index among the cells with proxy points
};

struct TreeBuilder {
  const PlanInput& c;
  const double* pbox;
  std::vector<int>& order;
  std::vector<HCell>& cells;
  std::vector<int>& leaf_of;

  int build(int pb, int pe, int depth) {
    HCell h;
    h.pb = pb;
    h.pe = pe;
    for (int d = 0; d < 3; ++d) {
      h.lo[d] = INFINITY;
      h.hi[d] = -INFINITY;
    }
    for (int q = pb; q < pe; ++q) {
      const int j = order[q];
      for (int d = 0; d < 3; ++d) {
        h.lo[d] = std::min(h.lo[d], pbox[6 * (size_t)j + d]);
        h.hi[d] = std::max(h.hi[d], pbox[6 * (size_t)j + 3 + d]);
      }
      h.nodes += c.offset[j + 1] - c.offset[j];
    }
    for (int d = 0; d < 3; ++d) h.cen[d] = 0.5 * (h.lo[d] + h.hi[d]);
    for (int q = pb; q < pe; ++q) {
      const int j = order[q];
      const double dx = c.centres[3 * j] - h.cen[0], dy = c.centres[3 * j + 1] - h.cen[1],
                   dz = c.centres[3 * j + 2] - h.cen[2];
      h.r = std::max(h.r, std::sqrt(dx * dx + dy * dy + dz * dz) + c.radius[j]);
    }
    const int id = (int)cells.size();
    cells.push_back(h);
    if (pe - pb > 1 && depth < 64) {
      double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
      for (int q = pb; q < pe; ++q)
        for (int d = 0; d < 3; ++d) {
          clo[d] = std::min(clo[d], c.centres[3 * order[q] + d]);
          chi[d] = std::max(chi[d], c.centres[3 * order[q] + d]);
        }
      double mid[3];
      for (int d = 0; d < 3; ++d) mid[d] = 0.5 * (clo[d] + chi[d]);
      // stable partition by octant (x the low bit), keeping ascending particle order in each
      std::vector<int> oct(pe - pb);
      int count[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int q = pb; q < pe; ++q) {
        const int j = order[q];
        const int o = (c.centres[3 * j] > mid[0] ? 1 : 0) + (c.centres[3 * j + 1] > mid[1] ? 2 : 0) +
                      (c.centres[3 * j + 2] > mid[2] ? 4 : 0);
        oct[q - pb] = o;
        ++count[o];
      }
      int groups = 0;
      for (int o = 0; o < 8; ++o) groups += count[o] > 0;
      if (groups > 1) {
        int start[8];
        int acc = pb;
        for (int o = 0; o < 8; ++o) {
          start[o] = acc;
          acc += count[o];
        }
        std::vector<int> tmp(pe - pb);
        int pos[8];
        for (int o = 0; o < 8; ++o) pos[o] = start[o] - pb;
        for (int q = pb; q < pe; ++q) tmp[pos[oct[q - pb]]++] = order[q];
        std::copy(tmp.begin(), tmp.end(), order.begin() + pb);
        int kids[8], nk = 0;
        for (int o = 0; o < 8; ++o)
          if (count[o] > 0) kids[nk++] = build(start[o], start[o] + count[o], depth + 1);
        for (int k = 0; k < nk; ++k) cells[id].kid[k] = kids[k];
        cells[id].nkid = nk;
        return id;
      }
    }
    for (int q = pb; q < pe; ++q) leaf_of[order[q]] = id;
    return id;
  }
};

}  // namespace

void TreeState::release() {
  active = false;
  tmax = 0;
  nt[0] = nt[1] = nt[2] = 0;
  n_cells = 0;
  n_src = 0;
  items.clear();
  segs.clear();
  charge_items.clear();
  for (DevBuf<float4>* b : {&d_hi, &d_lo, &d_q, &d_x3m, &d_wl}) b->release();
  d_items.release();
  d_segs.release();
  d_charge_items.release();
  d_order.release();
  d_box.release();
  d_cheb.release();
  d_cheb64.release();
  d_q64.release();
  df = false;
  direct_pairs = proxy_pairs = charge_work = 0;
}

double f32_operator_error(const Context& c) {
  constexpr double kF32OperatorError = 1e-5;  // float32 rounding of one apply (measured: a few 1e-7)
  if (!c.tree.active) return kF32OperatorError;
  // empirical model of the treecode's relative error: C(theta) rho^-n with rho the Bernstein ellipse
  // parameter 1/theta + sqrt(1/theta^2 - 1) and C = 0.25 max(1, (theta / 0.5)^2)
  const double th = c.tree.theta, a = 1.0 / th;
  const double C = 0.25 * std::max(1.0, (th / 0.5) * (th / 0.5));
  return kF32OperatorError + C * std::pow(a + std::sqrt(a * a - 1.0), -c.tree.degree);
}

Status plan_treecode(const PlanInput& c, double theta, int degree, TreePlan& T) {
  const int n = c.n;
  const int nq = degree + 1, npx = nq * nq * nq;
  const double* pbox = c.pbox;

  // 2. one octree per suspension (particles of a suspension are contiguous)
  std::vector<int> order(n), leaf_of(n, -1), root_of(n, -1);
  std::vector<HCell> cells;
  cells.reserve(2 * (size_t)n + 8);
  TreeBuilder tb{c, pbox, order, cells, leaf_of};
  for (int a = 0; a < n;) {
    int e = a + 1;
    while (e < n && c.sid[e] == c.sid[a]) ++e;
    for (int q = a; q < e; ++q) order[q] = q;
    const int root = tb.build(a, e, 0);
    for (int q = a; q < e; ++q) root_of[q] = root;
    a = e;
  }

  // 3. interaction lists and source segments per target particle
  const long long N = c.offset[n];
  std::vector<std::vector<int2>> seg_of(n);
  std::vector<long long> proxy_src(n, 0);
  int n_used = 0;
  std::vector<int> used_cells;
  std::vector<int> stack;
  for (int i = 0; i < n; ++i) {
    const HCell& B = cells[leaf_of[i]];
    std::vector<int2>& L = seg_of[i];
    const int np_i = (int)(c.offset[i + 1] - c.offset[i]);
    L.push_back(make_int2((int)c.offset[i], np_i));
    std::vector<int> approx;
    stack.clear();
    stack.push_back(root_of[i]);
    while (!stack.empty()) {
      const int id = stack.back();
      stack.pop_back();
      const HCell& C = cells[id];
      const double dx = B.cen[0] - C.cen[0], dy = B.cen[1] - C.cen[1], dz = B.cen[2] - C.cen[2];
      const double d = std::sqrt(dx * dx + dy * dy + dz * dz);
      const double rr = B.r + C.r;
      if (rr < theta * d && d >= rr + c.near_delta && (long long)npx < C.nodes) {
        approx.push_back(id);
      } else if (C.nkid > 0) {
        for (int k = C.nkid - 1; k >= 0; --k) stack.push_back(C.kid[k]);
      } else {
        for (int q = C.pb; q < C.pe; ++q) {
          const int j = order[q];
          if (j != i) L.push_back(make_int2((int)c.offset[j], (int)(c.offset[j + 1] - c.offset[j])));
        }
      }
    }
    for (int id : approx) {
      if (cells[id].used < 0) {
        cells[id].used = n_used++;
        used_cells.push_back(id);
      }
      const long long first = N + (long long)cells[id].used * npx;
      if (first + npx > INT_MAX) return Status::Err(RBS_ENOMEM, "treecode: more than 2^31 sources");
      L.push_back(make_int2((int)first, npx));
      proxy_src[i] += npx;
    }
  }
  T.n_cells = n_used;
  T.n_src = N + (long long)n_used * npx;
  if (T.n_src > INT_MAX) return Status::Err(RBS_ENOMEM, "treecode: more than 2^31 sources");

  // 4. work items: target parts of each particle times runs of its segments, split so that the grid
  // has about 96 items per SM.  A particle is one part where it has at most `cap` nodes, else
  // near-equal parts; cap is the candidate (multiples of 32 up to 512, and the particle sizes up to
  // 512) whose items waste the fewest thread slots when every block covers the largest part in
  // steps of 32 targets (ties: the larger cap, fewer stagings per pair).
  std::vector<int> caps;
  for (int cap = 32; cap <= kTreeMaxTargets; cap += 32) caps.push_back(cap);
  for (int i = 0; i < n; ++i) {
    const int np_i = (int)(c.offset[i + 1] - c.offset[i]);
    if (np_i <= kTreeMaxTargets) caps.push_back(np_i);
  }
  std::sort(caps.begin(), caps.end());
  caps.erase(std::unique(caps.begin(), caps.end()), caps.end());
  int cap = 128;
  double best_eff = -1.0;
  for (int cand : caps) {
    long long parts = 0;
    int tmax = 0;
    for (int i = 0; i < n; ++i) {
      const int np_i = (int)(c.offset[i + 1] - c.offset[i]);
      const int k = (np_i + cand - 1) / cand;
      parts += k;
      tmax = std::max(tmax, (np_i + k - 1) / k);
    }
    const double eff = (double)N / ((double)parts * (double)((tmax + 31) / 32 * 32));
    if (eff >= best_eff * (1.0 - 1e-12)) {
      best_eff = eff;
      cap = cand;
    }
  }
  long long tiles = 0;
  T.tmax = 0;
  for (int i = 0; i < n; ++i) {
    const int np_i = (int)(c.offset[i + 1] - c.offset[i]);
    const int k = (np_i + cap - 1) / cap;
    tiles += k;
    T.tmax = std::max(T.tmax, (np_i + k - 1) / k);
  }
  const long long want = 96LL * std::max(1, c.sm_count);
  const int splits = (int)std::max(1LL, (want + tiles - 1) / std::max(1LL, tiles));
  T.items.clear();
  T.segs.clear();
  T.direct_pairs = T.proxy_pairs = 0;
  for (int i = 0; i < n; ++i) {
    const std::vector<int2>& L = seg_of[i];
    const int base = (int)T.segs.size();
    T.segs.insert(T.segs.end(), L.begin(), L.end());
    long long total = 0;
    for (const int2& g : L) total += g.y;
    const int chunks = (int)std::min<long long>(splits, std::max(1LL, total / 2048));
    // cut points at segment boundaries, each run about total / chunks sources
    std::vector<int> cut = {0};
    long long acc = 0;
    for (int k = 0; k < (int)L.size(); ++k) {
      acc += L[k].y;
      const int runs = (int)cut.size();
      if (runs < chunks && k + 1 < (int)L.size() && acc * chunks >= total * runs) cut.push_back(k + 1);
    }
    cut.push_back((int)L.size());
    const int np_i = (int)(c.offset[i + 1] - c.offset[i]);
    const int nparts = (np_i + cap - 1) / cap, psize = (np_i + nparts - 1) / nparts;
    for (int t0 = (int)c.offset[i]; t0 < (int)c.offset[i + 1]; t0 += psize) {
      const int t1 = std::min(t0 + psize, (int)c.offset[i + 1]);
      for (size_t r = 0; r + 1 < cut.size(); ++r) {
        TreeItem it{};
        it.t0 = t0;
        it.t1 = t1;
        it.s0 = base + cut[r];
        it.s1 = base + cut[r + 1];
        it.nmask = r == 0 ? np_i : 0;
        T.items.push_back(it);
      }
    }
    T.direct_pairs += (long long)np_i * (total - proxy_src[i]);
    T.proxy_pairs += (long long)np_i * proxy_src[i];
  }

  // 5. cluster boxes, proxy points (float64, index a (n+1)^2 + b (n+1) + c per cluster) and charge
  // blocks
  T.box.assign(6 * (size_t)std::max(1, n_used), 0.0);
  T.proxy.assign(3 * (size_t)n_used * npx, 0.0);
  T.corder.clear();
  T.charge_items.clear();
  T.charge_work = 0;
  for (int u = 0; u < n_used; ++u) {
    const HCell& C = cells[used_cells[u]];
    double mid[3], half[3];
    for (int d = 0; d < 3; ++d) {
      mid[d] = 0.5 * (C.lo[d] + C.hi[d]);
      half[d] = 0.5 * (C.hi[d] - C.lo[d]);
      T.box[6 * (size_t)u + d] = mid[d];
      T.box[6 * (size_t)u + 3 + d] = half[d] > 0.0 ? 1.0 / half[d] : 0.0;
    }
    for (int a = 0; a < nq; ++a)
      for (int b = 0; b < nq; ++b)
        for (int e = 0; e < nq; ++e) {
          const size_t k = (size_t)u * npx + ((size_t)a * nq + b) * nq + e;
          T.proxy[3 * k] = mid[0] + half[0] * std::cos(a * kPi / degree);
          T.proxy[3 * k + 1] = mid[1] + half[1] * std::cos(b * kPi / degree);
          T.proxy[3 * k + 2] = mid[2] + half[2] * std::cos(e * kPi / degree);
        }
    // charge blocks over the cell's particles, about 4,096 nodes each
    int q = C.pb;
    while (q < C.pe) {
      const int first = (int)T.corder.size();
      long long nodes = 0;
      while (q < C.pe && (nodes == 0 || nodes + (c.offset[order[q] + 1] - c.offset[order[q]]) <= 4096)) {
        nodes += c.offset[order[q] + 1] - c.offset[order[q]];
        T.corder.push_back(order[q]);
        ++q;
      }
      T.charge_items.push_back(make_int4(u, first, (int)T.corder.size(), 0));
    }
    T.charge_work += C.nodes * (long long)npx;
  }
  return Status::Ok();
}

// Tree, lists, work items and proxy points of one treecode (theta, degree) over the particles'
// node boxes pbox, on the device; df: sources in the double-float layout (positions as exact
// three-float splits, weighted densities and charges as float32 pairs, charges accumulated in float64).
static Status build_lists(Context& c, TreeState& T, const std::vector<double>& pbox, double theta, int degree,
                          bool df) {
  cudaStream_t s = c.stream;
  const int nq = degree + 1, npx = nq * nq * nq;
  const long long N = c.N;
  std::vector<double> radius(c.n);
  for (int i = 0; i < c.n; ++i) radius[i] = c.shapes[c.shape_of[i]].radius;
  const PlanInput in{c.n, c.offset.data(), c.centres.data(), radius.data(), c.sid.data(), pbox.data(),
                     c.opt.near_delta, c.sm_count};
  TreePlan P;
  RBS_TRY(plan_treecode(in, theta, degree, P));
  T.degree = degree;
  T.npx = npx;
  T.theta = theta;
  T.df = df;
  if (P.tmax != T.tmax) T.nt[0] = T.nt[1] = T.nt[2] = 0;  // the block shape changed: time the variants again
  T.tmax = P.tmax;
  T.n_cells = P.n_cells;
  T.n_src = P.n_src;
  T.direct_pairs = P.direct_pairs;
  T.proxy_pairs = P.proxy_pairs;
  T.charge_work = P.charge_work;
  T.items.swap(P.items);
  T.segs.swap(P.segs);
  T.charge_items.swap(P.charge_items);
  const int n_used = P.n_cells;
  std::vector<double>& box = P.box;
  std::vector<int>& corder = P.corder;
  std::vector<float4> phi((size_t)n_used * npx), plo((size_t)n_used * npx), pm(df ? (size_t)n_used * npx : 0);
  std::vector<double> cheb(2 * (size_t)nq);
  for (int k = 0; k < nq; ++k) {
    cheb[k] = std::cos(k * kPi / degree);
    cheb[nq + k] = ((k & 1) ? -1.0 : 1.0) * ((k == 0 || k == degree) ? 0.5 : 1.0);
  }
  // proxy points carry kProxyPid in the w bits of their hi position, like a node's particle id
  float proxy_w;
  {
    const int v = kProxyPid;
    std::memcpy(&proxy_w, &v, sizeof(float));
  }
  for (size_t k = 0; k < (size_t)n_used * npx; ++k) {
    float h[3], m[3], l[3];
    for (int d = 0; d < 3; ++d) {
      const double v = P.proxy[3 * k + d];
      h[d] = (float)v;
      const double r = v - (double)h[d];
      m[d] = (float)r;
      l[d] = df ? (float)(r - (double)m[d]) : 0.0f;
    }
    phi[k] = make_float4(h[0], h[1], h[2], proxy_w);
    if (df) {  // exact three-float split, as the nodes' x3h / x3m / x3l
      pm[k] = make_float4(m[0], m[1], m[2], 0.0f);
      plo[k] = make_float4(l[0], l[1], l[2], 0.0f);
    } else {   // float32 hi + lo, as the nodes' xhi / xlo
      plo[k] = make_float4(m[0], m[1], m[2], 0.0f);
    }
  }

  // 6. device copies
  RBS_TRY(upload_vec(T.d_items, T.items, s));
  RBS_TRY(upload_vec(T.d_segs, T.segs, s));
  RBS_TRY(upload_vec(T.d_charge_items, T.charge_items, s));
  RBS_TRY(upload_vec(T.d_order, corder, s));
  RBS_TRY(upload_vec(T.d_box, box, s));
  {
    std::vector<float> cheb32(cheb.begin(), cheb.end());
    if (df)
      RBS_TRY(upload_vec(T.d_cheb64, cheb, s));
    else
      RBS_TRY(upload_vec(T.d_cheb, cheb32, s));
    RBS_TRY(T.d_hi.alloc(T.n_src));
    RBS_TRY(T.d_lo.alloc(T.n_src));
    RBS_TRY(T.d_q.alloc(T.n_src));  // float32 charges, or the hi parts of the double-float ones
    const float4* node_hi = df ? c.d_x3h.ptr : c.d_xhi.ptr;
    const float4* node_lo = df ? c.d_x3l.ptr : c.d_xlo.ptr;
    RBS_CUDA_TRY(cudaMemcpyAsync(T.d_hi.ptr, node_hi, sizeof(float4) * N, cudaMemcpyDeviceToDevice, s));
    RBS_CUDA_TRY(cudaMemcpyAsync(T.d_lo.ptr, node_lo, sizeof(float4) * N, cudaMemcpyDeviceToDevice, s));
    if (df) {
      RBS_TRY(T.d_x3m.alloc(T.n_src));
      RBS_TRY(T.d_wl.alloc(T.n_src));
      RBS_TRY(T.d_q64.alloc(std::max<size_t>(1, 3 * (size_t)n_used * npx)));
      RBS_CUDA_TRY(cudaMemcpyAsync(T.d_x3m.ptr, c.d_x3m.ptr, sizeof(float4) * N, cudaMemcpyDeviceToDevice, s));
    }
    if (n_used > 0) {
      RBS_CUDA_TRY(cudaMemcpyAsync(T.d_hi.ptr + N, phi.data(), sizeof(float4) * phi.size(), cudaMemcpyHostToDevice, s));
      RBS_CUDA_TRY(cudaMemcpyAsync(T.d_lo.ptr + N, plo.data(), sizeof(float4) * plo.size(), cudaMemcpyHostToDevice, s));
      if (df)
        RBS_CUDA_TRY(cudaMemcpyAsync(T.d_x3m.ptr + N, pm.data(), sizeof(float4) * pm.size(), cudaMemcpyHostToDevice, s));
    }
    // the host vectors above must outlive their copies
    RBS_CUDA_TRY(cudaStreamSynchronize(s));
  }
  T.active = true;
  return Status::Ok();
}

Status build_far_field(Context& c) {
  c.stats.tree_pairs = c.stats.tree_proxy_pairs = c.stats.tree_df_pairs = c.stats.tree_df_proxy_pairs = 0;
  c.stats.tree_cells = c.stats.tree_df_cells = 0;
  if (c.opt.far_field == RBS_FAR_DIRECT || !prec_f32(c.opt.precision) || c.n == 0) {
    c.tree.release();
    c.tree_df.release();
    return Status::Ok();
  }
  cudaStream_t s = c.stream;
  const int n = c.n;
  // 1. node bounding boxes of the particles
  std::vector<double> pbox(6 * (size_t)n);
  {
    DevBuf<double> d_pbox;
    RBS_TRY(d_pbox.alloc(6 * (size_t)n));
    k_particle_boxes<<<n, 128, 0, s>>>(n, c.d_offset.ptr, c.d_x.ptr, d_pbox.ptr);
    RBS_CUDA_TRY(cudaGetLastError());
    RBS_CUDA_TRY(cudaMemcpyAsync(pbox.data(), d_pbox.ptr, sizeof(double) * pbox.size(), cudaMemcpyDeviceToHost, s));
    RBS_CUDA_TRY(cudaStreamSynchronize(s));
  }
  RBS_TRY(build_lists(c, c.tree, pbox, c.opt.tree_theta, c.opt.tree_degree, false));
  c.stats.tree_pairs = c.tree.direct_pairs + c.tree.proxy_pairs;
  c.stats.tree_proxy_pairs = c.tree.proxy_pairs;
  c.stats.tree_cells = c.tree.n_cells;
  if (c.opt.far_field == RBS_FAR_TREECODE_DF) {
    RBS_TRY(build_lists(c, c.tree_df, pbox, c.opt.tree_df_theta, c.opt.tree_df_degree, true));
    c.stats.tree_df_pairs = c.tree_df.direct_pairs + c.tree_df.proxy_pairs;
    c.stats.tree_df_proxy_pairs = c.tree_df.proxy_pairs;
    c.stats.tree_df_cells = c.tree_df.n_cells;
  } else {
    c.tree_df.release();
  }
  return Status::Ok();
}

// Launch of the treecode pair sum over the first `items` work items with nt targets per thread,
// blocks just large enough for the largest item.
static Status launch_tree(Context& c, int kind, int nt, int items, double* y) {
  TreeState& T = c.tree;
  const int threads = ((T.tmax + nt - 1) / nt + 31) / 32 * 32;
  const size_t smem = (size_t)(threads / 32) * 7 * kTreeTile32 * sizeof(float);  // one tile per warp
#define RBS_TREE_ARGS items, T.d_items.ptr, T.d_segs.ptr, c.d_xhi.ptr, c.d_xlo.ptr, c.d_nrm32.ptr, T.d_hi.ptr, T.d_lo.ptr, \
                      T.d_q.ptr, y
  auto grid = [&](const void* k) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem) != cudaSuccess || per_sm < 1) per_sm = 1;
    return std::max(1, std::min(items, per_sm * std::max(1, c.sm_count)));
  };
  if (kind == 0) {
    if (nt == 1)
      k_tree32x2<0, 1><<<grid((const void*)k_tree32x2<0, 1>), threads, smem, c.stream>>>(RBS_TREE_ARGS);
    else if (nt == 4)
      k_tree32x2<0, 4><<<grid((const void*)k_tree32x2<0, 4>), threads, smem, c.stream>>>(RBS_TREE_ARGS);
    else
      k_tree32x2<0, 2><<<grid((const void*)k_tree32x2<0, 2>), threads, smem, c.stream>>>(RBS_TREE_ARGS);
  } else {
    if (nt == 1)
      k_tree32x2<1, 1><<<grid((const void*)k_tree32x2<1, 1>), threads, smem, c.stream>>>(RBS_TREE_ARGS);
    else if (nt == 4)
      k_tree32x2<1, 4><<<grid((const void*)k_tree32x2<1, 4>), threads, smem, c.stream>>>(RBS_TREE_ARGS);
    else
      k_tree32x2<1, 2><<<grid((const void*)k_tree32x2<1, 2>), threads, smem, c.stream>>>(RBS_TREE_ARGS);
  }
#undef RBS_TREE_ARGS
  RBS_CUDA_TRY(cudaGetLastError());
  return Status::Ok();
}

// Targets per thread of the treecode pair sum: rbs_options.pair_variant when set (its targets per
// thread), otherwise the fastest of 1, 2 and 4 timed once per geometry and kind on a prefix of the
// work items (the charges of the current apply as sources, into a scratch output).
static int tree_variant(Context& c, int kind) {
  TreeState& T = c.tree;
  if (c.opt.pair_variant > 0) {
    const int v = c.opt.pair_variant > kPacked ? c.opt.pair_variant - kPacked : c.opt.pair_variant;
    return (v == 1 || v == 4) ? v : 2;
  }
  if (T.nt[kind]) return T.nt[kind];
  int best = 2;
  const int items = std::min<int>((int)T.items.size(), 8 * std::max(1, c.sm_count));
  double* scratch = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaMalloc(&scratch, sizeof(double) * 3 * c.N) == cudaSuccess && cudaEventCreate(&a) == cudaSuccess &&
      cudaEventCreate(&b) == cudaSuccess) {
    float best_ms = 1e30f;
    for (int nt : {1, 2, 4}) {
      if (((T.tmax + nt - 1) / nt + 31) / 32 * 32 > kTreeMaxTargets / nt) continue;  // block too large
      if (!launch_tree(c, kind, nt, items, scratch).ok()) continue;  // warm
      cudaEventRecord(a, c.stream);
      if (!launch_tree(c, kind, nt, items, scratch).ok()) continue;
      cudaEventRecord(b, c.stream);
      float ms = 0.0f;
      if (cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        best = nt;
      }
      c.stats.launches += 2;
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (scratch) cudaFree(scratch);
  cudaGetLastError();
  T.nt[kind] = best;
  return best;
}

Status apply_tree(Context& c, int kind, const double* x, double* y, int nt) {
  TreeState& T = c.tree;
  const long long N = c.N;
  {
    KernelTimer timer(c, RBS_KC_TREE);
    k_tree_node_charges<<<cdiv(N, 256), 256, 0, c.stream>>>(N, c.d_x.ptr, x, T.d_q.ptr);
    int launches = 1;
    if (T.n_cells > 0) {
      RBS_CUDA_TRY(cudaMemsetAsync(T.d_q.ptr + N, 0, sizeof(float4) * (size_t)T.n_cells * T.npx, c.stream));
      k_tree_charges<<<(unsigned)T.charge_items.size(), kChargeThreads, 0, c.stream>>>(
          T.d_charge_items.ptr, T.d_order.ptr, c.d_offset.ptr, c.d_x.ptr, T.d_q.ptr, T.d_box.ptr, T.d_cheb.ptr,
          T.degree + 1, T.d_q.ptr + N);
      launches = 2;
    }
    RBS_CUDA_TRY(cudaGetLastError());
    timer.done((double)T.charge_work, launches);
  }
  const int items = (int)T.items.size();
  if (items == 0) return Status::Ok();
  if (nt <= 0) nt = tree_variant(c, kind);
  KernelTimer timer(c, kind == 0 ? RBS_KC_PAIR_K32 : RBS_KC_PAIR_S32);
  RBS_TRY(launch_tree(c, kind, nt, items, y));
  RBS_CUDA_TRY(cudaGetLastError());
  timer.done((double)(T.direct_pairs + T.proxy_pairs));
  return Status::Ok();
}

// Launch of the double-float treecode pair sum over the first `items` work items.
static Status launch_tree_df(Context& c, int kind, int nt, int items, double* y, double* y2) {
  TreeState& T = c.tree_df;
  const int threads = ((T.tmax + nt - 1) / nt + 31) / 32 * 32;
  const size_t smem = (size_t)(threads / 32) * (13 * kTreeTileDf + 12) * sizeof(float);  // one tile per warp
#define RBS_TREE_DF_ARGS items, T.d_items.ptr, T.d_segs.ptr, c.d_x3h.ptr, c.d_x3m.ptr, c.d_x3l.ptr, c.d_nrmh.ptr, \
                         c.d_nrml.ptr, T.d_hi.ptr, T.d_x3m.ptr, T.d_lo.ptr, T.d_q.ptr, T.d_wl.ptr, y, y2
  auto grid = [&](const void* k) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem) != cudaSuccess || per_sm < 1) per_sm = 1;
    return std::max(1, std::min(items, per_sm * std::max(1, c.sm_count)));
  };
  if (kind == 0) {
    if (nt == 1)
      k_tree_df2<0, 1><<<grid((const void*)k_tree_df2<0, 1>), threads, smem, c.stream>>>(RBS_TREE_DF_ARGS);
    else
      k_tree_df2<0, 2><<<grid((const void*)k_tree_df2<0, 2>), threads, smem, c.stream>>>(RBS_TREE_DF_ARGS);
  } else if (kind == 1) {
    if (nt == 1)
      k_tree_df2<1, 1><<<grid((const void*)k_tree_df2<1, 1>), threads, smem, c.stream>>>(RBS_TREE_DF_ARGS);
    else
      k_tree_df2<1, 2><<<grid((const void*)k_tree_df2<1, 2>), threads, smem, c.stream>>>(RBS_TREE_DF_ARGS);
  } else {
    if (nt == 1)
      k_tree_df2<2, 1><<<grid((const void*)k_tree_df2<2, 1>), threads, smem, c.stream>>>(RBS_TREE_DF_ARGS);
    else
      k_tree_df2<2, 2><<<grid((const void*)k_tree_df2<2, 2>), threads, smem, c.stream>>>(RBS_TREE_DF_ARGS);
  }
#undef RBS_TREE_DF_ARGS
  RBS_CUDA_TRY(cudaGetLastError());
  return Status::Ok();
}

// Targets per thread of the double-float treecode pair sum: 1 or 2, timed once per configuration and
// kind on a prefix of the work items (the current charges as sources, into scratch outputs).
static int tree_df_variant(Context& c, int kind) {
  TreeState& T = c.tree_df;
  if (c.opt.pair_variant > 0) return (c.opt.pair_variant == 2 || c.opt.pair_variant == kPacked + 2) ? 2 : 1;
  if (T.nt[kind]) return T.nt[kind];
  int best = 1;
  // a prefix of eight items per SM: whole rounds of the persistent grid for either variant
  const int items = std::min<int>((int)T.items.size(), 8 * std::max(1, c.sm_count));
  double* scratch = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaMalloc(&scratch, sizeof(double) * 6 * c.N) == cudaSuccess && cudaEventCreate(&a) == cudaSuccess &&
      cudaEventCreate(&b) == cudaSuccess) {
    float best_ms = 1e30f;
    for (int nt : {1, 2}) {
      if (!launch_tree_df(c, kind, nt, items, scratch, scratch + 3 * c.N).ok()) continue;  // warm
      cudaEventRecord(a, c.stream);
      if (!launch_tree_df(c, kind, nt, items, scratch, scratch + 3 * c.N).ok()) continue;
      cudaEventRecord(b, c.stream);
      float ms = 0.0f;
      if (cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        best = nt;
      }
      c.stats.launches += 2;
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (scratch) cudaFree(scratch);
  cudaGetLastError();
  T.nt[kind] = best;
  return best;
}

Status apply_tree_df(Context& c, int kind, const double* x, double* y, double* y2) {
  TreeState& T = c.tree_df;
  const long long N = c.N;
  {
    KernelTimer timer(c, RBS_KC_TREE);
    k_tree_df_node_charges<<<cdiv(N, 256), 256, 0, c.stream>>>(N, c.d_x.ptr, x, T.d_q.ptr, T.d_wl.ptr);
    int launches = 1;
    if (T.n_cells > 0) {
      const long long np = (long long)T.n_cells * T.npx;
      RBS_CUDA_TRY(cudaMemsetAsync(T.d_q64.ptr, 0, sizeof(double) * 3 * (size_t)np, c.stream));
      k_tree_charges64<<<(unsigned)T.charge_items.size(), kChargeThreads, 0, c.stream>>>(
          T.d_charge_items.ptr, T.d_order.ptr, c.d_offset.ptr, c.d_x.ptr, x, T.d_box.ptr, T.d_cheb64.ptr,
          T.degree + 1, T.d_q64.ptr);
      k_tree_q64_split<<<cdiv(np, 256), 256, 0, c.stream>>>(np, T.d_q64.ptr, T.d_q.ptr + N, T.d_wl.ptr + N);
      launches = 3;
    }
    RBS_CUDA_TRY(cudaGetLastError());
    timer.done((double)T.charge_work, launches);
  }
  const int items = (int)T.items.size();
  if (items == 0) return Status::Ok();
  const int nt = tree_df_variant(c, kind);
  KernelTimer timer(c, kind == 0 ? RBS_KC_PAIR_KDF : (kind == 1 ? RBS_KC_PAIR_SDF : RBS_KC_PAIR_KSDF));
  RBS_TRY(launch_tree_df(c, kind, nt, items, y, y2));
  timer.done((double)(T.direct_pairs + T.proxy_pairs));
  return Status::Ok();
}

}  // namespace rbs
