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
#include <type_traits>

#include <cuda_fp16.h>

#include "common.cuh"
#include "dfloat.cuh"
#include "pairs32.cuh"
#include "pairsdf.cuh"

namespace rbs {

namespace {


__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double rsq(double v) { return rsqrt(v); }

__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

template <typename TB>
__device__ __forceinline__ TB warp_sum_t(TB v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------------------------------
// Particle-block kernel.  Block = (particle i, node range); 256 threads.  The body-frame input
// z = R_i^T x_i is staged in shared memory; each warp produces the three rows of one node at a
// time as dot products over the 3 N_p columns, then rotates back and adds 1/2 x and L x as the mode
// asks.  TB is the storage type of the blocks (float64 or float32), and the arithmetic of the
// products and their sums.
template <typename TB>
__global__ void __launch_bounds__(256) k_blocks(int mode, const int4* __restrict__ bwork,
                                                const long long* __restrict__ offset, const int* __restrict__ nodes,
                                                const double* __restrict__ rot, const double* __restrict__ centre,
                                                const int* __restrict__ shape_of, const long long* __restrict__ block_off,
                                                const TB* __restrict__ blocks, const double4* __restrict__ x,
                                                const double* __restrict__ in, double* __restrict__ out,
                                                double* __restrict__ aux, double scale) {
  extern __shared__ __align__(16) unsigned char zs_raw[];
  TB* zs = reinterpret_cast<TB*>(zs_raw);  // 3 N_p values of the block type
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
      zs[3 * s + 0] = (TB)(R0 * a + R3 * b + R6 * cc);
      zs[3 * s + 1] = (TB)(R1 * a + R4 * b + R7 * cc);
      zs[3 * s + 2] = (TB)(R2 * a + R5 * b + R8 * cc);
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
  const int dim = 3 * np;  // even: n_phi is even, so N_p is
  const TB* A = blocks + (has_block ? block_off[shape_of[i]] : 0);
  // two nodes (six consecutive rows) per warp pass, two adjacent columns per lane
  for (int t0 = wk.y + 2 * warp; t0 < wk.z; t0 += 2 * (int)(blockDim.x >> 5)) {
    const int nn = (t0 + 1 < wk.z) ? 2 : 1;
    TB y[6] = {0, 0, 0, 0, 0, 0};
    if (has_block) {
      const TB* base = A + (long long)(3 * t0) * dim;
      for (int col = 2 * lane; col < dim; col += 64) {
        const TB z0 = zs[col], z1 = zs[col + 1];
#pragma unroll
        for (int r = 0; r < 6; ++r) {
          if (r < 3 * nn) {
            const TB v0 = __ldg(base + (long long)r * dim + col), v1 = __ldg(base + (long long)r * dim + col + 1);
            y[r] = fma_t(v0, z0, fma_t(v1, z1, y[r]));
          }
        }
      }
#pragma unroll
      for (int r = 0; r < 6; ++r) y[r] = warp_sum_t(y[r]);
    }
    if (lane < nn) {
      const int t = t0 + lane;
      const double y0 = (double)y[3 * lane], y1 = (double)y[3 * lane + 1], y2 = (double)y[3 * lane + 2];
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
// Particle-block kernel for shapes stored by the rows of their representative nodes (ellipsoids).
// The blocks commute with the grid's eight reflections g (node map g(.), sign matrix D_g):
// A_{g(t), g(s)} = D_g A_{t,s} D_g, so y_{g(t)} = D_g sum_s A_{t,s} (D_g z_{g(s)}) for each stored
// row t.  The eight reflected copies of z = R_i^T x_i are staged in shared memory, so each stored row
// is read once for all eight reflections (k_blocks_sym below); 1/2 x, L x and the preconditioner's
// copy of x are added as in k_blocks.
// Node (j, k) under the reflection g, without divisions (k in [0, n_phi)).
__device__ __forceinline__ int reflect_jk(int g, int j, int k, int p, int nphi) {
  if (g & 4) j = p - j;
  if (g & 2) k = k == 0 ? 0 : nphi - k;
  if (g & 1) {
    k = nphi / 2 - k;
    if (k < 0) k += nphi;
  }
  return j * nphi + k;
}

// Block entries stored as the bits of float16 / bfloat16.
struct F16Bits {
  uint16_t v;
};
struct BF16Bits {
  uint16_t v;
};

// Four consecutive entries of a staged block row, or of a staged input row, in the arithmetic type
// (one 16-, 8- or two 16-byte shared-memory loads; aligned to their size).
__device__ __forceinline__ void load_quad(const float* p, float (&v)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
}
__device__ __forceinline__ void load_quad(const double* p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
}
__device__ __forceinline__ void load_quad(const F16Bits* p, float (&v)[4]) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
  const float2 f1 = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  v[0] = f0.x, v[1] = f0.y, v[2] = f1.x, v[3] = f1.y;
}
__device__ __forceinline__ void load_quad(const BF16Bits* p, float (&v)[4]) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  v[0] = __uint_as_float(u.x << 16), v[1] = __uint_as_float(u.x & 0xffff0000u);
  v[2] = __uint_as_float(u.y << 16), v[3] = __uint_as_float(u.y & 0xffff0000u);
}

// Asynchronous global-to-shared copy of BYTES (4, 8 or 16) by one thread; src_bytes = 0 writes zeros
// and reads nothing.  Completion is tracked by commit groups.
template <int BYTES>
__device__ __forceinline__ void cp_async_zfill(uint32_t dst, const void* src, uint32_t src_bytes) {
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(dst), "l"(src), "n"(BYTES), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// TS: storage type of the block entries; TB: the arithmetic of the products and sums (float64 for
// float64 blocks, float32 otherwise).  One CTA of kSymWarps warps per particle.  Each warp takes one
// representative r at a time and streams its three rows through a ring of asynchronous copies, one
// step of 512 bytes a row (each lane copies 16 bytes of each row; the ring runs several steps ahead).
// Lane (c, h) = (lane mod 16, lane / 16) multiplies the column quads 4c + 64 s of the step with the
// reflected inputs z_g, g = 4h .. 4h + 3, keeping twelve partial sums; at the end of r a reduce-scatter
// over the sixteen column groups leaves reflection g's three sums in lanes 4g .. 4g + 3.  In float32
// arithmetic the row sums go to shared memory and every node is finished by the whole CTA at the end;
// in float64 lane 4g finishes node g(r) at once.
template <typename TS, typename TB>
__global__ void __launch_bounds__(kSymWarps * 32, sizeof(TB) == 4 ? 3 : 2)
    k_blocks_sym(int mode, const int* __restrict__ sym_list, const long long* __restrict__ offset,
                 const int* __restrict__ pvec, const int* __restrict__ nphivec, const double* __restrict__ rot,
                 const double* __restrict__ centre, const int* __restrict__ shape_of,
                 const long long* __restrict__ block_off, const TS* __restrict__ blocks, const double4* __restrict__ x,
                 const double* __restrict__ in, double* __restrict__ out, double* __restrict__ aux, double scale) {
  constexpr bool kF32 = sizeof(TB) == 4;
  constexpr int E = 16 / (int)sizeof(TS);  // entries of a 16-byte chunk
  constexpr int SC = 32 * E;               // columns of a step
  constexpr int S = sym_lane_bytes(sizeof(TS)) / 48;  // ring stages
  constexpr int kRingBytes = kSymWarps * 32 * sym_lane_bytes(sizeof(TS));
  extern __shared__ __align__(16) unsigned char zraw[];
  __shared__ TB red[kSymWarps][6];
  __shared__ TB mom[6];
  // float64 inputs in the block's arithmetic: float32 blocks convert on the integer pipe (the float64
  // pipe would otherwise bound this kernel: rotations, moments and the L term are float64-pipe work)
  auto cv = [](double d) -> TB {
    if constexpr (kF32)
      return f64_to_f32_trunc(d);
    else
      return d;
  };
  auto wide = [](TB v) -> double {
    if constexpr (kF32)
      return f32_to_f64_bits(v);
    else
      return v;
  };
  const int i = sym_list[blockIdx.x];
  const int p = pvec[i], nphi = nphivec[i], np = (p + 1) * nphi, dim = 3 * np;
  const int nk = nphi / 4 + 1, nrep = (p / 2 + 1) * nk;
  const int zs = sym_zstride(dim, sizeof(TB));
  TB* zg = reinterpret_cast<TB*>(zraw + kRingBytes);  // 8 rows of stride zs
  TB* ynode = zg + 8 * zs;                            // float32: 3 N_p row sums
  const long long o = offset[i];
  const double* R = rot + 9 * i;
  const TB R0 = cv(R[0]), R1 = cv(R[1]), R2 = cv(R[2]), R3 = cv(R[3]), R4 = cv(R[4]), R5 = cv(R[5]), R6 = cv(R[6]),
           R7 = cv(R[7]), R8 = cv(R[8]);
  const double cxd = centre[3 * i], cyd = centre[3 * i + 1], czd = centre[3 * i + 2];
  const TB sc = cv(scale);
  const bool has_block = (mode != kModeL);
  const bool has_L = (mode == kModeSelfK || mode == kModeL);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // the copies: step = (representative of this warp, SC-column slice), one commit group per step;
  // 16-byte copies where the rows are 16-byte aligned, else copies of two entries
  const TS* A = blocks + block_off[shape_of[i]];
  const int nst = (dim + SC - 1) / SC;
  const bool al16 = ((reinterpret_cast<uintptr_t>(A) & 15u) == 0) && (dim % E == 0);
  const uint32_t ring_l = static_cast<uint32_t>(__cvta_generic_to_shared(zraw)) + warp * (S * 3 * 512) + lane * 16;
  int iss_left = (has_block && warp < nrep) ? ((nrep - 1 - warp) / kSymWarps + 1) * nst : 0;
  int iss_it = 0, iss_slot = 0;
  const TS* iss_src = A + (long long)(3 * warp) * dim + E * lane;
  const long long rep_jump = (long long)3 * kSymWarps * dim - (long long)SC * nst;
  auto issue = [&]() {
    if (iss_left > 0) {
      // entries past the row end are zero-filled (nothing is read there)
      const int col = E * lane + SC * iss_it;
      const uint32_t dst = ring_l + iss_slot * (3 * 512);
      if (al16) {
        const bool inb = col < dim;
        const TS* s0 = inb ? iss_src : A;
        const long long d1 = inb ? dim : 0;
        const uint32_t nb = inb ? 16u : 0u;
        cp_async_zfill<16>(dst, s0, nb);
        cp_async_zfill<16>(dst + 512, s0 + d1, nb);
        cp_async_zfill<16>(dst + 1024, s0 + 2 * d1, nb);
      } else {
#pragma unroll
        for (int j = 0; j < E / 2; ++j) {
          constexpr int B2 = 2 * (int)sizeof(TS);
          const bool inb = col + 2 * j < dim;
          const TS* s0 = inb ? iss_src + 2 * j : A;
          const long long d1 = inb ? dim : 0;
          const uint32_t nb = inb ? (uint32_t)B2 : 0u;
          cp_async_zfill<B2>(dst + j * B2, s0, nb);
          cp_async_zfill<B2>(dst + 512 + j * B2, s0 + d1, nb);
          cp_async_zfill<B2>(dst + 1024 + j * B2, s0 + 2 * d1, nb);
        }
      }
      --iss_left;
      iss_src += SC;
      if (++iss_it == nst) {  // on to this warp's next representative
        iss_it = 0;
        iss_src += rep_jump;
      }
      iss_slot = (iss_slot + 1 == S) ? 0 : iss_slot + 1;
    }
    cp_async_commit();  // empty past the end
  };
  // the first stages load while the inputs are staged
  for (int q = 0; q < S - 1; ++q) issue();

  TB m[6] = {0, 0, 0, 0, 0, 0};
  for (int sp = threadIdx.x; sp < np; sp += blockDim.x) {
    const double* xs = in + 3 * (o + sp);
    const TB a = cv(xs[0]), b = cv(xs[1]), cc = cv(xs[2]);
    if (has_block) {
      const TB z0 = R0 * a + R3 * b + R6 * cc;
      const TB z1 = R1 * a + R4 * b + R7 * cc;
      const TB z2 = R2 * a + R5 * b + R8 * cc;
      const int js = sp / nphi, ks = sp - js * nphi;
#pragma unroll
      for (int g = 0; g < 8; ++g) {
        const int sn = reflect_jk(g, js, ks, p, nphi);  // g is an involution: z_{g(sn)} = z_{sp}
        TB* zz = zg + g * zs + 3 * sn;
        zz[0] = (g & 1) ? -z0 : z0;
        zz[1] = (g & 2) ? -z1 : z1;
        zz[2] = (g & 4) ? -z2 : z2;
      }
    }
    if (has_L) {
      const double4 q = x[o + sp];
      const TB rx = cv(q.x - cxd), ry = cv(q.y - cyd), rz = cv(q.z - czd), w = cv(q.w);
      m[0] += w * a;
      m[1] += w * b;
      m[2] += w * cc;
      m[3] += w * (ry * cc - rz * b);
      m[4] += w * (rz * a - rx * cc);
      m[5] += w * (rx * b - ry * a);
    }
  }
  if (has_block) {  // the padding columns [3 N_p, zs) of each z_g (their block entries are zero)
    const int pad = zs - dim;
    for (int e = threadIdx.x; e < 8 * pad; e += blockDim.x) {
      const int g = e / pad;
      zg[g * zs + dim + (e - g * pad)] = (TB)0;
    }
  }
  if (has_L) {
#pragma unroll
    for (int q = 0; q < 6; ++q) m[q] = warp_sum_t(m[q]);
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < 6; ++q) red[warp][q] = m[q];
  }
  __syncthreads();
  if (has_L && threadIdx.x < 6) {
    TB acc = 0;
    for (int w = 0; w < kSymWarps; ++w) acc += red[w][threadIdx.x];
    mom[threadIdx.x] = acc;
  }
  __syncthreads();
  // finish one node t of the particle from its body-frame block product (l0, l1, l2)
  auto finish = [&](int t, TB l0b, TB l1b, TB l2b) {
    const long long gi = o + t;
    TB l0 = R0 * l0b + R1 * l1b + R2 * l2b;
    TB l1 = R3 * l0b + R4 * l1b + R5 * l2b;
    TB l2 = R6 * l0b + R7 * l1b + R8 * l2b;
    const double* xt = in + 3 * gi;
    if (mode == kModeSelfK || mode == kModeSelfKNoL) {
      l0 += (TB)0.5 * cv(xt[0]);
      l1 += (TB)0.5 * cv(xt[1]);
      l2 += (TB)0.5 * cv(xt[2]);
    }
    if (has_L) {
      const double4 q = x[gi];
      const TB rx = cv(q.x - cxd), ry = cv(q.y - cyd), rz = cv(q.z - czd);
      l0 += mom[0] + (mom[4] * rz - mom[5] * ry);
      l1 += mom[1] + (mom[5] * rx - mom[3] * rz);
      l2 += mom[2] + (mom[3] * ry - mom[4] * rx);
    }
    if (mode == kModePrecond) {
      aux[3 * gi + 0] = xt[0];
      aux[3 * gi + 1] = xt[1];
      aux[3 * gi + 2] = xt[2];
    }
    out[3 * gi + 0] = wide(sc * l0);
    out[3 * gi + 1] = wide(sc * l1);
    out[3 * gi + 2] = wide(sc * l2);
  };
  if (!has_block) {
    for (int t = threadIdx.x; t < np; t += blockDim.x) finish(t, (TB)0, (TB)0, (TB)0);
    return;
  }

  const int kc = lane & 15, hg = lane >> 4;
  const TS* ring_k = reinterpret_cast<const TS*>(zraw) + warp * (S * 3 * SC) + 4 * kc;
  const TB* zl = zg + (4 * hg) * zs + 4 * kc;
  int slot = 0;
  for (int r = warp; r < nrep; r += kSymWarps) {
    float2 y2[4][3];
    TB yd[4][3];
#pragma unroll
    for (int gl = 0; gl < 4; ++gl)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        y2[gl][q] = make_float2(0.f, 0.f);
        yd[gl][q] = (TB)0;
      }
    for (int c0 = 0; c0 < SC * nst; c0 += SC) {
      issue();
      cp_async_wait<S - 1>();  // this lane's copies of the step have landed ...
      __syncwarp();            // ... and so have the other lanes'
      const TS* st = ring_k + slot * (3 * SC);
#pragma unroll
      for (int sq = 0; sq < SC / 64; ++sq) {
        if (c0 + 64 * sq + 4 * kc >= dim) continue;
        TB a[3][4];
#pragma unroll
        for (int q = 0; q < 3; ++q) load_quad(st + q * SC + 64 * sq, a[q]);
#pragma unroll
        for (int gl = 0; gl < 4; ++gl) {
          TB z[4];
          load_quad(zl + gl * zs + c0 + 64 * sq, z);
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            if constexpr (kF32) {
              y2[gl][q] = __ffma2_rn(make_float2(a[q][0], a[q][1]), make_float2(z[0], z[1]), y2[gl][q]);
              y2[gl][q] = __ffma2_rn(make_float2(a[q][2], a[q][3]), make_float2(z[2], z[3]), y2[gl][q]);
            } else {
              yd[gl][q] = fma(a[q][0], z[0], fma(a[q][1], z[1], fma(a[q][2], z[2], fma(a[q][3], z[3], yd[gl][q]))));
            }
          }
        }
      }
      __syncwarp();  // every lane has read the stage before it is refilled
      slot = (slot + 1 == S) ? 0 : slot + 1;
    }
    // reduce-scatter over the sixteen column groups: halve the set at lane bits 3 and 2, then sum
    TB v12[12], v6[6], v3[3];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      if constexpr (kF32)
        v12[k] = y2[k / 3][k % 3].x + y2[k / 3][k % 3].y;
      else
        v12[k] = yd[k / 3][k % 3];
    }
    {
      const bool hi = lane & 8;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const TB lo_v = v12[k], hi_v = v12[6 + k];
        v6[k] = (hi ? hi_v : lo_v) + __shfl_xor_sync(0xffffffffu, hi ? lo_v : hi_v, 8);
      }
    }
    {
      const bool hi = lane & 4;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const TB lo_v = v6[k], hi_v = v6[3 + k];
        v3[k] = (hi ? hi_v : lo_v) + __shfl_xor_sync(0xffffffffu, hi ? lo_v : hi_v, 4);
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      v3[k] += __shfl_xor_sync(0xffffffffu, v3[k], 2);
      v3[k] += __shfl_xor_sync(0xffffffffu, v3[k], 1);
    }
    // lane 4g holds reflection g's sums: node g(r) unless a smaller reflection reaches it
    const int g = lane >> 2;
    const int j0 = r / nk, k0 = r - j0 * nk;
    const int t = reflect_jk(g, j0, k0, p, nphi);
    bool first = true;
#pragma unroll
    for (int h = 0; h < 7; ++h) {
      const int th = __shfl_sync(0xffffffffu, t, 4 * h);
      if (h < g && th == t) first = false;
    }
    if ((lane & 3) == 0 && first) {
      const TB b0 = (g & 1) ? -v3[0] : v3[0], b1 = (g & 2) ? -v3[1] : v3[1], b2 = (g & 4) ? -v3[2] : v3[2];
      if constexpr (kF32) {
        ynode[3 * t] = b0;
        ynode[3 * t + 1] = b1;
        ynode[3 * t + 2] = b2;
      } else {
        finish(t, b0, b1, b2);
      }
    }
  }
  cp_async_wait<0>();
  if constexpr (kF32) {
    __syncthreads();
    for (int t = threadIdx.x; t < np; t += blockDim.x) finish(t, ynode[3 * t], ynode[3 * t + 1], ynode[3 * t + 2]);
  }
}

// ------------------------------------------------------------------------------------------
// Smooth pair sums in float64.  One block per work item (128 targets x a source range); each
// thread owns one target; sources are staged 128 at a time in shared memory with their weighted
// density w_s mu_s.  Pairs on the same particle are excluded (their contribution is the singular
// rule's); the select also removes the r = 0 self pair before it is used.
template <int KIND>
__global__ void __launch_bounds__(128) k_pairs64(int nitems, const longlong4* __restrict__ work, const double4* __restrict__ x,
                                                 const double4* __restrict__ nrm, const int* __restrict__ pid,
                                                 const double* __restrict__ dens, double* __restrict__ y) {
  constexpr int TS = 128;
  __shared__ double4 sp[TS];
  __shared__ double4 sd[TS];
  __shared__ int spid[TS];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
  const longlong4 w = work[it];
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
}

// ------------------------------------------------------------------------------------------
// Smooth pair sums in float32.  Coordinates are taken relative to the first target of the block in
// float64 before rounding, so a float32 difference keeps the relative accuracy of the separation
// rather than of the absolute position.  Each 256-source tile is summed in float32 and added into
// a compensated (two-sum) float32 accumulator.  Tiles whose particles cannot meet the block's
// targets skip the same-particle test.

template <int KIND, bool MASK, int NT>
__device__ __forceinline__ void pair_tile32(const float4* __restrict__ sp, const float4* __restrict__ sd, int cnt,
                                            const float (&xt)[NT][3], const float (&nt)[NT][3], const int (&pt)[NT],
                                            float (&acc)[NT][3]) {
#pragma unroll 4
  for (int l = 0; l < cnt; ++l) {
    const float4 ps = sp[l];
    const float4 ds = sd[l];
#pragma unroll
    for (int u = 0; u < NT; ++u) {
      const float dx = xt[u][0] - ps.x, dy = xt[u][1] - ps.y, dz = xt[u][2] - ps.z;
      const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      float inv = rsqrt_hw(r2);
      if (MASK && __float_as_int(ps.w) == pt[u]) inv = 0.0f;
      const float rr = fmaf(dx, ds.x, fmaf(dy, ds.y, dz * ds.z));
      if (KIND == 0) {
        const float inv2 = inv * inv;
        const float rn = fmaf(dx, nt[u][0], fmaf(dy, nt[u][1], dz * nt[u][2]));
        const float c = (rn * rr) * (inv2 * inv2 * inv);
        acc[u][0] = fmaf(c, dx, acc[u][0]);
        acc[u][1] = fmaf(c, dy, acc[u][1]);
        acc[u][2] = fmaf(c, dz, acc[u][2]);
      } else {
        const float c = rr * (inv * inv * inv);
        acc[u][0] = fmaf(c, dx, fmaf(ds.x, inv, acc[u][0]));
        acc[u][1] = fmaf(c, dy, fmaf(ds.y, inv, acc[u][1]));
        acc[u][2] = fmaf(c, dz, fmaf(ds.z, inv, acc[u][2]));
      }
    }
  }
}

// NT targets per thread (block = 128 / NT threads over a 128-target work item): each staged source
// feeds NT independent pair evaluations.
template <int KIND, int NT>
__global__ void __launch_bounds__(128 / NT, NT == 1 ? 1 : (NT == 2 ? 16 : 12)) k_pairs32(int nitems, const longlong4* __restrict__ work, const double4* __restrict__ x,
                                                      const double4* __restrict__ nrm, const int* __restrict__ pid,
                                                      const double* __restrict__ dens, double* __restrict__ y) {
  constexpr int TS = 256, NTH = 128 / NT;
  __shared__ float4 sp[TS];
  __shared__ float4 sd[TS];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
  const longlong4 w = work[it];
  const double4 org = x[w.x];
  float xt[NT][3], nt[NT][3];
  int pt[NT];
  bool valid[NT];
#pragma unroll
  for (int u = 0; u < NT; ++u) {
    const long long t = w.x + threadIdx.x + NTH * u;
    valid[u] = t < w.y;
    xt[u][0] = xt[u][1] = xt[u][2] = nt[u][0] = nt[u][1] = nt[u][2] = 0.0f;
    pt[u] = -1;
    if (valid[u]) {
      const double4 a = x[t], nn = nrm[t];
      xt[u][0] = (float)(a.x - org.x);
      xt[u][1] = (float)(a.y - org.y);
      xt[u][2] = (float)(a.z - org.z);
      nt[u][0] = (float)nn.x;
      nt[u][1] = (float)nn.y;
      nt[u][2] = (float)nn.z;
      pt[u] = pid[t];
    }
  }
  const int pid_lo = pid[w.x], pid_hi = pid[w.y - 1];
  float sa[NT][3], ea[NT][3];
#pragma unroll
  for (int u = 0; u < NT; ++u) sa[u][0] = sa[u][1] = sa[u][2] = ea[u][0] = ea[u][1] = ea[u][2] = 0.0f;
  for (long long s0 = w.z; s0 < w.w; s0 += TS) {
    const int cnt = (int)min((long long)TS, w.w - s0);
    __syncthreads();
    for (int l = threadIdx.x; l < cnt; l += NTH) {
      const long long s = s0 + l;
      const double4 ps = x[s];
      const double* d = dens + 3 * s;
      sp[l] = make_float4((float)(ps.x - org.x), (float)(ps.y - org.y), (float)(ps.z - org.z), __int_as_float(pid[s]));
      sd[l] = make_float4((float)(ps.w * d[0]), (float)(ps.w * d[1]), (float)(ps.w * d[2]), 0.0f);
    }
    __syncthreads();
    const int tlo = pid[s0], thi = pid[s0 + cnt - 1];
    float p[NT][3];
#pragma unroll
    for (int u = 0; u < NT; ++u) p[u][0] = p[u][1] = p[u][2] = 0.0f;
    if (thi < pid_lo || tlo > pid_hi)
      pair_tile32<KIND, false, NT>(sp, sd, cnt, xt, nt, pt, p);
    else
      pair_tile32<KIND, true, NT>(sp, sd, cnt, xt, nt, pt, p);
#pragma unroll
    for (int u = 0; u < NT; ++u)
#pragma unroll
      for (int c = 0; c < 3; ++c) two_sum_acc(sa[u][c], ea[u][c], p[u][c]);
  }
  const double sc = KIND == 0 ? kTractionScale : kStokesletScale;
#pragma unroll
  for (int u = 0; u < NT; ++u) {
    if (!valid[u]) continue;
    const long long t = w.x + threadIdx.x + NTH * u;
#pragma unroll
    for (int c = 0; c < 3; ++c) atomicAdd(y + 3 * t + c, sc * ((double)sa[u][c] + (double)ea[u][c]));
  }
  }
}

// ------------------------------------------------------------------------------------------
// Weighted density in float32 for the packed kernels: wmu[t] = (w_t mu_t, 0).
__global__ void k_weight_f32(long long N, const double4* __restrict__ x, const double* __restrict__ dens,
                             float4* __restrict__ wmu) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= N) return;
  const double w = x[t].w;
  wmu[t] = make_float4((float)(w * dens[3 * t]), (float)(w * dens[3 * t + 1]), (float)(w * dens[3 * t + 2]), 0.0f);
}

// Sources and targets are read as float32 hi + lo position pairs and float32 weighted densities, so
// the kernel runs no float64 arithmetic but its final accumulation: a coordinate relative to the work
// item's origin o is (y_hi - o_hi) + (y_lo - o_lo), within one rounding of the exact difference.
template <int KIND, int NT>
__global__ void __launch_bounds__(128 / NT, NT == 4 ? 12 : (NT == 2 ? 10 : 8)) k_pairs32x2(int nitems, const longlong4* __restrict__ work, const float4* __restrict__ xhi,
                                                       const float4* __restrict__ xlo, const float4* __restrict__ nrm32,
                                                       const float4* __restrict__ wmu, double* __restrict__ y) {
  constexpr int TS = 512, NTH = 128 / NT;  // 512 sources per tile: the staging latency is amortised over more pairs
  __shared__ __align__(16) float ssx[TS], ssy[TS], ssz[TS], srx[TS], sry[TS], srz[TS];
  __shared__ __align__(16) int spid[TS];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
  const longlong4 w = work[it];
  const float4 oh = xhi[w.x], ol = xlo[w.x];
  float2 xt[NT][3], nt[NT][3];
  int pt[NT];
  bool valid[NT];
#pragma unroll
  for (int u = 0; u < NT; ++u) {
    const long long t = w.x + threadIdx.x + NTH * u;
    valid[u] = t < w.y;
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
  const int pid_lo = __float_as_int(oh.w), pid_hi = __float_as_int(xhi[w.y - 1].w);
  float sa[NT][3], ea[NT][3];
#pragma unroll
  for (int u = 0; u < NT; ++u) sa[u][0] = sa[u][1] = sa[u][2] = ea[u][0] = ea[u][1] = ea[u][2] = 0.0f;
  for (long long s0 = w.z; s0 < w.w; s0 += TS) {
    const int cnt = (int)min((long long)TS, w.w - s0);
    const int cnt4 = (cnt + 3) & ~3;
    __syncthreads();
    for (int l = threadIdx.x; l < cnt4; l += NTH) {
      if (l < cnt) {
        const long long s = s0 + l;
        const float4 ph = xhi[s], pl = xlo[s], q = wmu[s];
        ssx[l] = (oh.x - ph.x) + (ol.x - pl.x);
        ssy[l] = (oh.y - ph.y) + (ol.y - pl.y);
        ssz[l] = (oh.z - ph.z) + (ol.z - pl.z);
        srx[l] = q.x;
        sry[l] = q.y;
        srz[l] = q.z;
        spid[l] = __float_as_int(ph.w);
      } else {
        ssx[l] = ssy[l] = ssz[l] = 1.0e4f;
        srx[l] = sry[l] = srz[l] = 0.0f;
        spid[l] = -2;
      }
    }
    __syncthreads();
    const int tlo = spid[0], thi = spid[cnt - 1];
    float2 p[NT][3];
#pragma unroll
    for (int u = 0; u < NT; ++u) p[u][0] = p[u][1] = p[u][2] = f2(0.0f, 0.0f);
    if (thi < pid_lo || tlo > pid_hi)
      pair_tile32x2<KIND, false, NT>(ssx, ssy, ssz, srx, sry, srz, spid, cnt4, xt, nt, pt, p);
    else
      pair_tile32x2<KIND, true, NT>(ssx, ssy, ssz, srx, sry, srz, spid, cnt4, xt, nt, pt, p);
#pragma unroll
    for (int u = 0; u < NT; ++u)
#pragma unroll
      for (int c = 0; c < 3; ++c) two_sum_acc(sa[u][c], ea[u][c], p[u][c].x + p[u][c].y);
  }
  const double sc = KIND == 0 ? kTractionScale : kStokesletScale;
#pragma unroll
  for (int u = 0; u < NT; ++u) {
    if (!valid[u]) continue;
    const long long t = w.x + threadIdx.x + NTH * u;
#pragma unroll
    for (int c = 0; c < 3; ++c) atomicAdd(y + 3 * t + c, sc * ((double)sa[u][c] + (double)ea[u][c]));
  }
  }
}

// ------------------------------------------------------------------------------------------
// Smooth pair sums in double-float arithmetic (dfloat.cuh): about 44 bits per float32-pipe operation;
// each tile of sources is summed in double-float and the tile sums accumulate in double-float.

// KIND 0: traction into acc; 1: Stokeslet into acc; 2: both for the same density, traction into acc
// and Stokeslet into acc2, sharing the separation, its inverse powers and r . w rho.
template <int KIND, bool MASK, int NT>
__device__ __forceinline__ void pair_tile_df(const float4* __restrict__ sph, const float4* __restrict__ spl,
                                             const float4* __restrict__ sdh, const float4* __restrict__ sdl, int cnt,
                                             const dflt (&xt)[NT][3], const dflt (&nt)[NT][3], const int (&pt)[NT],
                                             dflt (&acc)[NT][3], dflt (&acc2)[NT][3]) {
  for (int l = 0; l < cnt; ++l) {
    const float4 yh = sph[l], yl = spl[l], dh = sdh[l], dl = sdl[l];
    const dflt den[3] = {{dh.x, dl.x}, {dh.y, dl.y}, {dh.z, dl.z}};
#pragma unroll
    for (int u = 0; u < NT; ++u) {
      dflt d[3];
      d[0] = df_two_sum(xt[u][0].h, -yh.x);
      d[0].l += xt[u][0].l - yl.x;
      d[1] = df_two_sum(xt[u][1].h, -yh.y);
      d[1].l += xt[u][1].l - yl.y;
      d[2] = df_two_sum(xt[u][2].h, -yh.z);
      d[2].l += xt[u][2].l - yl.z;
      // r^2 = sum of d_c^2
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
      // 1 / sqrt(r^2): hardware estimate y0, one Newton step
      const float y0 = rsqrt_hw(r2h);
      const float q = y0 * y0;
      const float qe = fmaf(y0, y0, -q);
      float t = fmaf(r2h, q, -1.0f);
      t = fmaf(r2h, qe, t);
      t = fmaf(r2l, q, t);
      dflt inv = {y0, -0.5f * t * y0};
      if (MASK && __float_as_int(yh.w) == pt[u]) inv = {0.0f, 0.0f};
      const dflt rr = df_dot3(d[0], den[0], d[1], den[1], d[2], den[2]);
      const dflt inv2 = df_mul(inv, inv);
      const dflt inv3 = df_mul(inv2, inv);
      if (KIND == 0) {
        const dflt inv5 = df_mul(inv3, inv2);
        const dflt rn = df_dot3(d[0], nt[u][0], d[1], nt[u][1], d[2], nt[u][2]);
        const dflt cc = df_mul(df_mul(rn, rr), inv5);
#pragma unroll
        for (int c = 0; c < 3; ++c) df_acc(acc[u][c], df_mul(cc, d[c]));
      } else if (KIND == 2) {
        const dflt inv5 = df_mul(inv3, inv2);
        const dflt rn = df_dot3(d[0], nt[u][0], d[1], nt[u][1], d[2], nt[u][2]);
        const dflt ck = df_mul(df_mul(rn, rr), inv5);
        const dflt cs = df_mul(rr, inv3);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          df_acc(acc[u][c], df_mul(ck, d[c]));
          df_acc(acc2[u][c], df_mul(den[c], inv));
          df_acc(acc2[u][c], df_mul(cs, d[c]));
        }
      } else {
        const dflt cc = df_mul(rr, inv3);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          df_acc(acc[u][c], df_mul(den[c], inv));
          df_acc(acc[u][c], df_mul(cc, d[c]));
        }
      }
    }
  }
}

// Weighted density as double-float pairs for the double-float kernels: (w mu) rounded to float32 and
// the rounded remainder.
__global__ void k_weight_df(long long N, const double4* __restrict__ x, const double* __restrict__ dens,
                            float4* __restrict__ wh, float4* __restrict__ wl) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= N) return;
  const double w = x[t].w;
  const dflt a = df_split(w * dens[3 * t]), b = df_split(w * dens[3 * t + 1]), c = df_split(w * dens[3 * t + 2]);
  wh[t] = make_float4(a.h, b.h, c.h, 0.0f);
  wl[t] = make_float4(a.l, b.l, c.l, 0.0f);
}


// y += traction sum (KIND 0, 2) or Stokeslet sum (KIND 1); KIND 2 also y2 += Stokeslet sum.  No float64
// arithmetic runs per pair or per staged source: positions come as exact three-float splits, the
// weighted density and normals as double-float pairs, and tile sums are accumulated in double-float;
// the total is converted to float64 once per target.
template <int KIND, int NT>
__global__ void __launch_bounds__(128 / NT, 8) k_pairs_df(int nitems, const longlong4* __restrict__ work,
                                                       const float4* __restrict__ x3h, const float4* __restrict__ x3m,
                                                       const float4* __restrict__ x3l, const float4* __restrict__ nh,
                                                       const float4* __restrict__ nl, const float4* __restrict__ wh,
                                                       const float4* __restrict__ wl, double* __restrict__ y,
                                                       double* __restrict__ y2) {
  constexpr int TS = 128, NTH = 128 / NT;
  __shared__ float4 sph[TS], spl[TS], sdh[TS], sdl[TS];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
  const longlong4 w = work[it];
  const float4 oh = x3h[w.x], om = x3m[w.x], ol = x3l[w.x];
  dflt xt[NT][3], nt[NT][3];
  int pt[NT];
  bool valid[NT];
#pragma unroll
  for (int u = 0; u < NT; ++u) {
    const long long t = w.x + threadIdx.x + NTH * u;
    valid[u] = t < w.y;
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
    xt[u][0] = df_diff3(ah.x, am.x, al.x, oh.x, om.x, ol.x);
    xt[u][1] = df_diff3(ah.y, am.y, al.y, oh.y, om.y, ol.y);
    xt[u][2] = df_diff3(ah.z, am.z, al.z, oh.z, om.z, ol.z);
    nt[u][0] = {bh.x, bl.x};
    nt[u][1] = {bh.y, bl.y};
    nt[u][2] = {bh.z, bl.z};
  }
  const int pid_lo = __float_as_int(oh.w), pid_hi = __float_as_int(x3h[w.y - 1].w);
  dflt a[NT][3], a2[NT][3];
#pragma unroll
  for (int u = 0; u < NT; ++u)
#pragma unroll
    for (int c = 0; c < 3; ++c) a[u][c] = a2[u][c] = dflt{0.0f, 0.0f};
  for (long long s0 = w.z; s0 < w.w; s0 += TS) {
    const int cnt = (int)min((long long)TS, w.w - s0);
    __syncthreads();
    for (int l = threadIdx.x; l < cnt; l += NTH) {
      const long long s = s0 + l;
      const float4 ph = x3h[s], pm = x3m[s], pl = x3l[s];
      const dflt px = df_diff3(ph.x, pm.x, pl.x, oh.x, om.x, ol.x);
      const dflt py = df_diff3(ph.y, pm.y, pl.y, oh.y, om.y, ol.y);
      const dflt pz = df_diff3(ph.z, pm.z, pl.z, oh.z, om.z, ol.z);
      sph[l] = make_float4(px.h, py.h, pz.h, ph.w);
      spl[l] = make_float4(px.l, py.l, pz.l, 0.0f);
      sdh[l] = wh[s];
      sdl[l] = wl[s];
    }
    __syncthreads();
    const int tlo = __float_as_int(sph[0].w), thi = __float_as_int(sph[cnt - 1].w);
    dflt acc[NT][3], acc2[NT][3];
#pragma unroll
    for (int u = 0; u < NT; ++u)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[u][c] = acc2[u][c] = dflt{0.0f, 0.0f};
    if (thi < pid_lo || tlo > pid_hi)
      pair_tile_df<KIND, false, NT>(sph, spl, sdh, sdl, cnt, xt, nt, pt, acc, acc2);
    else
      pair_tile_df<KIND, true, NT>(sph, spl, sdh, sdl, cnt, xt, nt, pt, acc, acc2);
#pragma unroll
    for (int u = 0; u < NT; ++u)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        a[u][c] = df_add_accurate(a[u][c], acc[u][c]);
        if (KIND == 2) a2[u][c] = df_add_accurate(a2[u][c], acc2[u][c]);
      }
  }
  const double sc = KIND == 1 ? kStokesletScale : kTractionScale;
#pragma unroll
  for (int u = 0; u < NT; ++u) {
    if (!valid[u]) continue;
    const long long t = w.x + threadIdx.x + NTH * u;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      atomicAdd(y + 3 * t + c, sc * ((double)a[u][c].h + (double)a[u][c].l));
      if (KIND == 2) atomicAdd(y2 + 3 * t + c, kStokesletScale * ((double)a2[u][c].h + (double)a2[u][c].l));
    }
  }
  }
}

// ------------------------------------------------------------------------------------------
template <int KIND, int NT>
__global__ void __launch_bounds__(128 / NT, NT == 1 ? 5 : 6) k_pairs_df2(int nitems, const longlong4* __restrict__ work,
                                                        const float4* __restrict__ x3h, const float4* __restrict__ x3m,
                                                        const float4* __restrict__ x3l, const float4* __restrict__ nh,
                                                        const float4* __restrict__ nl, const float4* __restrict__ wh,
                                                        const float4* __restrict__ wl, double* __restrict__ y,
                                                        double* __restrict__ y2) {
  constexpr int TS = 128, NTH = 128 / NT;
  // structure of arrays: separation parts x, y, z (hi, lo), weighted density (hi, lo), particle id
  __shared__ __align__(16) float sa[12][TS];
  __shared__ __align__(16) int spid[TS];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
  const longlong4 w = work[it];
  const float4 oh = x3h[w.x], om = x3m[w.x], ol = x3l[w.x];
  df2 xt[NT][3], nt[NT][3];
  int pt[NT];
  bool valid[NT];
#pragma unroll
  for (int u = 0; u < NT; ++u) {
    const long long t = w.x + threadIdx.x + NTH * u;
    valid[u] = t < w.y;
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
  const int pid_lo = __float_as_int(oh.w), pid_hi = __float_as_int(x3h[w.y - 1].w);
  dflt a[NT][3], a2[NT][3];
#pragma unroll
  for (int u = 0; u < NT; ++u)
#pragma unroll
    for (int c = 0; c < 3; ++c) a[u][c] = a2[u][c] = dflt{0.0f, 0.0f};
  for (long long s0 = w.z; s0 < w.w; s0 += TS) {
    const int cnt = (int)min((long long)TS, w.w - s0);
    const int cnt2 = (cnt + 1) & ~1;
    __syncthreads();
    for (int l = threadIdx.x; l < cnt2; l += NTH) {
      if (l < cnt) {
        const long long s = s0 + l;
        const float4 ph = x3h[s], pm = x3m[s], pl = x3l[s], qh = wh[s], ql = wl[s];
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
      } else {
        sa[0][l] = sa[2][l] = sa[4][l] = 1.0e4f;
        sa[1][l] = sa[3][l] = sa[5][l] = 0.0f;
        for (int q = 6; q < 12; ++q) sa[q][l] = 0.0f;
        spid[l] = -2;
      }
    }
    __syncthreads();
    const int tlo = spid[0], thi = spid[cnt - 1];
    const bool masked = !(thi < pid_lo || tlo > pid_hi);
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
        if (masked)
          pair2_df<KIND, true>(ys, den, pp, xt[u], nt[u], pt[u], acc[u], acc2[u]);
        else
          pair2_df<KIND, false>(ys, den, pp, xt[u], nt[u], pt[u], acc[u], acc2[u]);
      }
    }
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
    const long long t = w.x + threadIdx.x + NTH * u;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      atomicAdd(y + 3 * t + c, sc * ((double)a[u][c].h + (double)a[u][c].l));
      if (KIND == 2) atomicAdd(y2 + 3 * t + c, kStokesletScale * ((double)a2[u][c].h + (double)a2[u][c].l));
    }
  }
  }
}

// ------------------------------------------------------------------------------------------
// Upsampled densities of the near-source particles: mu_up = U mu_j with U stored transposed
// (N_p x N_up), one thread per upsampled node reading U coalesced and mu_j from shared memory; the
// arithmetic is that of U's storage type (float32 for the inner solve, float64 otherwise).
template <typename TU>
__global__ void __launch_bounds__(128) k_upsample(int n_up, const int* __restrict__ up_particle,
                                                  const long long* __restrict__ up_off,
                                                  const long long* __restrict__ offset, const int* __restrict__ nodes,
                                                  const TU* const* __restrict__ Umats, const double* __restrict__ dens,
                                                  double* __restrict__ upmu) {
  extern __shared__ double mus_raw[];  // 3 N_p values of type TU
  TU* mus = reinterpret_cast<TU*>(mus_raw);
  for (int u = blockIdx.y; u < n_up; u += gridDim.y) {
    const int j = up_particle[u];
    const int np = nodes[j];
    const long long o = offset[j];
    __syncthreads();
    for (int l = threadIdx.x; l < 3 * np; l += blockDim.x) mus[l] = (TU)dens[3 * o + l];
    __syncthreads();
    const long long base = up_off[u];
    const int nup = (int)(up_off[u + 1] - base);
    const TU* Ut = Umats[u];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nup; r += gridDim.x * blockDim.x) {
      TU a0 = 0, a1 = 0, a2 = 0;
      for (int s = 0; s < np; ++s) {
        const TU uv = Ut[(long long)s * nup + r];
        a0 = fma_t(uv, mus[3 * s], a0);
        a1 = fma_t(uv, mus[3 * s + 1], a1);
        a2 = fma_t(uv, mus[3 * s + 2], a2);
      }
      upmu[3 * (base + r) + 0] = (double)a0;
      upmu[3 * (base + r) + 1] = (double)a1;
      upmu[3 * (base + r) + 2] = (double)a2;
    }
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

// Near correction in float32 or double-float, sharing the tile loops of the smooth sums.  One
// block per near pair; the block size covers the largest target particle in one or two passes;
// sources (upsampled nodes of j with +w, base nodes of j with -w) are staged relative to the target
// particle's centre.  Tile partials are added in float64.
template <int KIND, bool DF>
__global__ void __launch_bounds__(512) k_near_tiled(const int2* __restrict__ near, const long long* __restrict__ offset,
                                                    const int* __restrict__ nodes, const double* __restrict__ centre,
                                                    const int* __restrict__ up_index, const long long* __restrict__ up_off,
                                                    const double4* __restrict__ x, const double4* __restrict__ nrm,
                                                    const double* __restrict__ dens, const double4* __restrict__ upx,
                                                    const double* __restrict__ upmu, double* __restrict__ y) {
  constexpr int TS = 256;
  __shared__ float4 s0[TS], s1[TS], s2[DF ? TS : 1], s3[DF ? TS : 1];
  const int2 pr = near[blockIdx.x];
  const int i = pr.x, j = pr.y;
  const double ox = centre[3 * i], oy = centre[3 * i + 1], oz = centre[3 * i + 2];
  const long long oi = offset[i], oj = offset[j];
  const int npi = nodes[i], npj = nodes[j];
  const int u = up_index[j];
  const long long ub = up_off[u];
  const int nup = (int)(up_off[u + 1] - ub);
  const int total = nup + npj;
  for (int tb = 0; tb < npi; tb += blockDim.x) {
    const int tl = tb + threadIdx.x;
    const bool valid = tl < npi;
    double4 xt = make_double4(0, 0, 0, 0), nt = make_double4(0, 0, 0, 0);
    if (valid) {
      xt = x[oi + tl];
      nt = nrm[oi + tl];
    }
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int sb = 0; sb < total; sb += TS) {
      const int cnt = min(TS, total - sb);
      __syncthreads();
      for (int l = threadIdx.x; l < cnt; l += blockDim.x) {
        const int s = sb + l;
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
        if (DF) {
          const dflt px = df_split(ps.x - ox), py = df_split(ps.y - oy), pz = df_split(ps.z - oz);
          const dflt q0 = df_split(wgt * d0), q1 = df_split(wgt * d1), q2 = df_split(wgt * d2);
          s0[l] = make_float4(px.h, py.h, pz.h, 0.0f);
          s1[l] = make_float4(px.l, py.l, pz.l, 0.0f);
          s2[l] = make_float4(q0.h, q1.h, q2.h, 0.0f);
          s3[l] = make_float4(q0.l, q1.l, q2.l, 0.0f);
        } else {
          s0[l] = make_float4((float)(ps.x - ox), (float)(ps.y - oy), (float)(ps.z - oz), 0.0f);
          s1[l] = make_float4((float)(wgt * d0), (float)(wgt * d1), (float)(wgt * d2), 0.0f);
        }
      }
      __syncthreads();
      if (DF) {
        const dflt xd[1][3] = {{df_split(xt.x - ox), df_split(xt.y - oy), df_split(xt.z - oz)}};
        const dflt nd[1][3] = {{df_split(nt.x), df_split(nt.y), df_split(nt.z)}};
        const int none[1] = {-1};
        dflt acc[1][3] = {{{0, 0}, {0, 0}, {0, 0}}};
        pair_tile_df<KIND, false, 1>(s0, s1, s2, s3, cnt, xd, nd, none, acc, acc);
        a0 += (double)acc[0][0].h + (double)acc[0][0].l;
        a1 += (double)acc[0][1].h + (double)acc[0][1].l;
        a2 += (double)acc[0][2].h + (double)acc[0][2].l;
      } else {
        const float xf[1][3] = {{(float)(xt.x - ox), (float)(xt.y - oy), (float)(xt.z - oz)}};
        const float nf[1][3] = {{(float)nt.x, (float)nt.y, (float)nt.z}};
        const int none[1] = {-1};
        float p[1][3] = {{0, 0, 0}};
        pair_tile32<KIND, false, 1>(s0, s1, cnt, xf, nf, none, p);
        a0 += p[0][0];
        a1 += p[0][1];
        a2 += p[0][2];
      }
    }
    if (valid) {
      const double sc = KIND == 0 ? kTractionScale : kStokesletScale;
      atomicAdd(y + 3 * (oi + tl) + 0, sc * a0);
      atomicAdd(y + 3 * (oi + tl) + 1, sc * a1);
      atomicAdd(y + 3 * (oi + tl) + 2, sc * a2);
    }
  }
}

}  // namespace

// Blocks of `kernel` that fit on the GPU at once (occupancy x SMs), capped at the item count: the
// pair kernels loop over their work items with this persistent grid, so the last wave is not a
// mostly idle second pass over the SMs.
static int resident_grid(Context& c, const void* kernel, int threads, int items) {
  auto it = c.resident.find(kernel);
  int per_sm = 0;
  if (it == c.resident.end()) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
      per_sm = 1;
    c.resident[kernel] = per_sm;
  } else {
    per_sm = it->second;
  }
  return std::max(1, std::min(items, per_sm * std::max(1, c.sm_count)));
}

// Launch of the smooth pair sum over the first `items` work items with NT targets per thread.
// KIND 2 (traction into y and Stokeslet into y2 in one pass) exists in double-float only.
template <int KIND>
static void launch_pairs_kind(Context& c, int prec, int nt, int items, const double* x, double* y, double* y2) {
#define RBS_PAIR_ARGS items, c.d_work.ptr, c.d_x.ptr, c.d_nrm.ptr, c.d_pid.ptr, x, y
  if (prec == RBS_PREC_DF) {
#define RBS_DF_ARGS items, c.d_work.ptr, c.d_x3h.ptr, c.d_x3m.ptr, c.d_x3l.ptr, c.d_nrmh.ptr, c.d_nrml.ptr, \
                    c.d_wmuh.ptr, c.d_wmul.ptr, y, y2
    k_weight_df<<<cdiv(c.N, 256), 256, 0, c.stream>>>(c.N, c.d_x.ptr, x, c.d_wmuh.ptr, c.d_wmul.ptr);
    if (nt == 1)
      k_pairs_df<KIND, 1><<<resident_grid(c, (const void*)k_pairs_df<KIND, 1>, 128, items), 128, 0, c.stream>>>(RBS_DF_ARGS);
    else if (nt == 2)
      k_pairs_df<KIND, 2><<<resident_grid(c, (const void*)k_pairs_df<KIND, 2>, 64, items), 64, 0, c.stream>>>(RBS_DF_ARGS);
    else if (nt == 4)
      k_pairs_df<KIND, 4><<<resident_grid(c, (const void*)k_pairs_df<KIND, 4>, 32, items), 32, 0, c.stream>>>(RBS_DF_ARGS);
    else if (nt == kPacked + 1)
      k_pairs_df2<KIND, 1><<<resident_grid(c, (const void*)k_pairs_df2<KIND, 1>, 128, items), 128, 0, c.stream>>>(RBS_DF_ARGS);
    else
      k_pairs_df2<KIND, 2><<<resident_grid(c, (const void*)k_pairs_df2<KIND, 2>, 64, items), 64, 0, c.stream>>>(RBS_DF_ARGS);
#undef RBS_DF_ARGS
  } else if constexpr (KIND == 2) {
    return;
  } else if (prec == RBS_PREC_FP64) {
    k_pairs64<KIND><<<resident_grid(c, (const void*)k_pairs64<KIND>, 128, items), 128, 0, c.stream>>>(RBS_PAIR_ARGS);
  } else {
    if (nt == 1)
      k_pairs32<KIND, 1><<<resident_grid(c, (const void*)k_pairs32<KIND, 1>, 128, items), 128, 0, c.stream>>>(RBS_PAIR_ARGS);
    else if (nt == 2)
      k_pairs32<KIND, 2><<<resident_grid(c, (const void*)k_pairs32<KIND, 2>, 64, items), 64, 0, c.stream>>>(RBS_PAIR_ARGS);
    else if (nt == 4)
      k_pairs32<KIND, 4><<<resident_grid(c, (const void*)k_pairs32<KIND, 4>, 32, items), 32, 0, c.stream>>>(RBS_PAIR_ARGS);
    else {
#define RBS_PACKED_ARGS items, c.d_work.ptr, c.d_xhi.ptr, c.d_xlo.ptr, c.d_nrm32.ptr, c.d_wmu32.ptr, y
      k_weight_f32<<<cdiv(c.N, 256), 256, 0, c.stream>>>(c.N, c.d_x.ptr, x, c.d_wmu32.ptr);
      if (nt == kPacked + 1)
        k_pairs32x2<KIND, 1><<<resident_grid(c, (const void*)k_pairs32x2<KIND, 1>, 128, items), 128, 0, c.stream>>>(RBS_PACKED_ARGS);
      else if (nt == kPacked + 2)
        k_pairs32x2<KIND, 2><<<resident_grid(c, (const void*)k_pairs32x2<KIND, 2>, 64, items), 64, 0, c.stream>>>(RBS_PACKED_ARGS);
      else
        k_pairs32x2<KIND, 4><<<resident_grid(c, (const void*)k_pairs32x2<KIND, 4>, 32, items), 32, 0, c.stream>>>(RBS_PACKED_ARGS);
#undef RBS_PACKED_ARGS
    }
  }
#undef RBS_PAIR_ARGS
}

static Status launch_pairs(Context& c, int kind, int prec, int nt, int items, const double* x, double* y,
                           double* y2 = nullptr) {
  if (kind == 0)
    launch_pairs_kind<0>(c, prec, nt, items, x, y, y2);
  else if (kind == 1)
    launch_pairs_kind<1>(c, prec, nt, items, x, y, y2);
  else
    launch_pairs_kind<2>(c, prec, nt, items, x, y, y2);
  RBS_CUDA_TRY(cudaGetLastError());
  return Status::Ok();
}

// Pair-kernel variant: targets per thread (1, 2 or 4), plus kPacked for the float32 kernels that take
// two sources per packed instruction.  rbs_options.pair_variant when set (its targets per thread for
// the double-float kernels), otherwise the fastest candidate timed once per (kernel, arithmetic) on a
// prefix of the work list (the same items for every variant, into a scratch output).
static int pair_variant(Context& c, int kind, int prec, const double* x) {
  if (c.opt.pair_variant > 0)
    return (prec == RBS_PREC_DF && c.opt.pair_variant == kPacked + 4) ? 4 : c.opt.pair_variant;
  const int key = kind == 2 ? 4 : 2 * (prec == RBS_PREC_DF ? 1 : 0) + kind;
  if (c.tuned[key]) return c.tuned[key];
  int best = 2;
  const int items = std::min<int>((int)c.work.size(), 2 * 32 * std::max(1, c.sm_count));
  double* scratch = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaMalloc(&scratch, sizeof(double) * 6 * c.N) == cudaSuccess && cudaEventCreate(&a) == cudaSuccess &&
      cudaEventCreate(&b) == cudaSuccess) {
    float best_ms = 1e30f;
    std::vector<int> cands = {1, 2, 4};
    if (prec_f32(prec)) cands.insert(cands.end(), {kPacked + 1, kPacked + 2, kPacked + 4});
    if (prec == RBS_PREC_DF) cands.insert(cands.end(), {kPacked + 1, kPacked + 2});
    for (int nt : cands) {
      launch_pairs(c, kind, prec, nt, items, x, scratch, scratch + 3 * c.N);  // warm (first launch of this variant)
      cudaEventRecord(a, c.stream);
      launch_pairs(c, kind, prec, nt, items, x, scratch, scratch + 3 * c.N);
      cudaEventRecord(b, c.stream);
      float ms = 0.0f;
      if (cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        best = nt;
      }
      c.stats.launches += 2;
    }
    c.tune_ms[key] = best_ms;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (scratch) cudaFree(scratch);
  cudaGetLastError();
  c.tuned[key] = best;
  return best;
}

// ------------------------------------------------------------------------------------------

Status apply_blocks(Context& c, int mode, int prec, const double* x, double* y, double* aux, double scale) {
  if (mode == kModeZero) {
    c.stats.launches += 1;
    RBS_CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(double) * 3 * c.N, c.stream));
    return Status::Ok();
  }
  const int nb = (int)c.bwork.size();
  const int ns = (int)c.sym_list.size();
  const bool kblock = mode == kModeSelfK || mode == kModeSelfKNoL || mode == kModeKOnlySelf || mode == kModePrecond;
  const bool use32 = prec_f32(prec) && kblock;
  // 16-bit entries for the ellipsoid blocks of the inner solve's arithmetic (coefficient surfaces,
  // which store every row, keep float32 blocks)
  const bool use16 = prec_16(prec) && kblock && c.d_blockK16.ptr;
  const double bytes = (mode == kModeL) ? 0.0 : (double)c.particle_block_entries * (use16 ? 2.0 : use32 ? 4.0 : 8.0);
  KernelTimer timer(c, use32 ? RBS_KC_BLOCKS : RBS_KC_BLOCKS_F64);
  // 16-bit modes: ellipsoids of shapes shared by many particles go through the tensor-core GEMM, the
  // others through the CUDA-core kernel below
  const bool gemm = use16 && !c.gemm.empty();
  const int* sym_ids = gemm ? c.d_sym_rest.ptr : c.d_sym_list.ptr;
  const int nsym = gemm ? (int)c.sym_rest.size() : ns;
  if (gemm) RBS_TRY(apply_self_gemm(c, mode, x, y, aux, scale));
  if (nsym > 0) {
    const size_t zs = (size_t)sym_smem_bytes(c.max_np_sym, use16 ? 2 : use32 ? 4 : 8, use32 ? 4 : 8);
#define RBS_SYM_ARGS                                                                                              \
  mode, sym_ids, c.d_offset.ptr, c.d_p.ptr, c.d_nphi.ptr, c.d_rot.ptr, c.d_centre.ptr, c.d_shape.ptr, \
      c.d_block_off.ptr, B, c.d_x.ptr, x, y, aux, scale
    if (use16) {
      const uint16_t* B16 = (mode == kModePrecond) ? c.d_precond16.ptr : c.d_blockK16.ptr;
      if (prec == RBS_PREC_MIXED_FP16) {
        const F16Bits* B = reinterpret_cast<const F16Bits*>(B16);
        if (zs > 48 * 1024)
          RBS_CUDA_TRY(cudaFuncSetAttribute(k_blocks_sym<F16Bits, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)zs));
        k_blocks_sym<F16Bits, float><<<nsym, kSymWarps * 32, zs, c.stream>>>(RBS_SYM_ARGS);
      } else {
        const BF16Bits* B = reinterpret_cast<const BF16Bits*>(B16);
        if (zs > 48 * 1024)
          RBS_CUDA_TRY(cudaFuncSetAttribute(k_blocks_sym<BF16Bits, float>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zs));
        k_blocks_sym<BF16Bits, float><<<nsym, kSymWarps * 32, zs, c.stream>>>(RBS_SYM_ARGS);
      }
    } else if (use32) {
      const float* B = (mode == kModePrecond) ? c.d_precond32.ptr : c.d_blockK32.ptr;
      if (zs > 48 * 1024)
        RBS_CUDA_TRY(cudaFuncSetAttribute(k_blocks_sym<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)zs));
      k_blocks_sym<float, float><<<nsym, kSymWarps * 32, zs, c.stream>>>(RBS_SYM_ARGS);
    } else {
      const double* B = (mode == kModePrecond) ? c.d_precond.ptr : (mode == kModeSelfS ? c.d_blockS.ptr : c.d_blockK.ptr);
      if (zs > 48 * 1024)
        RBS_CUDA_TRY(cudaFuncSetAttribute(k_blocks_sym<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)zs));
      k_blocks_sym<double, double><<<nsym, kSymWarps * 32, zs, c.stream>>>(RBS_SYM_ARGS);
    }
#undef RBS_SYM_ARGS
    RBS_CUDA_TRY(cudaGetLastError());
  }
  if (nb == 0) {
    timer.done(bytes);
    return Status::Ok();
  }
  const size_t smem = (use32 ? sizeof(float) : sizeof(double)) * 3 * (size_t)c.max_np;
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

// Near correction, step 1: upsampled densities of the near-source particles (float32 interpolation
// for the inner solve, float64 otherwise).
static Status near_upsample(Context& c, bool f32, const double* x) {
  size_t smem = sizeof(double) * 3 * (size_t)c.max_np;
  if (smem > 48 * 1024) {
    RBS_CUDA_TRY(cudaFuncSetAttribute(k_upsample<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RBS_CUDA_TRY(cudaFuncSetAttribute(k_upsample<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  int maxup = 0;
  for (Grid* g : c.grids) maxup = std::max(maxup, g->nup);
  const int nup_p = (int)c.up_particle.size();
  dim3 gu(cdiv(maxup, 128), (unsigned)std::min(nup_p, 65535));
  if (f32)
    k_upsample<float><<<gu, 128, smem, c.stream>>>(nup_p, c.d_up_particle.ptr, c.d_up_off.ptr, c.d_offset.ptr, c.d_nodes.ptr,
                                                   c.d_upU32.ptr, x, c.d_up_mu.ptr);
  else
    k_upsample<double><<<gu, 128, smem, c.stream>>>(nup_p, c.d_up_particle.ptr, c.d_up_off.ptr, c.d_offset.ptr,
                                                    c.d_nodes.ptr, c.d_upU.ptr, x, c.d_up_mu.ptr);
  RBS_CUDA_TRY(cudaGetLastError());
  return Status::Ok();
}

// Near correction, step 2: for every near pair, the base-grid term is replaced by the upsampled one.
static Status near_sums(Context& c, int kind, int prec, const double* x, double* y) {
  const int nn = (int)c.near_pairs.size();
#define RBS_NEAR_ARGS                                                                                            \
  c.d_near.ptr, c.d_offset.ptr, c.d_nodes.ptr, c.d_centre.ptr, c.d_up_index.ptr, c.d_up_off.ptr, c.d_x.ptr, \
      c.d_nrm.ptr, x, c.d_up_x.ptr, c.d_up_mu.ptr, y
  const int nthr = std::min(512, std::max(64, (c.max_np + 31) / 32 * 32));
  if (prec == RBS_PREC_DF) {
    if (kind == 0)
      k_near_tiled<0, true><<<nn, nthr, 0, c.stream>>>(RBS_NEAR_ARGS);
    else
      k_near_tiled<1, true><<<nn, nthr, 0, c.stream>>>(RBS_NEAR_ARGS);
  } else if (prec_f32(prec)) {
    if (kind == 0)
      k_near_tiled<0, false><<<nn, nthr, 0, c.stream>>>(RBS_NEAR_ARGS);
    else
      k_near_tiled<1, false><<<nn, nthr, 0, c.stream>>>(RBS_NEAR_ARGS);
  } else {
    if (kind == 0)
      k_near<0, double><<<nn, 256, 0, c.stream>>>(RBS_NEAR_ARGS);
    else
      k_near<1, double><<<nn, 256, 0, c.stream>>>(RBS_NEAR_ARGS);
  }
#undef RBS_NEAR_ARGS
  RBS_CUDA_TRY(cudaGetLastError());
  return Status::Ok();
}

Status apply_pairs(Context& c, int kind, int prec, const double* x, double* y) {
  const int nw = (int)c.work.size();
  const bool f32 = prec_f32(prec);
  if (f32 && c.tree.active) {
    RBS_TRY(apply_tree(c, kind, x, y, 0));  // treecode in place of the direct float32 sum
  } else if (prec == RBS_PREC_DF && c.tree_df.active) {
    RBS_TRY(apply_tree_df(c, kind, x, y, nullptr));  // and of the direct double-float sum
  } else if (nw > 0) {
    int cls = f32 ? (kind == 0 ? RBS_KC_PAIR_K32 : RBS_KC_PAIR_S32) : (kind == 0 ? RBS_KC_PAIR_K64 : RBS_KC_PAIR_S64);
    if (prec == RBS_PREC_DF) cls = kind == 0 ? RBS_KC_PAIR_KDF : RBS_KC_PAIR_SDF;
    const int nt = (prec == RBS_PREC_FP64) ? 1 : pair_variant(c, kind, prec, x);
    KernelTimer timer(c, cls);
    RBS_TRY(launch_pairs(c, kind, prec, nt, nw, x, y));
    RBS_CUDA_TRY(cudaGetLastError());
    timer.done((double)c.stats.far_pairs);
  }
  if (!c.near_pairs.empty()) {
    KernelTimer timer(c, RBS_KC_NEAR);
    RBS_TRY(near_upsample(c, f32, x));
    RBS_TRY(near_sums(c, kind, prec, x, y));
    timer.done((double)c.near_pair_nodes, 2);
  }
  return Status::Ok();
}

Status apply_pairs_both(Context& c, int prec, const double* x, double* yK, double* yS) {
  if (prec_f32(prec)) {
    RBS_TRY(apply_pairs(c, 0, prec, x, yK));
    return apply_pairs(c, 1, prec, x, yS);
  }
  const int nw = (int)c.work.size();
  if (prec == RBS_PREC_DF && c.tree_df.active) {
    RBS_TRY(apply_tree_df(c, 2, x, yK, yS));
  } else if (nw > 0) {
    if (prec == RBS_PREC_DF) {
      const int nt = pair_variant(c, 2, prec, x);
      KernelTimer timer(c, RBS_KC_PAIR_KSDF);
      RBS_TRY(launch_pairs(c, 2, prec, nt, nw, x, yK, yS));
      timer.done((double)c.stats.far_pairs);
    } else {
      {
        KernelTimer timer(c, RBS_KC_PAIR_K64);
        RBS_TRY(launch_pairs(c, 0, prec, 1, nw, x, yK));
        timer.done((double)c.stats.far_pairs);
      }
      KernelTimer timer(c, RBS_KC_PAIR_S64);
      RBS_TRY(launch_pairs(c, 1, prec, 1, nw, x, yS));
      timer.done((double)c.stats.far_pairs);
    }
  }
  if (!c.near_pairs.empty()) {
    KernelTimer timer(c, RBS_KC_NEAR);
    RBS_TRY(near_upsample(c, false, x));
    RBS_TRY(near_sums(c, 0, prec, x, yK));
    RBS_TRY(near_sums(c, 1, prec, x, yS));
    timer.done(2.0 * c.near_pair_nodes, 3);
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
