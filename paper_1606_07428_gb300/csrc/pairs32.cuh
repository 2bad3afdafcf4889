// Float32 smooth pair-sum arithmetic shared by the direct sums (operators.cu) and the treecode
// (treecode.cu): the kernels' constant factors, compensated tile accumulation and the packed tile
// loop that evaluates a target against two sources per instruction.
#pragma once

#include "common.cuh"
#include "dfloat.cuh"

namespace rbs {

// Constant factors of the traction kernel (Eqs. 13 and 22) and the Stokeslet (Eq. 10), applied once
// per target after the pair sums.
constexpr double kTractionScale = -3.0 / (4.0 * kPi);
constexpr double kStokesletScale = 1.0 / (8.0 * kPi);

// Adds v into the compensated float32 sum (s, e) (Knuth's two-sum).
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float v) {
  float t = s + v;
  float bp = t - s;
  e += (s - (t - bp)) + (v - bp);
  s = t;
}

// Smooth pair sums in float32 with two sources per instruction: Blackwell's packed float32
// instructions (__fadd2_rn, __fmul2_rn, __ffma2_rn: two round-to-nearest operations per lane, one
// issue slot) evaluate a target against two sources at once, so the kernel is bound by the float32
// pipe rather than by instruction issue.  Sources are staged structure-of-arrays in shared memory,
// four per 128-bit load, coordinates negated (x_t + (-y_s) is the separation) and relative to the
// work item's first target; the tile is padded to a multiple of four with zero-density sources far
// away (they add exactly zero).  The reciprocal square root stays one hardware instruction per pair.
// Each target thread keeps float2 partial sums over the two source streams and adds their total into
// a compensated (two-sum) accumulator once per tile.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

template <int KIND, bool MASK>
__device__ __forceinline__ void pair2_f32(float2 sx, float2 sy, float2 sz, float2 rx, float2 ry, float2 rz, int2 spid,
                                          const float2 (&xt)[3], const float2 (&nt)[3], int pt, float2 (&acc)[3]) {
  const float2 dx = __fadd2_rn(xt[0], sx), dy = __fadd2_rn(xt[1], sy), dz = __fadd2_rn(xt[2], sz);
  const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
  float2 inv = f2(rsqrt_hw(r2.x), rsqrt_hw(r2.y));
  if (MASK) {
    if (spid.x == pt) inv.x = 0.0f;
    if (spid.y == pt) inv.y = 0.0f;
  }
  const float2 rr = __ffma2_rn(dz, rz, __ffma2_rn(dy, ry, __fmul2_rn(dx, rx)));
  if (KIND == 0) {
    const float2 rn = __ffma2_rn(dz, nt[2], __ffma2_rn(dy, nt[1], __fmul2_rn(dx, nt[0])));
    const float2 inv2 = __fmul2_rn(inv, inv);
    const float2 inv3 = __fmul2_rn(inv2, inv);
    const float2 c = __fmul2_rn(__fmul2_rn(__fmul2_rn(rn, rr), inv2), inv3);
    acc[0] = __ffma2_rn(c, dx, acc[0]);
    acc[1] = __ffma2_rn(c, dy, acc[1]);
    acc[2] = __ffma2_rn(c, dz, acc[2]);
  } else {
    const float2 inv3 = __fmul2_rn(__fmul2_rn(inv, inv), inv);
    const float2 c = __fmul2_rn(rr, inv3);
    acc[0] = __ffma2_rn(c, dx, __ffma2_rn(rx, inv, acc[0]));
    acc[1] = __ffma2_rn(c, dy, __ffma2_rn(ry, inv, acc[1]));
    acc[2] = __ffma2_rn(c, dz, __ffma2_rn(rz, inv, acc[2]));
  }
}

// Targets u < NU of the thread's NT (the rest of the arrays untouched): a warp whose later target
// slots are all empty skips them.
template <int KIND, bool MASK, int NT, int NU = NT>
__device__ __forceinline__ void pair_tile32x2(const float* __restrict__ ssx, const float* __restrict__ ssy,
                                              const float* __restrict__ ssz, const float* __restrict__ srx,
                                              const float* __restrict__ sry, const float* __restrict__ srz,
                                              const int* __restrict__ spid, int cnt4, const float2 (&xt)[NT][3],
                                              const float2 (&nt)[NT][3], const int (&pt)[NT], float2 (&acc)[NT][3]) {
#pragma unroll 2
  for (int l = 0; l < cnt4; l += 4) {
    const float4 ax = *reinterpret_cast<const float4*>(ssx + l), ay = *reinterpret_cast<const float4*>(ssy + l);
    const float4 az = *reinterpret_cast<const float4*>(ssz + l), bx = *reinterpret_cast<const float4*>(srx + l);
    const float4 by = *reinterpret_cast<const float4*>(sry + l), bz = *reinterpret_cast<const float4*>(srz + l);
    int4 pp = make_int4(-1, -1, -1, -1);
    if (MASK) pp = *reinterpret_cast<const int4*>(spid + l);
#pragma unroll
    for (int u = 0; u < NU; ++u) {
      pair2_f32<KIND, MASK>(f2(ax.x, ax.y), f2(ay.x, ay.y), f2(az.x, az.y), f2(bx.x, bx.y), f2(by.x, by.y),
                            f2(bz.x, bz.y), make_int2(pp.x, pp.y), xt[u], nt[u], pt[u], acc[u]);
      pair2_f32<KIND, MASK>(f2(ax.z, ax.w), f2(ay.z, ay.w), f2(az.z, az.w), f2(bx.z, bx.w), f2(by.z, by.w),
                            f2(bz.z, bz.w), make_int2(pp.z, pp.w), xt[u], nt[u], pt[u], acc[u]);
    }
  }
}

}  // namespace rbs
