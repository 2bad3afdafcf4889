// Packed double-float pair arithmetic shared by the direct sums (operators.cu) and the treecode
// (treecode.cu).
#pragma once

#include "common.cuh"
#include "dfloat.cuh"

namespace rbs {

// Double-float pair sums with two sources per instruction: the operations of pair_tile_df on float2
// pairs (__fadd2_rn, __fmul2_rn, __ffma2_rn, each two round-to-nearest float32 operations, so the
// error-free transformations stay exact per source), sources staged structure-of-arrays and padded
// to an even count with zero-density sources far away (they add exactly zero).
struct df2 {
  float2 h, l;
};
__device__ __forceinline__ float2 ng2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ df2 two_sum2(float2 a, float2 b) {
  const float2 s = __fadd2_rn(a, b);
  const float2 bb = __fadd2_rn(s, ng2(a));
  const float2 e = __fadd2_rn(__fadd2_rn(a, ng2(__fadd2_rn(s, ng2(bb)))), __fadd2_rn(b, ng2(bb)));
  return {s, e};
}
__device__ __forceinline__ df2 mul2(df2 a, df2 b) {
  const float2 p = __fmul2_rn(a.h, b.h);
  float2 e = __ffma2_rn(a.h, b.h, ng2(p));
  e = __ffma2_rn(a.h, b.l, e);
  e = __ffma2_rn(a.l, b.h, e);
  return {p, e};
}
__device__ __forceinline__ df2 dot3_2(df2 a0, df2 b0, df2 a1, df2 b1, df2 a2, df2 b2) {
  const df2 p0 = mul2(a0, b0), p1 = mul2(a1, b1), p2 = mul2(a2, b2);
  const df2 s1 = two_sum2(p0.h, p1.h);
  const df2 s2 = two_sum2(s1.h, p2.h);
  return {s2.h, __fadd2_rn(__fadd2_rn(__fadd2_rn(s1.l, s2.l), __fadd2_rn(p0.l, p1.l)), p2.l)};
}
__device__ __forceinline__ void acc2_add(df2& acc, df2 v) {
  const df2 s = two_sum2(acc.h, v.h);
  acc.h = s.h;
  acc.l = __fadd2_rn(acc.l, __fadd2_rn(s.l, v.l));
}
// the two lanes' double-float values added into one (unnormalised) pair
__device__ __forceinline__ dflt fold2(const df2& a) {
  const dflt s = df_two_sum(a.h.x, a.h.y);
  return {s.h, s.l + (a.l.x + a.l.y)};
}

template <int KIND, bool MASK>
__device__ __forceinline__ void pair2_df(const df2 (&y)[3], const df2 (&den)[3], int2 spid, const df2 (&xt)[3],
                                         const df2 (&nt)[3], int pt, df2 (&acc)[3], df2 (&acc2)[3]) {
  df2 d[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    d[c] = two_sum2(xt[c].h, ng2(y[c].h));
    d[c].l = __fadd2_rn(d[c].l, __fadd2_rn(xt[c].l, ng2(y[c].l)));
  }
  float2 p[3], e[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    p[c] = __fmul2_rn(d[c].h, d[c].h);
    e[c] = __ffma2_rn(d[c].h, d[c].h, ng2(p[c]));
    e[c] = __ffma2_rn(__fadd2_rn(d[c].h, d[c].h), d[c].l, e[c]);
  }
  const df2 s1 = two_sum2(p[0], p[1]);
  const df2 s2 = two_sum2(s1.h, p[2]);
  const float2 r2l = __fadd2_rn(__fadd2_rn(__fadd2_rn(__fadd2_rn(s1.l, s2.l), e[0]), e[1]), e[2]);
  const float2 r2h = s2.h;
  const float2 y0 = make_float2(rsqrt_hw(r2h.x), rsqrt_hw(r2h.y));
  const float2 q = __fmul2_rn(y0, y0);
  const float2 qe = __ffma2_rn(y0, y0, ng2(q));
  float2 t = __ffma2_rn(r2h, q, dup2(-1.0f));
  t = __ffma2_rn(r2h, qe, t);
  t = __ffma2_rn(r2l, q, t);
  df2 inv = {y0, __fmul2_rn(__fmul2_rn(dup2(-0.5f), t), y0)};
  if (MASK) {
    if (spid.x == pt) inv.h.x = inv.l.x = 0.0f;
    if (spid.y == pt) inv.h.y = inv.l.y = 0.0f;
  }
  const df2 rr = dot3_2(d[0], den[0], d[1], den[1], d[2], den[2]);
  const df2 inv2 = mul2(inv, inv);
  const df2 inv3 = mul2(inv2, inv);
  if (KIND == 0 || KIND == 2) {
    const df2 inv5 = mul2(inv3, inv2);
    const df2 rn = dot3_2(d[0], nt[0], d[1], nt[1], d[2], nt[2]);
    const df2 ck = mul2(mul2(rn, rr), inv5);
#pragma unroll
    for (int c = 0; c < 3; ++c) acc2_add(acc[c], mul2(ck, d[c]));
  }
  if (KIND == 1 || KIND == 2) {
    const df2 cs = mul2(rr, inv3);
    df2(&as)[3] = KIND == 2 ? acc2 : acc;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc2_add(as[c], mul2(den[c], inv));
      acc2_add(as[c], mul2(cs, d[c]));
    }
  }
}

}  // namespace rbs
