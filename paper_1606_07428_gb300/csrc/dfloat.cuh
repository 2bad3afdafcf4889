// Double-float arithmetic on the float32 pipes, shared by the pair-sum kernels of the mobility and
// magnetostatic operators.
#pragma once

#include "common.cuh"

namespace rbs {

// Hardware reciprocal square root (PTX rsqrt.approx.ftz.f32, relative error below 2^-22): one
// instruction, where rsqrtf without flush-to-zero adds a denormal guard.  The pair separations are
// at least the particle gap, far from the float32 denormal range; r^2 = 0 (the excluded self pair)
// gives +inf, which the callers replace by 0.
__device__ __forceinline__ float rsqrt_hw(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Double-float arithmetic: each value is an unevaluated sum hi + lo of two float32 numbers (Dekker's
// and Knuth's error-free transformations with fused multiply-add), so the float32 pipes deliver about
// 44 bits per operation.
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
// a0 b0 + a1 b1 + a2 b2: products exact to the low part, the three high parts added with two-sums
// and every low part folded into one float32 sum (unnormalised result)
__device__ __forceinline__ dflt df_dot3(dflt a0, dflt b0, dflt a1, dflt b1, dflt a2, dflt b2) {
  const dflt p0 = df_mul(a0, b0), p1 = df_mul(a1, b1), p2 = df_mul(a2, b2);
  const dflt s1 = df_two_sum(p0.h, p1.h);
  const dflt s2 = df_two_sum(s1.h, p2.h);
  return {s2.h, ((s1.l + s2.l) + (p0.l + p1.l)) + p2.l};
}
// acc += v with the low parts carried unnormalised (renormalised when the tile is flushed)
__device__ __forceinline__ void df_acc(dflt& acc, dflt v) {
  const dflt s = df_two_sum(acc.h, v.h);
  acc.h = s.h;
  acc.l += s.l + v.l;
}

// y - o for y = yh + ym + yl and o = oh + om + ol (exact three-float splits), as a double-float pair:
// the three part differences are formed exactly by two-sums, the leading pair is added exactly, and
// the remaining small terms (at most 2^-48 |y| in size) are summed in float32 before renormalising.
__device__ __forceinline__ dflt df_diff3(float yh, float ym, float yl, float oh, float om, float ol) {
  const dflt s = df_two_sum(yh, -oh), t = df_two_sum(ym, -om), u = df_two_sum(yl, -ol);
  const dflt h = df_two_sum(s.h, t.h);
  const float l = ((s.l + t.l) + (u.h + u.l)) + h.l;
  const float hi = h.h + l;
  return {hi, l - (hi - h.h)};
}

// a + b for double-float pairs, both parts added with two-sums and the result renormalised twice.
__device__ __forceinline__ dflt df_add_accurate(dflt a, dflt b) {
  dflt s = df_two_sum(a.h, b.h);
  const dflt t = df_two_sum(a.l, b.l);
  s.l += t.h;
  float h = s.h + s.l;
  float l = s.l - (h - s.h);
  l += t.l;
  const float h2 = h + l;
  return {h2, l - (h2 - h)};
}

}  // namespace rbs
