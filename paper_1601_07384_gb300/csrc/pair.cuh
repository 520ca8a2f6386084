// Binary64-accurate arithmetic on unevaluated pairs of binary32 numbers (hi, lo), value hi + lo:
// products split exactly by fused multiply-adds, sums kept error-free (TwoSum), so a sum of products
// is accurate to about 2^-48 of the sum of |terms| at a few binary32 operations per term, on a pipe
// 64 times faster than sm_103a's binary64 pipe.  Shared by the convection and support kernels.
#pragma once
#include "lp_ptx.cuh"

namespace stdg {

__device__ __forceinline__ float2 pair_split(double a) {
  const float h = (float)a;
  return make_float2(h, (float)(a - (double)h));
}
// The rounded products below are formed with __fmul_rn, which is never fused into a multiply-add:
// with the compiler's default contraction a plain product feeding the sum s + p may become
// fma(a, b, s), and the error-free sum would then no longer see the p whose rounding error it adds,
// leaving a binary32-sized error in the pair (measured: 3.5e-8 relative in convection).
// (s, c) += a b for pairs a, b: TwoProd of the high parts, cross terms into the error, TwoSum into s
__device__ __forceinline__ void pair_fma(float2 a, float2 b, float& s, float& c) {
  const float p = __fmul_rn(a.x, b.x);
  const float e = fmaf(a.x, b.x, -p);
  const float t = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
  const float s2 = s + p;
  const float bb = s2 - s;
  c += ((s - (s2 - bb)) + (p - bb)) + t;
  s = s2;
}
__device__ __forceinline__ double pair_value(float s, float c) { return (double)s + (double)c; }
// (s, c) with |c| small against |s| -> a normalised pair (hi, lo), hi = fl32(s + c) (Fast2Sum)
__device__ __forceinline__ float2 pair_norm(float s, float c) {
  const float h = s + c;
  return make_float2(h, c - (h - s));
}
// the product of two pairs as a normalised pair: the high parts' product exactly (FMA), the cross terms
// into its error
__device__ __forceinline__ float2 pair_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  const float e = fmaf(a.x, b.y, fmaf(a.y, b.x, fmaf(a.x, b.x, -p)));
  return pair_norm(p, e);
}
// a + b and a - b of pairs (TwoSum of the high parts, low parts added to its error)
__device__ __forceinline__ float2 pair_add(float2 a, float2 b) {
  const float s = a.x + b.x;
  const float bb = s - a.x;
  const float e = ((a.x - (s - bb)) + (b.x - bb)) + (a.y + b.y);
  return pair_norm(s, e);
}
__device__ __forceinline__ float2 pair_neg(float2 a) { return make_float2(-a.x, -a.y); }

// (s, c) += a b on both halves of (s, c): a broadcast (ah2 = (a_hi, a_hi), nah2 = -ah2,
// al2 = (a_lo, a_lo)), b one pair per half (bh2 = high parts, bl2 = low parts)
__device__ __forceinline__ void pair_fma2(float2 ah2, float2 nah2, float2 al2, float2 bh2, float2 bl2, float2& s,
                                          float2& c) {
  const float2 pn = __fmul2_rn(nah2, bh2);       // -(a_hi b_hi) rounded
  float2 e = __ffma2_rn(ah2, bh2, pn);           // its rounding error, exact
  e = __ffma2_rn(al2, bh2, e);
  e = __ffma2_rn(ah2, bl2, e);
  float2 s2, err;
  df_two_diff2(s, pn, s2, err);                   // s + a_hi b_hi, error-free
  c = __fadd2_rn(c, __fadd2_rn(err, e));
  s = s2;
}

}  // namespace stdg
