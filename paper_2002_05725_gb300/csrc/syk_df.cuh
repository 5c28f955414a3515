// Double-float ("double-single") arithmetic for the complex128 matvec.
//
// GB300 executes FP64 FMA at 1/64 of the FP32 rate, so a complex128 matvec done in FP64 is
// bound by that pipe.  Here a double is carried as an unevaluated sum hi + lo of two floats
// (|lo| <= ulp(hi)/2, 48 significand bits), and the multiply-adds are done in FP32 with
// error-free transformations:
//   * Knuth's TwoSum: s = fl(a + b) and the exact error e = (a + b) - s, 6 additions, any
//     magnitudes (Knuth, TAOCP vol. 2, 4.2.2);
//   * the FMA form of Dekker's TwoProduct: p = fl(a b), e = fma(a, b, -p) exactly;
//   * Dekker's Fast2Sum (QuickTwoSum) to renormalise a pair with |hi| >= |lo|.
// Products hi*lo are needed only to FP32 accuracy (they are 2^-24 of the result); lo*lo is
// dropped.  The sum's low words are accumulated in FP32 and the pair is renormalised every
// few terms, so each sum of n terms carries a relative error of order n 2^-48 in the worst
// case (FP64: n 2^-53).  The operations use the _rn intrinsics so that the compiler never
// contracts a product into a later addition, which would break the exactness of TwoSum.
#pragma once
#include <cuda_runtime.h>

#include "syk_cplx.cuh"

namespace syk {

// Tag type selecting double-float arithmetic in the tiled matvec templates; its vector
// elements and complex coefficients are float4 (re_hi, im_hi, re_lo, im_lo).
struct DF {};
template <>
struct CT<DF> {
  using T = float4;
};

// s + e = a + b exactly
__device__ __forceinline__ float df_two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
  return s;
}

// (hi, lo) <- Fast2Sum(hi, lo), assuming |hi| >= |lo| or hi = 0
__device__ __forceinline__ void df_renorm(float& hi, float& lo) {
  const float s = __fadd_rn(hi, lo);
  lo = __fsub_rn(lo, __fsub_rn(s, hi));
  hi = s;
}

// Complex double-float values are packed in a float4 as (re_hi, im_hi, re_lo, im_lo).
// a += c * v for an accumulator a, coefficient c and vector element v of that form.
__device__ __forceinline__ void df_cmac(float4& a, const float4 c, const float4 v) {
  // real part: c.re v.re - c.im v.im
  const float p1 = __fmul_rn(c.x, v.x);
  float e1 = __fmaf_rn(c.x, v.x, -p1);
  e1 = __fmaf_rn(c.x, v.z, e1);
  e1 = __fmaf_rn(c.z, v.x, e1);
  const float p2 = __fmul_rn(c.y, v.y);
  float e2 = __fmaf_rn(c.y, v.y, -p2);
  e2 = __fmaf_rn(c.y, v.w, e2);
  e2 = __fmaf_rn(c.w, v.y, e2);
  float t1, t2;
  float s = df_two_sum(a.x, p1, t1);
  s = df_two_sum(s, -p2, t2);
  a.x = s;
  a.z = __fadd_rn(a.z, __fadd_rn(__fadd_rn(t1, t2), __fsub_rn(e1, e2)));
  // imaginary part: c.re v.im + c.im v.re
  const float q1 = __fmul_rn(c.x, v.y);
  float f1 = __fmaf_rn(c.x, v.y, -q1);
  f1 = __fmaf_rn(c.x, v.w, f1);
  f1 = __fmaf_rn(c.z, v.y, f1);
  const float q2 = __fmul_rn(c.y, v.x);
  float f2 = __fmaf_rn(c.y, v.x, -q2);
  f2 = __fmaf_rn(c.y, v.z, f2);
  f2 = __fmaf_rn(c.w, v.x, f2);
  float u1, u2;
  float r = df_two_sum(a.y, q1, u1);
  r = df_two_sum(r, q2, u2);
  a.y = r;
  a.w = __fadd_rn(a.w, __fadd_rn(__fadd_rn(u1, u2), __fadd_rn(f1, f2)));
}

__device__ __forceinline__ void df_renorm4(float4& a) {
  df_renorm(a.x, a.z);
  df_renorm(a.y, a.w);
}

// a += s * w for a real double-float w = (hi, lo) and a sign s = +-1 (exact negation)
__device__ __forceinline__ void df_add_signed(float& hi, float& lo, float whi, float wlo, bool neg) {
  float e;
  hi = df_two_sum(hi, neg ? -whi : whi, e);
  lo = __fadd_rn(lo, __fadd_rn(e, neg ? -wlo : wlo));
}

// (hi + lo) as a double, rounded once (to nearest) in FP64
__device__ __forceinline__ double2 df_to_double2(const float4 a) {
  return make_double2(__dadd_rn((double)a.x, (double)a.z), __dadd_rn((double)a.y, (double)a.w));
}

}  // namespace syk
