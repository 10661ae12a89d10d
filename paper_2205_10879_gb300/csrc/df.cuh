// Double-float ("DF") arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.
//
// On GB300 the FP64 pipe runs at 1/62 of the FP32 rate and CUDA's FP64 exp
// at about 1/130 of expf, so the mixed-precision path forms its refinement
// residuals and cross-covariances in DF on the FP32 pipe instead of FP64.
//
// Building blocks are the classical error-free transformations: TwoSum
// (Knuth, TAOCP vol. 2, 4.2.2), FastTwoSum (Dekker 1971) and TwoProduct via
// a fused multiply-add; the compound operations follow the double-double
// algorithms of Hida, Li & Bailey (QD library, 2001) carried over to float
// pairs.  Explicit _rn intrinsics keep the compiler from contracting or
// reordering the error terms.
#pragma once
#include <cuda_runtime.h>

namespace fmgp {

struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
  return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ dfl df_quick(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}

__device__ __forceinline__ dfl df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  return {p, e};
}

__device__ __forceinline__ dfl df_neg(dfl x) { return {-x.hi, -x.lo}; }

// Accurate sum (handles cancellation between x and y).
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  dfl s = df_two_sum(x.hi, y.hi);
  const dfl t = df_two_sum(x.lo, y.lo);
  float e = __fadd_rn(s.lo, t.hi);
  s = df_quick(s.hi, e);
  e = __fadd_rn(s.lo, t.lo);
  return df_quick(s.hi, e);
}

// Cheaper sum whose error is bounded by ~2^-47 (|x| + |y|): for sums of
// same-sign terms, or differences whose absolute error that bound covers.
__device__ __forceinline__ dfl df_add_fast(dfl x, dfl y) {
  const dfl s = df_two_sum(x.hi, y.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return df_quick(s.hi, e);
}

__device__ __forceinline__ dfl df_add_f(dfl x, float y) {
  const dfl s = df_two_sum(x.hi, y);
  const float e = __fadd_rn(s.lo, x.lo);
  return df_quick(s.hi, e);
}

__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
  const dfl p = df_two_prod(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.lo, p.lo);
  e = __fmaf_rn(x.lo, y.hi, e);
  return df_quick(p.hi, e);
}

__device__ __forceinline__ dfl df_mul_f(dfl x, float y) {
  const dfl p = df_two_prod(x.hi, y);
  const float e = __fmaf_rn(x.lo, y, p.lo);
  return df_quick(p.hi, e);
}

__device__ __forceinline__ dfl df_sqr(dfl x) {
  const dfl p = df_two_prod(x.hi, x.hi);
  const float e = __fmaf_rn(__fmul_rn(2.0f, x.hi), x.lo, p.lo);
  return df_quick(p.hi, e);
}

// acc + x*y (x, y, acc DF), the product rounded to DF first.
__device__ __forceinline__ dfl df_fma(dfl x, dfl y, dfl acc) { return df_add(acc, df_mul(x, y)); }

// Square root by one Newton (Karp-Markstein) correction of an FP32 root:
// s ~ sqrt(hi), result s + (x - s^2) / (2 s) with x - s^2 formed exactly.
// Written without an early return (0 for x <= 0 by selection) so that
// several independent evaluations can interleave.
__device__ __forceinline__ dfl df_sqrt(dfl x) {
  const bool pos = x.hi > 0.0f;
  const float xh = pos ? x.hi : 1.0f;
  // s needs only FP32-level accuracy: the correction below restores ~2^-46
  const float rs = rsqrtf(xh);
  const float s = __fmul_rn(xh, rs);
  const dfl p = df_two_prod(s, s);
  const float e = __fadd_rn(__fsub_rn(__fsub_rn(xh, p.hi), p.lo), pos ? x.lo : 0.0f);
  const float c = e * (0.5f * rs);
  const dfl r = df_quick(s, c);
  return {pos ? r.hi : 0.0f, pos ? r.lo : 0.0f};
}

// Constants of the DF exponential, filled on the host from FP64 values:
// ln 2 = ln2_1 + ln2_2 + ln2_3 (Cody & Waite 1980; ln2_1 has 14 significant
// bits so n * ln2_1 is exact for |n| < 2^10) and E[j + 24] = exp(-j/64) for
// j = -24..24 as DF pairs.
struct DfConsts {
  float ln2_1, ln2_2, ln2_3;
  float e_hi[49], e_lo[49];
};

// exp(-a) for a >= 0 (DF), relative error about 1e-13:
//   a = n ln2 + r, |r| <= ln2/2 (Cody-Waite reduction: a.hi - n ln2_1 is
//   exact by Sterbenz's lemma, the remaining small terms are summed in DF);
//   r = j/64 + s, |s| <= 1/128 (r.hi - j/64 is exact as well);
//   exp(-a) = 2^-n exp(-j/64) exp(-s),
//   exp(-s) = 1 - s + s^2/2 in DF + s^3 (-1/6 + s/24 - s^2/120 + s^3/720) in
//   FP32 (that tail is below 1e-7, so FP32 keeps it to ~1e-14).
// Arguments at or above 87 (and NaN) give 0, by selection rather than an
// early return; 2^-n is applied as an exact multiplication by a power of two.
__device__ __forceinline__ dfl df_exp_neg(dfl a, const DfConsts& K) {
  const bool in_range = a.hi < 87.0f;
  if (!in_range) a = {87.0f, 0.0f};
  const float nf = rintf(__fmul_rn(a.hi, 1.4426950408889634f));
  const float r1 = __fsub_rn(a.hi, __fmul_rn(nf, K.ln2_1));  // exact
  const dfl p2 = df_two_prod(nf, K.ln2_2);                    // n ln2_2 exactly
  const dfl c = df_two_sum(a.lo, -p2.hi);                     // a.lo - n ln2_2 (hi part)
  const float cl = __fsub_rn(__fsub_rn(c.lo, p2.lo), __fmul_rn(nf, K.ln2_3));
  dfl r = df_two_sum(r1, c.hi);
  r = df_quick(r.hi, __fadd_rn(r.lo, cl));
  int j = (int)rintf(__fmul_rn(r.hi, 64.0f));
  j = max(-24, min(24, j));
  const dfl s = df_quick(__fsub_rn(r.hi, (float)j * 0.015625f), r.lo);  // exact difference
  const dfl s2 = df_sqr(s);
  const dfl h1 = df_quick(1.0f, -s.hi);                   // 1 - s.hi, exact as a pair
  const dfl h2 = df_two_sum(h1.hi, __fmul_rn(0.5f, s2.hi));
  const float t = s.hi;
  const float tail =
      t * t * t *
      (-0.16666667f + t * (0.041666668f + t * (-0.008333334f + t * 0.0013888889f)));
  const float lo = __fadd_rn(__fadd_rn(__fsub_rn(__fadd_rn(h2.lo, h1.lo), s.lo),
                                       __fmul_rn(0.5f, s2.lo)), tail);
  const dfl e = df_quick(h2.hi, lo);
  dfl v = df_mul(dfl{K.e_hi[j + 24], K.e_lo[j + 24]}, e);
  const int ni = (int)nf;  // 0 <= ni <= 126
  const float sc = __int_as_float((127 - ni) << 23);
  return {in_range ? __fmul_rn(v.hi, sc) : 0.0f, in_range ? __fmul_rn(v.lo, sc) : 0.0f};
}

__device__ __forceinline__ double df_to_double(dfl x) { return (double)x.hi + (double)x.lo; }

}  // namespace fmgp
