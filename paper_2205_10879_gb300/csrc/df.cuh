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

// Tables of the DF exponential, filled on the host from FP64 values (each
// entry the DF rounding of the FP64 exp): e4[i] = exp(-i/4) for i < 128 and
// e256[i] = exp(-i/256) for i < 64, so exp(-j/256) = e4[j >> 6] * e256[j & 63]
// for j/256 < 32.
constexpr int kDfExpRange = 88;  // arguments at or above give 0 (exp(-88) < FLT_MIN)
constexpr int kDfExpTable = 32;  // arguments below use the tables
struct DfConsts {
  float2 e4[kDfExpTable * 4];
  float2 e256[64];
};

// exp(-a) for a >= 0 (DF).  For a < 32 the relative error is below 1e-13
// (the table entries and the two DF products contribute a few 2^-47 each,
// the series about 1e-15); from 32 on, where exp(-a) < 1.3e-14, the value is
// the FP32 exp2f of -a log2(e) (relative error below 2e-5 from the FP32
// product and the dropped a.lo, absolute below 5e-19),
// which keeps every kernel entry's absolute error far below 1e-13.  For a < 32:
//   j = floor(256 a.hi), and a.hi - j/256 in [0, 1/256) exactly (the
//   fractional part of the exactly scaled 256 a.hi); s = that + a.lo,
//   renormalised by TwoSum so that s.lo is below 2^-32;
//   exp(-a) = exp(-j/256) exp(-s), the first factor from the two tables;
//   exp(-s) = 1 - s + s^2/2 - s^3/6 + s^4/24 - s^5/120 (the next term is
//   below 1e-14): 1 - s.hi exactly as a pair, s.hi^2 exactly as a product
//   pair, the small rest in FP32.
// Arguments at or above 88, and NaN, give 0 by selection rather than an
// early return, so that several evaluations can interleave.
__device__ __forceinline__ dfl df_exp_neg(dfl a, const DfConsts& K) {
  const bool in_range = a.hi < (float)kDfExpRange;  // false for NaN
  const bool tail = a.hi >= (float)kDfExpTable;
  float tail_v = 0.0f;
  if (tail && in_range) tail_v = exp2f(-1.44269504f * a.hi);  // rare: a branch, not a select
  const float ah = in_range && !tail ? fmaxf(a.hi, 0.0f) : 0.0f;  // table indices stay in range
  const float al = in_range && !tail ? a.lo : 0.0f;
  const int j = (int)__fmul_rz(ah, 256.0f);                  // ah * 256 is exact
  const float sh = __fmaf_rn((float)j, -0.00390625f, ah);   // exact: frac(256 ah) / 256
  const dfl sv = df_two_sum(sh, al);                         // s, |sv.lo| <= 2^-33
  const dfl q = df_two_prod(sv.hi, sv.hi);                   // s.hi^2 = q.hi + q.lo
  const dfl h = df_quick(1.0f, -sv.hi);                      // 1 - s.hi
  const dfl t = df_two_sum(h.hi, __fmul_rn(0.5f, q.hi));     // + s.hi^2 / 2
  float lo = __fadd_rn(h.lo, t.lo);
  lo = __fmaf_rn(0.5f, q.lo, lo);
  lo = __fsub_rn(lo, sv.lo);                                 // - s.lo
  lo = __fmaf_rn(sv.hi, sv.lo, lo);                          // + s.hi s.lo (s^2 / 2)
  const float x = sv.hi;
  const float poly = x * (-0.16666667f + x * (0.041666668f - x * 0.008333334f));
  lo = __fmaf_rn(q.hi, poly, lo);                            // -s^3/6 + s^4/24 - s^5/120
  const dfl e = df_quick(t.hi, lo);
  const float2 u = K.e4[j >> 6], w = K.e256[j & 63];
  const dfl v = df_mul(df_mul(dfl{u.x, u.y}, dfl{w.x, w.y}), e);
  if (!in_range) return {0.0f, 0.0f};
  return tail ? dfl{tail_v, 0.0f} : v;
}

__device__ __forceinline__ double df_to_double(dfl x) { return (double)x.hi + (double)x.lo; }

}  // namespace fmgp
