// Double-float ("df") arithmetic on the FP32 pipes.
//
// GB300 issues one FP64 warp-instruction per ~84 cycles per SM sub-partition
// (1.0 TFLOP/s) against one FP32 warp-instruction per cycle (67 TFLOP/s).  The
// per-pair and per-rotation arithmetic of the timestep therefore runs on
// unevaluated sums hi + lo of two floats (about 48 significant bits) built from
// the error-free transformations of Dekker (1971) and Knuth (TAOCP vol. 2):
// two_sum, fast_two_sum and the FMA-based two_prod; the algorithms follow the
// double-double arithmetic of Hida, Li and Bailey (2001) with float in place
// of double.  The FP64 state is converted to and from df with integer bit
// operations, so no FP64 instruction is needed for the conversions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sl_tables.h"

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float h, float l) { df r; r.hi = h; r.lo = l; return r; }
__device__ __forceinline__ df df_f(float h) { return df_make(h, 0.0f); }

// s + e == a + b exactly.
__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df_make(s, e);
}
// Requires |a| >= |b| (or a == 0).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return df_make(s, e);
}
// p + e == a * b exactly.
__device__ __forceinline__ df two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return df_make(p, e);
}

__device__ __forceinline__ df df_neg(df a) { return df_make(-a.hi, -a.lo); }

// Accurate sum (both parts combined with error-free transformations).
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  df t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
// The cheaper sum of Hida, Li and Bailey's "sloppy" addition (one
// error-free sum of the high parts, the low parts added in float): its error
// is below ~2^-47 of max(|a|, |b|) rather than of |a + b|, so it is used only
// where that absolute error is already within the operands' own (a sum with
// no cancellation, or a difference of quantities that carry an error of that
// size, such as r - r0 with r from r^2 and 1/sqrt(r^2)).
__device__ __forceinline__ df df_add_sloppy(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_add_f(df a, float b) {
  df s = two_sum(a.hi, b);
  s.lo = __fadd_rn(s.lo, a.lo);
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_sqr(df a) {
  df p = two_prod(a.hi, a.hi);
  p.lo = __fmaf_rn(2.0f * a.hi, a.lo, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
// a * b + c
__device__ __forceinline__ df df_fma(df a, df b, df c) { return df_add(df_mul(a, b), c); }
// Multiply by an exact power of two.
__device__ __forceinline__ df df_scale(df a, float p2) { return df_make(a.hi * p2, a.lo * p2); }

// 1/sqrt(a), a > 0: hardware estimate, one Newton step in float (~2^-23),
// then one correction with the residual 1 - a y^2 in df: relative error
// below 5e-14 (4.6e-14 the largest over 4 million points of r^2 in
// [1, 64] against FP64).
__device__ __forceinline__ df df_rsqrt(df a) {
  float y = rsqrtf(a.hi);
  y = y * __fmaf_rn(-0.5f * a.hi * y, y, 1.5f);
  const df e = df_add_f(df_neg(df_mul(a, two_prod(y, y))), 1.0f);   // 1 - a y^2
  return fast_two_sum(y, 0.5f * y * e.hi);
}

// exp(x): x = n ln2/64 + r, n = 64 m + j, |r| <= ln2/128; n ln2/64 is exact in
// its first 14-bit piece for |n| < 1024 (|x| < 11; beyond, the relative error
// grows to ~1e-7, where every caller's exp(x) is below 2e-5 of its largest
// value or x is out of its range); exp(x) = 2^m T[j] (1 + p(r)),
// p(r) = r + q, q = r^2/2 + r^3 (1/6 + r/24 + r^2/120): r^2/2 from the exact
// square of r.hi plus r.hi r.lo, the cubic tail (< 2.7e-8) in float.
// Relative error below 7e-14 (6.1e-14 the largest over 4 million points
// of x in [-12, 6] against FP64 at the same input; 1e-14 for 99.99 % of
// them).
__device__ __forceinline__ df df_exp(df x) {
  float nf = rintf(x.hi * SL_64_LN2);
  int n = (int)nf;
  // r = x - n ln2/64 (n * C1 exact; x.hi - n C1 exact by Sterbenz)
  float r1 = __fsub_rn(x.hi, nf * SL_LN2_64_C1);
  // (r1, x.lo) is not normalised (x.lo belongs to |x|, not to |r1|): an
  // accurate sum; the two below have no cancellation (|q| < r^2, |T p| <
  // 0.011 T) and take the sloppy one
  df r = df_add(df_make(r1, x.lo), df_neg(df_add_f(two_prod(nf, SL_LN2_64_C2), nf * SL_LN2_64_C3)));
  const df P = two_prod(r.hi, r.hi);
  const float tail = r.hi * P.hi * __fmaf_rn(r.hi, __fmaf_rn(r.hi, 1.0f / 120.0f, 1.0f / 24.0f), 1.0f / 6.0f);
  const df q = df_make(0.5f * P.hi, __fmaf_rn(r.hi, r.lo, __fmaf_rn(0.5f, P.lo, tail)));
  const df p = df_add_sloppy(r, q);
  int j = n & 63, m = n >> 6;
  float2 t = __ldg(kSlExp2Table + j);
  df T = df_make(t.x, t.y);
  df e = df_add_sloppy(T, df_mul(T, p));
  float s = __int_as_float((127 + m) << 23);  // 2^m, |m| < 126
  return df_scale(e, s);
}

// Exact float of an integer m < 2^23 without a conversion instruction:
// the float 2^23 + m has m in its low mantissa bits.
__device__ __forceinline__ float u23_to_float(unsigned m) {
  return __fsub_rn(__uint_as_float(0x4B000000u | m), 8388608.0f);
}

// ---------------------------------------------------------------------------
// FP64 <-> float pieces by integer bit operations (no FP64 instruction).
// Values here are finite and far from the float range limits; pieces below
// 2^-126 are flushed to zero.
// ---------------------------------------------------------------------------

// x = hi + lo to ~48 bits: hi holds the top 24 significant bits of x
// (truncated), lo the next 24 (rounded).
__device__ __forceinline__ df df_from_double(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  int e = (int)((b >> 52) & 0x7ff);
  if (e == 0) return df_make(0.0f, 0.0f);
  if (e == 0x7ff) return df_make(__int_as_float(0x7fffffff), 0.0f);   // NaN/Inf -> NaN
  int ef = e - 1023 + 127;
  if (ef <= 0) return df_make(0.0f, 0.0f);
  if (ef >= 255) return df_make(__int_as_float(0x7fffffff), 0.0f);
  unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  float hi = __uint_as_float(sign | ((unsigned)ef << 23) | (unsigned)(mant >> 29));
  unsigned rest = (unsigned)(mant & 0x1FFFFFFFull);     // 29 bits below hi, units 2^(e-1075)
  int el = ef - 52;                                     // float exponent of 2^(e-1075)
  float lo = 0.0f;
  if (rest && el > 0) {
    // rest = 64 rh + rl; 64 rh + rl rounded once to 24 bits
    float r = __fmaf_rn(u23_to_float(rest >> 6), 64.0f, u23_to_float(rest & 63u));
    lo = r * __int_as_float(el << 23);
    if (sign) lo = -lo;
  }
  return df_make(hi, lo);
}

// Exact three-piece split of a double: x = h + m + l (all floats, exact).
// Exact float -> double by bit operations (finite, normal or zero inputs).
__device__ __forceinline__ double double_from_float(float f) {
  unsigned u = __float_as_uint(f);
  unsigned sign = u & 0x80000000u;
  unsigned e = (u >> 23) & 0xffu;
  if (e == 0) return 0.0;
  unsigned m = u & 0x7FFFFFu;
  if (e == 0xffu) return __hiloint2double((int)(sign | 0x7FF00000u | (m >> 3) | (m ? 0x80000u : 0u)), 0);
  unsigned hi = sign | ((e - 127u + 1023u) << 20) | (m >> 3);
  unsigned lo = m << 29;
  return __hiloint2double((int)hi, (int)lo);
}

// hi + lo as a double: two exact conversions and one FP64 add.
__device__ __forceinline__ double df_to_double(df a) {
  return double_from_float(a.hi) + double_from_float(a.lo);
}

// Running sum of products (h, l) += a * b, renormalised after every term so
// that l stays below half an ulp of h (its rounding is then relative to the
// partial sum, not to the sum of the terms' magnitudes).
__device__ __forceinline__ void acc_prod(float& h, float& l, df a, df b) {
  df p = two_prod(a.hi, b.hi);
  float lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  df s = two_sum(h, p.hi);
  df r = fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(l, lo)));
  h = r.hi;
  l = r.lo;
}
__device__ __forceinline__ df acc_done(float h, float l) { return fast_two_sum(h, l); }

// a < b for normalised df values.
__device__ __forceinline__ bool df_lt(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

// a / b: quotient, two corrections (~2^-46).
__device__ __forceinline__ df df_div(df a, df b) {
  const float q1 = a.hi / b.hi;
  const df r = df_sub(a, df_mul_f(b, q1));
  const float q2 = r.hi / b.hi;
  const df r2 = df_sub(r, df_mul_f(b, q2));
  const float q3 = r2.hi / b.hi;
  return df_add_f(fast_two_sum(q1, q2), q3);
}

// sqrt(a), a > 0: correctly rounded float root, one Newton correction;
// relative error below 2e-14 (1.5e-14 the largest over [0.5, 64]).
__device__ __forceinline__ df df_sqrt(df a) {
  const float y = sqrtf(a.hi);
  const df e = df_sub(a, two_prod(y, y));
  return fast_two_sum(y, e.hi / (2.0f * y));
}

// ln(u) for a normal positive u: u = m 2^e with m in [1/sqrt2, sqrt2),
// ln m = 2 atanh(z), z = (m - 1)/(m + 1), |z| <= 0.172, as the odd series
// 2 z sum_k z^(2k)/(2k+1) (terms beyond z^20 below 2^-48; the ones from
// 1/13 on summed in float), ln u = e ln2 + ln m.  No cancellation for u
// near 1 (e = 0, z small).
__device__ __forceinline__ df df_log(df u) {
  int e = ((__float_as_int(u.hi) >> 23) & 0xff) - 127;
  const float sc = __int_as_float((127 - e) << 23);     // 2^-e, exact
  df m = df_make(u.hi * sc, u.lo * sc);
  if (m.hi > SL_SQRT2_HI) { m = df_scale(m, 0.5f); e += 1; }
  const df z = df_div(df_add_f(m, -1.0f), df_add_f(m, 1.0f));
  const df w = df_sqr(z);
  const float wf = w.hi;
  const float tail = 1.0f / 13.0f + wf * (1.0f / 15.0f + wf * (1.0f / 17.0f + wf * (1.0f / 19.0f + wf * (1.0f / 21.0f))));
  df S = df_add_f(df_make(SL_INV_ODD11_HI, SL_INV_ODD11_LO), wf * tail);
  S = df_add(df_mul(w, S), df_make(SL_INV_ODD9_HI, SL_INV_ODD9_LO));
  S = df_add(df_mul(w, S), df_make(SL_INV_ODD7_HI, SL_INV_ODD7_LO));
  S = df_add(df_mul(w, S), df_make(SL_INV_ODD5_HI, SL_INV_ODD5_LO));
  S = df_add(df_mul(w, S), df_make(SL_INV_ODD3_HI, SL_INV_ODD3_LO));
  S = df_add_f(df_mul(w, S), 1.0f);
  const df lnm = df_scale(df_mul(z, S), 2.0f);
  return df_add(df_mul_f(df_make(SL_LN2_HI, SL_LN2_LO), (float)e), lnm);
}

// sin(2 pi u), cos(2 pi u) for u in [0, 1]: quadrant k = rint(4u),
// a = 2 pi (u - k/4) in [-pi/4, pi/4] (u - k/4 is exact), Taylor series of
// sin a / a and cos a to a^18 (the terms from 1/11! and 1/10! on in float),
// then the quadrant's swap and signs.
__device__ __forceinline__ void df_sincos_2pi(df u, df& sn, df& cs) {
  const float kf = rintf(u.hi * 4.0f);
  const df fr = df_add_f(u, -0.25f * kf);
  const df a = df_mul(fr, df_make(SL_2PI_HI, SL_2PI_LO));
  const df a2 = df_sqr(a);
  const float t = a2.hi;
  float tail = SL_INV_FAC11_HI - t * (SL_INV_FAC13_HI - t * (SL_INV_FAC15_HI - t * SL_INV_FAC17_HI));
  df S = df_add_f(df_make(SL_INV_FAC9_HI, SL_INV_FAC9_LO), -t * tail);
  S = df_sub(df_make(SL_INV_FAC7_HI, SL_INV_FAC7_LO), df_mul(a2, S));
  S = df_sub(df_make(SL_INV_FAC5_HI, SL_INV_FAC5_LO), df_mul(a2, S));
  S = df_sub(df_make(SL_INV_FAC3_HI, SL_INV_FAC3_LO), df_mul(a2, S));
  S = df_add_f(df_neg(df_mul(a2, S)), 1.0f);
  const df s = df_mul(a, S);
  tail = SL_INV_FAC10_HI - t * (SL_INV_FAC12_HI - t * (SL_INV_FAC14_HI - t * (SL_INV_FAC16_HI - t * SL_INV_FAC18_HI)));
  df Cc = df_add_f(df_make(SL_INV_FAC8_HI, SL_INV_FAC8_LO), -t * tail);
  Cc = df_sub(df_make(SL_INV_FAC6_HI, SL_INV_FAC6_LO), df_mul(a2, Cc));
  Cc = df_sub(df_make(SL_INV_FAC4_HI, SL_INV_FAC4_LO), df_mul(a2, Cc));
  Cc = df_sub(df_make(SL_INV_FAC2_HI, SL_INV_FAC2_LO), df_mul(a2, Cc));
  const df c = df_add_f(df_neg(df_mul(a2, Cc)), 1.0f);
  const int q = ((int)kf) & 3;
  if (q == 0) { sn = s; cs = c; }
  else if (q == 1) { sn = c; cs = df_neg(s); }
  else if (q == 2) { sn = df_neg(s); cs = df_neg(c); }
  else { sn = df_neg(c); cs = s; }
}
