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

// 1/sqrt(a), a > 0: hardware estimate, one Newton step with float
// corrections (~2^-44), then one in df (~2^-48).
__device__ __forceinline__ df df_rsqrt(df a) {
  float y = rsqrtf(a.hi);
  df y2 = two_prod(y, y);
  df e = df_add_f(df_neg(df_mul(a, y2)), 1.0f);          // 1 - a y^2
  df yd = df_add_f(df_f(y), 0.5f * y * e.hi);
  df e2 = df_add_f(df_neg(df_mul(a, df_sqr(yd))), 1.0f);  // 1 - a yd^2
  return df_add(yd, df_mul_f(yd, 0.5f * e2.hi));
}

// exp(x) for |x| < 80: x = n ln2/64 + r, n = 64 m + j, |r| <= ln2/128;
// exp(x) = 2^m * T[j] * (1 + p(r)), p(r) = r + r^2/2 + r^3 (1/6 + r/24 + r^2/120).
__device__ __forceinline__ df df_exp(df x) {
  float nf = rintf(x.hi * SL_64_LN2);
  int n = (int)nf;
  // r = x - n ln2/64 (n * C1 exact; x.hi - n C1 exact by Sterbenz)
  float r1 = __fsub_rn(x.hi, nf * SL_LN2_64_C1);
  df r = df_add(df_make(r1, x.lo), df_neg(df_add_f(two_prod(nf, SL_LN2_64_C2), nf * SL_LN2_64_C3)));
  r = fast_two_sum(r.hi, r.lo);
  const df c6 = df_make(SL_INV_FACT3_HI, SL_INV_FACT3_LO);  // 1/6 = hi + lo
  float tail = __fmaf_rn(r.hi, __fmaf_rn(r.hi, 1.0f / 120.0f, 1.0f / 24.0f), 0.0f);
  df c = df_add_f(c6, tail);
  df r2 = df_sqr(r);
  df r3 = df_mul(r2, r);
  df p = df_add(df_add(r, df_scale(r2, 0.5f)), df_mul(r3, c));
  int j = n & 63, m = n >> 6;
  float2 t = __ldg(kSlExp2Table + j);
  df T = df_make(t.x, t.y);
  df e = df_add(T, df_mul(T, p));
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
struct f3 {
  float h, m, l;
};
__device__ __forceinline__ f3 f3_from_double(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  int e = (int)((b >> 52) & 0x7ff);
  f3 r;
  r.h = r.m = r.l = 0.0f;
  int ef = e - 1023 + 127;
  if (e == 0 || ef <= 52) return r;                     // |x| < 2^-74: treat as zero
  if (ef >= 255) { r.h = __int_as_float(0x7fffffff); return r; }   // out of float range: NaN
  unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  r.h = __uint_as_float(sign | ((unsigned)ef << 23) | (unsigned)(mant >> 29));
  unsigned mid = (unsigned)((mant >> 5) & 0xFFFFFFu);   // next 24 bits, units 2^(e-1023-47)
  unsigned low = (unsigned)(mant & 0x1Fu);              // last 5 bits, units 2^(e-1023-52)
  float sm = __int_as_float((ef - 47) << 23);
  float sl = __int_as_float((ef - 52) << 23);
  r.m = __fmaf_rn(u23_to_float(mid >> 1), 2.0f, u23_to_float(mid & 1u)) * sm;  // exact: < 2^24
  r.l = u23_to_float(low) * sl;
  if (sign) { r.m = -r.m; r.l = -r.l; }
  return r;
}

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

// Minimum-image separation d = b - a - k L of exactly split coordinates,
// k = rint((b - a)/L), to df accuracy relative to d itself: the large pieces
// are differenced (and k L subtracted) with error-free two_sum before any
// rounding, so the cancellation across the periodic boundary is exact.
__device__ __forceinline__ df f3_sep(f3 b, f3 a, f3 L, float invL) {
  df hs = two_sum(b.h, -a.h);
  float k = rintf(hs.hi * invL);
  df h2 = two_sum(hs.hi, -k * L.h);                 // k L.h exact: |k| <= 1
  df ms = two_sum(b.m, -a.m);
  df m2 = two_sum(ms.hi, -k * L.m);
  float small = __fadd_rn(__fsub_rn(b.l, a.l), -k * L.l);
  df r = df_add(h2, m2);
  r = df_add_f(r, hs.lo);
  r = df_add_f(r, ms.lo);
  return df_add_f(r, small);
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
