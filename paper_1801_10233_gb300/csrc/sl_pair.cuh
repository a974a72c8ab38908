// Device helpers shared by the kernels that gather pairs and rotate spins:
// split positions and spins, exact minimum-image separations in
// double-float, the spin bath's counter-based normals, and the single-spin
// propagator.
#pragma once

#include "sl_internal.cuh"
#include "sl_df64.cuh"

namespace {

__device__ __forceinline__ df F2(float2 v) { return df_make(v.x, v.y); }
__device__ __forceinline__ float2 D2(df a) { return make_float2(a.hi, a.lo); }

struct df3 {
  df x, y, z;
};
// Positions in fixed point for the pair kernels: X = rint(r 2^F), 64-bit
// integers, F = SL_FX_BITS, so that |X| < 2^61 for every position within a
// box length of the box.  The difference of two positions
// and its periodic shift by the integer box length are exact integer
// operations; the separation is then rounded once to double-float.
struct p3 {
  long long x, y, z;
};

// Positions, lists and tables are read-only in every kernel that gathers
// them; their loads go through the read-only path and may be issued early.
// A position (32 bytes, fixed point) and a spin's float split (32 bytes: hi
// then lo halves) each come in one 256-bit load.
__device__ __forceinline__ p3 load_pos(const SlDev& d, int j) {
  long long x, y, z, w;
  asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(x), "=l"(y), "=l"(z), "=l"(w) : "l"(d.rx + j));
  (void)w;
  p3 p;
  p.x = x; p.y = y; p.z = z;
  return p;
}

// sdf[2j] and sdf[2j + 1] (hi, lo float4) of spin j in one load.
__device__ __forceinline__ void load_sdf(const float4* sdf, int j, float4& h, float4& l) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(h.x), "=f"(h.y), "=f"(h.z), "=f"(h.w), "=f"(l.x), "=f"(l.y), "=f"(l.z), "=f"(l.w)
      : "l"(sdf + 2 * (size_t)j));
}

__device__ __forceinline__ df3 load_spin(const SlDev& d, int j) {
  float4 h, l;
  load_sdf(d.sdf, j, h, l);
  df3 s;
  s.x = df_make(h.x, l.x); s.y = df_make(h.y, l.y); s.z = df_make(h.z, l.z);
  return s;
}

// The replica's box and half box in fixed point, and the scales that bring
// the 20-bit pieces of a fixed-point difference back to Angstrom.
struct box3 {
  long long L[3], H[3];
  float s40, s20, s0;
};
__device__ __forceinline__ box3 load_box(const SlDev& d, const SlRep& R) {
  box3 b;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    b.L[a] = R.boxX[a];
    b.H[a] = R.halfX[a];
  }
  b.s40 = d.fx_s40; b.s20 = d.fx_s20; b.s0 = d.fx_s0;
  return b;
}

// Minimum-image difference b - a in fixed point (|b - a| < 1.5 L before the shift).
// A difference whose high word lies strictly inside (-H_hi, H_hi) is below H
// in magnitude and needs no shift: one 32-bit test decides that for all but
// the pairs across the box faces, which take the 64-bit comparisons (the
// result is the same either way).
__device__ __forceinline__ long long fx_diff(long long b, long long a, long long L, long long H) {
  long long D = b - a;
  const int hi = (int)(D >> 32), hh = (int)(H >> 32);
  if (hi > -hh && hi < hh) return D;
  D = D > H ? D - L : D;
  D = D < -H ? D + L : D;
  return D;
}

// m 2^e exactly for an integer 0 <= m < 2^23 (E = the float bits of
// 2^(23+e)): the float 2^(23+e) + m 2^e has m in its low mantissa bits, so
// one subtraction of 2^(23+e) gives the scaled piece without a conversion
// or a multiply.
__device__ __forceinline__ float u23_scaled(unsigned m, unsigned E, float two23e) {
  return __fsub_rn(__uint_as_float(E | m), two23e);
}
static_assert(SL_FX_BITS == 48, "the piece scales below are those of F = 48");
// D 2^-F (|D| < 2^61) as df: D = A 2^40 + B 2^20 + C with |A| < 2^21 and
// B, C < 2^20, each piece exact in a float (A 2^-8 from A + 2^21 under the
// exponent of 2^15, B 2^-28 under 2^-5, C 2^-48 under 2^-25); two error-free
// additions round the sum.
__device__ __forceinline__ df fx_to_df(long long D, const box3& B) {
  (void)B;
  const int A = (int)(D >> 40);
  const unsigned Bm = (unsigned)(D >> 20) & 0xFFFFFu, Cm = (unsigned)D & 0xFFFFFu;
  const float fa = u23_scaled((unsigned)(A + (1 << 21)), 0x47000000u, 40960.0f);   // 2^15 + 2^21 2^-8
  const float fb = u23_scaled(Bm, 0x3D000000u, 0.03125f);                            // 2^-5
  const float fc = u23_scaled(Cm, 0x33000000u, 2.98023223876953125e-8f);             // 2^-25
  const df s = fast_two_sum(fa, fb);          // |fa| >= |fb| unless A = 0
  const df t = two_sum(s.hi, fc);
  return fast_two_sum(t.hi, __fadd_rn(t.lo, s.lo));
}
// The same value to about float precision (the cutoff pre-checks).
__device__ __forceinline__ float fx_to_float(long long D, const box3& B) {
  (void)B;
  const int A = (int)(D >> 40);
  const unsigned Bm = (unsigned)(D >> 20) & 0xFFFFFu;
  return __fadd_rn(u23_scaled((unsigned)(A + (1 << 21)), 0x47000000u, 40960.0f),
                   u23_scaled(Bm, 0x3D000000u, 0.03125f));
}

__device__ __forceinline__ df3 pair_sep(const box3& B, const p3& a, const p3& b) {
  df3 r;
  r.x = fx_to_df(fx_diff(b.x, a.x, B.L[0], B.H[0]), B);
  r.y = fx_to_df(fx_diff(b.y, a.y, B.L[1], B.H[1]), B);
  r.z = fx_to_df(fx_diff(b.z, a.z, B.L[2], B.H[2]), B);
  return r;
}

// Minimum-image difference of a pair and its float r^2, for a cutoff test
// before the exact separation: the float value is within 2^-20 A of the
// exact one per component, far inside the 1e-4 relative margin the callers
// allow on r^2.
struct pre3 {
  float r2;
  long long dx, dy, dz;
};
__device__ __forceinline__ pre3 pair_pre(const box3& B, const p3& a, const p3& b) {
  pre3 q;
  q.dx = fx_diff(b.x, a.x, B.L[0], B.H[0]);
  q.dy = fx_diff(b.y, a.y, B.L[1], B.H[1]);
  q.dz = fx_diff(b.z, a.z, B.L[2], B.H[2]);
  const float x = fx_to_float(q.dx, B), y = fx_to_float(q.dy, B), z = fx_to_float(q.dz, B);
  q.r2 = x * x + y * y + z * z;
  return q;
}
// The exact separation from pair_pre's differences: the same value as pair_sep.
__device__ __forceinline__ df3 pair_sep_k(const box3& B, const p3& a, const p3& b, const pre3& q) {
  df3 r;
  r.x = fx_to_df(q.dx, B);
  r.y = fx_to_df(q.dy, B);
  r.z = fx_to_df(q.dz, B);
  return r;
}

// |d|^2 of a separation: three exact squares of the high parts, the cross
// and low terms in float, the three (positive) high products summed
// error-free and the low parts folded in once; about 2^-47 relative, as for
// a running df sum of the three squares.
__device__ __forceinline__ df sep_r2(const df3& d) {
  const df px = two_prod(d.x.hi, d.x.hi), py = two_prod(d.y.hi, d.y.hi), pz = two_prod(d.z.hi, d.z.hi);
  const float lx = __fmaf_rn(2.0f * d.x.hi, d.x.lo, px.lo), ly = __fmaf_rn(2.0f * d.y.hi, d.y.lo, py.lo),
              lz = __fmaf_rn(2.0f * d.z.hi, d.z.lo, pz.lo);
  const df s = two_sum(px.hi, py.hi);
  const df t = two_sum(s.hi, pz.hi);
  return fast_two_sum(t.hi, __fadd_rn(__fadd_rn(t.lo, s.lo), __fadd_rn(__fadd_rn(lx, ly), lz)));
}

__device__ __forceinline__ df dot3(const df3& a, const df3& b) {
  float h = 0.0f, l = 0.0f;
  acc_prod(h, l, a.x, b.x);
  acc_prod(h, l, a.y, b.y);
  acc_prod(h, l, a.z, b.z);
  return acc_done(h, l);
}

__device__ __forceinline__ df3 cross3(const df3& a, const df3& b) {
  df3 c;
  float h, l;
  h = l = 0.0f; acc_prod(h, l, a.y, b.z); acc_prod(h, l, df_neg(a.z), b.y); c.x = acc_done(h, l);
  h = l = 0.0f; acc_prod(h, l, a.z, b.x); acc_prod(h, l, df_neg(a.x), b.z); c.y = acc_done(h, l);
  h = l = 0.0f; acc_prod(h, l, a.x, b.y); acc_prod(h, l, df_neg(a.y), b.x); c.z = acc_done(h, l);
  return c;
}

// rint(x 2^48), ties to even, from the IEEE-754 fields of x by integer
// operations (GB300's FP64 pipe is slow): x 2^48 = m 2^(e - 1027) with the
// 53-bit significand m and biased exponent e.  Values of 2^14 A or more (and
// non-finite ones) saturate to +-2^62; they occur only before the first wrap
// into the box, when no pair kernel reads them.
__device__ __forceinline__ long long fx_from_double(double x) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0) return 0;
  const long long m = (b & 0xFFFFFFFFFFFFFll) | (1ll << 52);
  const int sh = e - 1075 + SL_FX_BITS;
  long long X;
  if (sh >= 10) {
    X = 1ll << 62;
  } else if (sh >= 0) {
    X = m << sh;
  } else if (sh > -54) {
    const int s = -sh;
    const long long q = m >> s, rem = m & ((1ll << s) - 1), half = 1ll << (s - 1);
    X = q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
  } else {
    X = 0;
  }
  return b < 0 ? -X : X;
}

// Fixed-point copy of a position.
__device__ __forceinline__ SlFix fx_pos(double4_32a r) {
  SlFix x;
  x.x = fx_from_double(r.x);
  x.y = fx_from_double(r.y);
  x.z = fx_from_double(r.z);
  x.w = 0;
  return x;
}
__device__ __forceinline__ void store_pos_split(const SlDev& d, int k, double4_32a r) { d.rx[k] = fx_pos(r); }

// |a - b|^2 in A^2 (float) of two fixed-point positions (no periodic shift).
__device__ __forceinline__ float fx_dist2(const SlFix& a, const SlFix& b) {
  const float s = 3.5527136788005009e-15f;   // 2^-48
  const float x = (float)(a.x - b.x) * s, y = (float)(a.y - b.y) * s, z = (float)(a.z - b.z) * s;
  return x * x + y * y + z * z;
}

// r has finite components (exponent field not all ones).
__device__ __forceinline__ bool finite3(double4_32a r) {
  const unsigned hx = (unsigned)(__double_as_longlong(r.x) >> 32), hy = (unsigned)(__double_as_longlong(r.y) >> 32),
                 hz = (unsigned)(__double_as_longlong(r.z) >> 32);
  return ((hx & 0x7ff00000u) != 0x7ff00000u) && ((hy & 0x7ff00000u) != 0x7ff00000u) &&
         ((hz & 0x7ff00000u) != 0x7ff00000u);
}

__device__ __forceinline__ void store_spin_split(const SlDev& d, int k, double4_32a s) {
  df x = df_from_double(s.x), y = df_from_double(s.y), z = df_from_double(s.z);
  d.sdf[2 * (size_t)k] = make_float4(x.hi, y.hi, z.hi, 0.0f);
  d.sdf[2 * (size_t)k + 1] = make_float4(x.lo, y.lo, z.lo, 0.0f);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11) and Box-Muller normals for the spin bath.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
    unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ double3 gauss3(uint64_t seed, int replica, long long step, int subpass, int atom) {
  uint4 x = philox4x32_10(make_uint4((unsigned)atom, (unsigned)step, (unsigned)subpass, (unsigned)replica),
                          make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
  const double inv32 = 2.3283064365386962890625e-10;  // 2^-32
  const double twopi = 6.283185307179586476925286766559;
  double u0 = ((double)x.x + 0.5) * inv32, u1 = ((double)x.y + 0.5) * inv32;
  double u2 = ((double)x.z + 0.5) * inv32, u3 = ((double)x.w + 0.5) * inv32;
  double ra = sqrt(-2.0 * log(u0)), rb = sqrt(-2.0 * log(u2));
  double s1, c1, s3, c3;
  sincos(twopi * u1, &s1, &c1);
  sincos(twopi * u3, &s3, &c3);
  return make_double3(ra * c1, ra * s1, rb * c3);
}

// The same three normals in double-float on the FP32 pipes (Box-Muller with
// the double-float log, sqrt and sincos of sl_df64.cuh), within ~1e-14 of the
// FP64 values.
__device__ __forceinline__ df unit_from_word(unsigned x) {
  // (x + 1/2) 2^-32 exactly: 24 high bits and the rest as two floats
  const df u = fast_two_sum(__uint2float_rn(x >> 8) * 256.0f, __uint2float_rn(x & 255u) + 0.5f);
  return df_scale(u, 2.3283064365386962890625e-10f);
}
__device__ __forceinline__ df3 gauss3_df(uint64_t seed, int replica, long long step, int subpass, int atom) {
  uint4 x = philox4x32_10(make_uint4((unsigned)atom, (unsigned)step, (unsigned)subpass, (unsigned)replica),
                          make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
  const df ra = df_sqrt(df_scale(df_log(unit_from_word(x.x)), -2.0f));
  const df rb = df_sqrt(df_scale(df_log(unit_from_word(x.z)), -2.0f));
  df s1, c1, s3, c3;
  df_sincos_2pi(unit_from_word(x.y), s1, c1);
  df_sincos_2pi(unit_from_word(x.w), s3, c3);
  df3 g;
  g.x = df_mul(ra, c1);
  g.y = df_mul(ra, s1);
  g.z = df_mul(rb, c3);
  return g;
}

// Lattice bath over |dt|/2 (Eq. p_advance_T without the conservative force),
// the exact Ornstein-Uhlenbeck flow v <- c1 v + sig xi, xi ~ N(0, 1) per
// component from Philox (seed; atom id within its replica, step, sub-pass,
// replica); sub-pass 4 before the first half-kick, 5 after the closing one.
__device__ __forceinline__ double4_32a lattice_bath(const SlDev& d, int i, double4_32a v, int subpass) {
  const SlRep& R = d.reps[__ldg(d.arep + i)];
  if (R.lat_c1 == 1.0 && R.lat_sig == 0.0) return v;
  double xi[3] = {0.0, 0.0, 0.0};
  if (R.lat_sig > 0.0) {
    const df3 g = gauss3_df(d.seed, R.replica, d.ctrl->step, subpass, d.perm[i] - R.atom0);
    xi[0] = df_to_double(g.x); xi[1] = df_to_double(g.y); xi[2] = df_to_double(g.z);
  }
  v.x = R.lat_c1 * v.x + R.lat_sig * xi[0];
  v.y = R.lat_c1 * v.y + R.lat_sig * xi[1];
  v.z = R.lat_c1 * v.z + R.lat_sig * xi[2];
  return v;
}

// ---------------------------------------------------------------------------
// Single-spin propagator e^{L_si tau} as an increment of s:
//   s' - s = -u B s + tau A (w x s) + tau^2 B (w.s) w,      u = tau^2 |w|^2.
// Exact rotation by theta = |w| tau: A = sin(theta)/theta,
// B = (1 - cos theta)/theta^2 (even series in theta; for u <= 1e-3 the series
// are summed in df, beyond that A and B come from FP64 sin).  Cayley map of
// Sec. 3: A = 1/(1 + u/4), B = A/2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void rot_coeffs(df u, int cayley, df& A, df& B) {
  if (cayley) {
    df den = df_add_f(df_scale(u, 0.25f), 1.0f);
    float y0 = __frcp_rn(den.hi);
    df e = df_add_f(df_neg(df_mul_f(den, y0)), 1.0f);     // 1 - den y0
    A = df_add_f(df_f(y0), y0 * e.hi);                     // 1 / den
    B = df_scale(A, 0.5f);
  } else if (u.hi <= 2e-4f) {
    // theta <= 0.014: A = 1 - u (1/6 - u/120 + u^2/5040), B = 1/2 - u (1/24 - u/720 + u^2/40320);
    // the u^2 terms and beyond are below 1e-17 of A and B
    const df c6 = df_make(SL_INV_FACT3_HI, SL_INV_FACT3_LO);
    const df c24 = df_make(SL_INV_FACT4_HI, SL_INV_FACT4_LO);
    df a1 = df_add_f(c6, -u.hi * __fmaf_rn(-u.hi, 1.0f / 5040.0f, 1.0f / 120.0f));
    df b1 = df_add_f(c24, -u.hi * __fmaf_rn(-u.hi, 1.0f / 40320.0f, 1.0f / 720.0f));
    A = df_add_f(df_neg(df_mul(u, a1)), 1.0f);
    B = df_add_f(df_neg(df_mul(u, b1)), 0.5f);
  } else if (u.hi <= 1e-3f) {
    const df c6 = df_make(SL_INV_FACT3_HI, SL_INV_FACT3_LO);       // 1/3!
    const df c120 = df_make(SL_INV_FACT5_HI, SL_INV_FACT5_LO);     // 1/5!
    const df c24 = df_make(SL_INV_FACT4_HI, SL_INV_FACT4_LO);      // 1/4!
    const df c720 = df_make(SL_INV_FACT6_HI, SL_INV_FACT6_LO);     // 1/6!
    float ta = __fmaf_rn(-u.hi, __fmaf_rn(-u.hi, 1.0f / 39916800.0f, 1.0f / 362880.0f), 1.0f / 5040.0f);
    float tb = __fmaf_rn(-u.hi, __fmaf_rn(-u.hi, 1.0f / 479001600.0f, 1.0f / 3628800.0f), 1.0f / 40320.0f);
    df a1 = df_sub(c6, df_mul(u, df_add_f(c120, -u.hi * ta)));     // 1/6 - u/120 + u^2/5040 - ...
    df b1 = df_sub(c24, df_mul(u, df_add_f(c720, -u.hi * tb)));    // 1/24 - u/720 + u^2/40320 - ...
    A = df_add_f(df_neg(df_mul(u, a1)), 1.0f);
    B = df_add_f(df_neg(df_mul(u, b1)), 0.5f);
  } else {
    double ud = df_to_double(u);
    double th = sqrt(ud);
    double hs = sin(0.5 * th);
    A = df_from_double(sin(th) / th);
    B = df_from_double(2.0 * hs * hs / ud);
  }
}

// a0 b0 + a1 b1 + a2 b2 and a0 b0 - a1 b1 with the products formed side by
// side (exact high products, cross and low terms in float), the high parts
// combined by error-free sums and the low parts folded in once: the same
// accuracy as a running sum (about 2^-47 of the largest term, absolute) in
// far fewer dependent steps, for the single-spin propagator, whose chain of
// dependent rotations sets the colour pass's latency.
__device__ __forceinline__ float prod_lo(df a, df b, float plo) {
  return __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, plo));
}
__device__ __forceinline__ df sum3_prod(df a0, df b0, df a1, df b1, df a2, df b2) {
  const df p0 = two_prod(a0.hi, b0.hi), p1 = two_prod(a1.hi, b1.hi), p2 = two_prod(a2.hi, b2.hi);
  const float l = __fadd_rn(__fadd_rn(prod_lo(a0, b0, p0.lo), prod_lo(a1, b1, p1.lo)), prod_lo(a2, b2, p2.lo));
  const df s = two_sum(p0.hi, p1.hi);
  const df t = two_sum(s.hi, p2.hi);
  return fast_two_sum(t.hi, __fadd_rn(__fadd_rn(t.lo, s.lo), l));
}
__device__ __forceinline__ df diff2_prod(df a0, df b0, df a1, df b1) {
  const df p0 = two_prod(a0.hi, b0.hi), p1 = two_prod(a1.hi, b1.hi);
  const float l = __fsub_rn(prod_lo(a0, b0, p0.lo), prod_lo(a1, b1, p1.lo));
  const df s = two_sum(p0.hi, -p1.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, l));
}

__device__ __forceinline__ df3 rot_increment(const df3& w, const df3& s, df tau, int cayley) {
  const df w2 = sum3_prod(w.x, w.x, w.y, w.y, w.z, w.z);
  const df tau2 = df_sqr(tau);
  const df u = df_mul(w2, tau2);
  df A, B;
  rot_coeffs(u, cayley, A, B);
  // w.s and w x s do not depend on A, B: they overlap rot_coeffs
  const df ws = sum3_prod(w.x, s.x, w.y, s.y, w.z, s.z);
  df3 c;
  c.x = diff2_prod(w.y, s.z, w.z, s.y);
  c.y = diff2_prod(w.z, s.x, w.x, s.z);
  c.z = diff2_prod(w.x, s.y, w.y, s.x);
  const df nuB = df_neg(df_mul(u, B));
  const df tA = df_mul(tau, A);
  const df tBws = df_mul(df_mul(tau2, B), ws);
  df3 inc;
  inc.x = sum3_prod(nuB, s.x, tA, c.x, tBws, w.x);
  inc.y = sum3_prod(nuB, s.y, tA, c.y, tBws, w.y);
  inc.z = sum3_prod(nuB, s.z, tA, c.z, tBws, w.z);
  return inc;
}

// ---------------------------------------------------------------------------
// Tabulated embedded-atom potential (App. B): natural cubic splines on
// uniform grids.  Interval k = floor(x/h) (clamped to the grid; a value just
// below a knot may take the next interval at u ~ -1e-16, where the two cubics
// agree to rounding), u = x/h - k, value c0 + u (c1 + u (c2 + u c3)), slope
// (c1 + u (2 c2 + 3 u c3))/h.  A table not yet set (tab_n = 0) is zero.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int tab_interval(const SlDev& d, int t, float uhi) {
  const int k = (int)floorf(uhi);
  return max(0, min(k, d.tab_n[t] - 2));
}

// Value (double-float); *slope (if not NULL) the derivative.
__device__ __forceinline__ df tab_value_df(const SlDev& d, int t, df x, df* slope) {
  if (d.tab_n[t] < 2) {
    if (slope) *slope = df_f(0.0f);
    return df_f(0.0f);
  }
  const df ih = F2(d.tab_ih_f[t]);
  const df ux = df_mul(x, ih);
  const int k = tab_interval(d, t, ux.hi);
  const df u = df_add_f(ux, -(float)k);
  const float4 a = __ldg(d.tab_f[t] + 2 * (size_t)k), b = __ldg(d.tab_f[t] + 2 * (size_t)k + 1);
  const df c0 = df_make(a.x, a.y), c1 = df_make(a.z, a.w), c2 = df_make(b.x, b.y), c3 = df_make(b.z, b.w);
  if (slope) {
    const df q = df_add(df_scale(c2, 2.0f), df_mul(df_mul_f(c3, 3.0f), u));
    *slope = df_mul(df_add(c1, df_mul(u, q)), ih);
  }
  return df_add(c0, df_mul(u, df_add(c1, df_mul(u, df_add(c2, df_mul(u, c3))))));
}

// Slope only (the force kernel's pair terms).
__device__ __forceinline__ df tab_slope_df(const SlDev& d, int t, df x) {
  if (d.tab_n[t] < 2) return df_f(0.0f);
  const df ih = F2(d.tab_ih_f[t]);
  const df ux = df_mul(x, ih);
  const int k = tab_interval(d, t, ux.hi);
  const df u = df_add_f(ux, -(float)k);
  const float4 a = __ldg(d.tab_f[t] + 2 * (size_t)k), b = __ldg(d.tab_f[t] + 2 * (size_t)k + 1);
  const df c1 = df_make(a.z, a.w), c2 = df_make(b.x, b.y), c3 = df_make(b.z, b.w);
  const df q = df_add(df_scale(c2, 2.0f), df_mul(df_mul_f(c3, 3.0f), u));
  return df_mul(df_add(c1, df_mul(u, q)), ih);
}

// FP64 value (the energies).
__device__ __forceinline__ double tab_value_d(const SlDev& d, int t, double x) {
  if (d.tab_n[t] < 2) return 0.0;
  const double ux = x * d.tab_ih[t];
  int k = (int)floor(ux);
  k = max(0, min(k, d.tab_n[t] - 2));
  const double u = ux - (double)k;
  const double* c = d.tab_d[t] + 4 * (size_t)k;
  return c[0] + u * (c[1] + u * (c[2] + u * c[3]));
}

// ---------------------------------------------------------------------------
// Spin-orbit terms (App. A.2)
// ---------------------------------------------------------------------------
// f(r) = 4 alpha x (1 - gamma x) e^{-x}, x = r^2/delta^2 (Eq. BSfunction), and
// f'(r)/r = 8 alpha/delta^2 e^{-x} (1 - x (1 + 2 gamma - gamma x)), from r^2.
__device__ __forceinline__ void bs_eval(const SlBsF& c, df r2, df& f, df& fpr) {
  const df x = df_mul(r2, F2(c.ix));
  const df ex = df_exp(df_neg(x));
  const df g = F2(c.g);
  f = df_mul(df_mul(F2(c.a4), x), df_mul(df_add_f(df_neg(df_mul(g, x)), 1.0f), ex));
  const df poly = df_add_f(df_neg(df_mul(x, df_add_f(df_sub(df_scale(g, 2.0f), df_mul(g, x)), 1.0f))), 1.0f);
  fpr = df_mul(df_mul(F2(c.a8d2), ex), poly);
}

// One exchange-list entry with its spin-orbit coefficients: J, g1, d and the
// unit vector e from atom i to its neighbour.
struct SoEntry {
  df J, g, dm;
  df3 e;
};

__device__ __forceinline__ SoEntry load_so(const SlDev& d, size_t e) {
  const size_t P = (size_t)d.max_ex * (size_t)d.n;
  SoEntry q;
  q.J = F2(__ldg(d.exJ + e));
  q.g = F2(__ldg(d.exso + e));
  q.dm = F2(__ldg(d.exso + P + e));
  q.e.x = F2(__ldg(d.exso + 2 * P + e));
  q.e.y = F2(__ldg(d.exso + 3 * P + e));
  q.e.z = F2(__ldg(d.exso + 4 * P + e));
  return q;
}

// (h, l) += J s_j + g1 ((e.s_j) e - s_j/3) + d e x s_j: minus the derivative of
// the exchange, Neel and DMI energies of the pair with respect to s_i.
__device__ __forceinline__ void so_field_acc(const SoEntry& q, const df3& sj, float& hx, float& lx, float& hy,
                                             float& ly, float& hz, float& lz) {
  const df A = df_sub(q.J, df_mul(q.g, df_make(SL_INV_ODD3_HI, SL_INV_ODD3_LO)));
  const df c = df_mul(q.g, dot3(q.e, sj));
  const df3 X = cross3(q.e, sj);
  acc_prod(hx, lx, A, sj.x); acc_prod(hx, lx, c, q.e.x); acc_prod(hx, lx, q.dm, X.x);
  acc_prod(hy, ly, A, sj.y); acc_prod(hy, ly, c, q.e.y); acc_prod(hy, ly, q.dm, X.y);
  acc_prod(hz, lz, A, sj.z); acc_prod(hz, lz, c, q.e.z); acc_prod(hz, lz, q.dm, X.z);
}

// Anisotropy precession vector c (s.n) n, c = 2K/hbar (or over 1 + lambda^2).
__device__ __forceinline__ df3 aniso_vec(const SlDev& d, const df3& s, df c) {
  df3 n;
  n.x = F2(d.an_n_f[0]); n.y = F2(d.an_n_f[1]); n.z = F2(d.an_n_f[2]);
  const df k = df_mul(c, dot3(s, n));
  df3 a;
  a.x = df_mul(k, n.x); a.y = df_mul(k, n.y); a.z = df_mul(k, n.z);
  return a;
}

// The increment of one anisotropy turn over tau: rot_increment with
// w = c (s.n) n and |n| = 1, i.e. theta = c (s.n) tau, u = theta^2 and
//   s' - s = -u B (s - (s.n) n) + theta A (n x s).
__device__ __forceinline__ df3 aniso_increment(const SlDev& d, const df3& s, df c, df tau, int cayley) {
  df3 n;
  n.x = F2(d.an_n_f[0]); n.y = F2(d.an_n_f[1]); n.z = F2(d.an_n_f[2]);
  const df sn = dot3(s, n);
  const df th = df_mul(df_mul(c, sn), tau);
  const df u = df_sqr(th);
  df A, B;
  rot_coeffs(u, cayley, A, B);
  const df nuB = df_neg(df_mul(u, B)), tA = df_mul(th, A);
  const df3 x = cross3(n, s);
  df3 inc;
  float h = 0.0f, l = 0.0f;
  acc_prod(h, l, nuB, df_sub(s.x, df_mul(sn, n.x))); acc_prod(h, l, tA, x.x);
  inc.x = acc_done(h, l);
  h = l = 0.0f;
  acc_prod(h, l, nuB, df_sub(s.y, df_mul(sn, n.y))); acc_prod(h, l, tA, x.y);
  inc.y = acc_done(h, l);
  h = l = 0.0f;
  acc_prod(h, l, nuB, df_sub(s.z, df_mul(sn, n.z))); acc_prod(h, l, tA, x.z);
  inc.z = acc_done(h, l);
  return inc;
}

// FP64 versions for the observables: the spin-orbit field of one entry and
// the pair's spin-orbit energy, from the tables.
__device__ __forceinline__ double d_of(float2 v) { return double_from_float(v.x) + double_from_float(v.y); }

__device__ __forceinline__ void so_field_d(const SlDev& d, size_t e, const double4_32a& sj, double& hx, double& hy,
                                           double& hz) {
  const size_t P = (size_t)d.max_ex * (size_t)d.n;
  const double g = d_of(d.exso[e]), dm = d_of(d.exso[P + e]);
  const double ex = d_of(d.exso[2 * P + e]), ey = d_of(d.exso[3 * P + e]), ez = d_of(d.exso[4 * P + e]);
  const double es = ex * sj.x + ey * sj.y + ez * sj.z;
  hx += g * (es * ex - sj.x / 3.0) + dm * (ey * sj.z - ez * sj.y);
  hy += g * (es * ey - sj.y / 3.0) + dm * (ez * sj.x - ex * sj.z);
  hz += g * (es * ez - sj.z / 3.0) + dm * (ex * sj.y - ey * sj.x);
}

__device__ __forceinline__ double so_pair_energy_d(const SlDev& d, size_t e, const double4_32a& si,
                                                   const double4_32a& sj) {
  const size_t P = (size_t)d.max_ex * (size_t)d.n;
  const double g = d_of(d.exso[e]), dm = d_of(d.exso[P + e]);
  const double ex = d_of(d.exso[2 * P + e]), ey = d_of(d.exso[3 * P + e]), ez = d_of(d.exso[4 * P + e]);
  const double a = ex * sj.x + ey * sj.y + ez * sj.z, b = ex * si.x + ey * si.y + ez * si.z;
  const double c = si.x * sj.x + si.y * sj.y + si.z * sj.z;
  const double X = si.y * sj.z - si.z * sj.y, Y = si.z * sj.x - si.x * sj.z, Z = si.x * sj.y - si.y * sj.x;
  return -g * (a * b - c / 3.0) + dm * (ex * X + ey * Y + ez * Z);
}

}  // namespace
