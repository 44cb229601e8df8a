// Double-word arithmetic and FP64 <-> float conversions that stay off the FP64 pipe.
//
// B300 issues FP64 at 1/64 of the FP32 rate, and its float <-> double conversions
// queue on the same narrow path, so code outside FP64 mode keeps FP64-level accuracy
// with pairs of floats (a value is the unevaluated sum h + l, |l| <= ulp(h), about 48
// significant bits) and moves between double and float pairs with integer operations
// on the IEEE-754 encodings (binary64: 1 sign, 11 exponent bits biased by 1023, 52
// fraction bits; binary32: 1, 8 biased by 127, 23).
//
// Products take the exact remainder of h_a h_b from a fused multiply-add (Dekker's
// product); sums take the exact error of h_a + h_b from Knuth's TwoSum and renormalise
// (the double-word algorithms analysed by Joldes, Muller and Popescu, ACM TOMS 44,
// 2017).  The _rn intrinsics keep the compiler from contracting a product into the
// following sum, which would lose the remainder.
#pragma once
#include <cstdint>

namespace pta {

__device__ __forceinline__ float2 dw_renorm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ float2 dw_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float q = __fmaf_rn(a.x, b.x, -p);
  q = __fmaf_rn(a.x, b.y, q);
  q = __fmaf_rn(a.y, b.x, q);
  return dw_renorm(p, q);
}
// a b for a float b
__device__ __forceinline__ float2 dw_mulf(float2 a, float b) {
  const float p = __fmul_rn(a.x, b);
  float q = __fmaf_rn(a.x, b, -p);
  q = __fmaf_rn(a.y, b, q);
  return dw_renorm(p, q);
}
// c - a b
__device__ __forceinline__ float2 dw_fms(float2 c, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float q = __fmaf_rn(a.x, b.x, -p);
  q = __fmaf_rn(a.x, b.y, q);
  q = __fmaf_rn(a.y, b.x, q);
  const float s = __fsub_rn(c.x, p);
  const float t = __fsub_rn(s, c.x);
  float e = __fsub_rn(__fsub_rn(c.x, __fsub_rn(s, t)), __fadd_rn(p, t));  // (c.x - p) - s exactly
  e = __fadd_rn(e, __fsub_rn(c.y, q));
  return dw_renorm(s, e);
}
__device__ __forceinline__ float2 dw_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float t = __fsub_rn(s, a.x);
  float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, t)), __fsub_rn(b.x, t));
  e = __fadd_rn(e, __fadd_rn(a.y, b.y));
  return dw_renorm(s, e);
}
// a + b for a float b
__device__ __forceinline__ float2 dw_addf(float2 a, float b) {
  const float s = __fadd_rn(a.x, b);
  const float t = __fsub_rn(s, a.x);
  float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, t)), __fsub_rn(b, t));
  e = __fadd_rn(e, a.y);
  return dw_renorm(s, e);
}
__device__ __forceinline__ float2 dw_neg(float2 a) { return make_float2(-a.x, -a.y); }
// 1 / d for d > 0: one Newton step from the correctly rounded float reciprocal
// (relative error ~2^-47: the step squares the float's 2^-24)
__device__ __forceinline__ float2 dw_recip(float2 d) {
  const float r = __frcp_rn(d.x);
  float e = __fmaf_rn(-d.x, r, 1.0f);  // exact: |1 - d.x r| < 2^-23 has at most 24 significant bits
  e = __fmaf_rn(-d.y, r, e);
  return dw_renorm(r, __fmul_rn(r, e));
}

// sqrt(d) for d > 0: the float reciprocal square root refined once in FP32, then one
// Newton correction s0 + (d - s0^2) / (2 s0) with d - s0^2 formed in double words
// (relative error ~2^-45)
__device__ __forceinline__ float2 dw_sqrt(float2 d) {
  float y = rsqrtf(d.x);
  y = __fmul_rn(y, __fmaf_rn(__fmul_rn(-0.5f * d.x, y), y, 1.5f));
  const float s0 = __fmul_rn(d.x, y);
  const float2 e = dw_fms(d, make_float2(s0, 0.0f), make_float2(s0, 0.0f));
  return dw_addf(make_float2(s0, 0.0f), __fmul_rn(__fmul_rn(e.x, y), 0.5f));
}

// Exact float -> double: the exponent rebias 127 -> 1023 and the 23-bit fraction moved
// to the top of the 52-bit one; zero and subnormals give 0, infinities and NaNs keep
// their class.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f), e = (u >> 23) & 0xffu;
  const unsigned ef = (e == 0xffu) ? 0x7ffu : e + 896u;
  const unsigned hi = (u & 0x80000000u) | (ef << 20) | ((u & 0x7fffffu) >> 3);
  return (e == 0u) ? 0.0 : __hiloint2double((int)hi, (int)(u << 29));
}
__device__ __forceinline__ double dw2d(float2 v) { return f2d_bits(v.x) + f2d_bits(v.y); }

// double -> float pair without the FP64 pipe: h is v truncated to 24 significant bits
// (the top 23 fraction bits), l the remaining 29 fraction bits truncated to 24, so
// |v - (h + l)| < 2^-47 |v| and |l| < ulp(h).  |v| below 2^-126 gives (0, 0); parts
// of l below the float normal range are dropped (relative error then < 2^-24 |l|
// only while |v| >= 2^-74); |v| >= 2^128 gives an infinite h.
__device__ __forceinline__ float2 d2dw_bits(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned whi = (unsigned)(u >> 32), wlo = (unsigned)u;
  const int e = (int)((whi >> 20) & 0x7ffu);
  const unsigned sgn = whi & 0x80000000u;
  if (e < 897) return make_float2(0.0f, 0.0f);
  if (e > 1150) return make_float2(__uint_as_float(sgn | 0x7f800000u), 0.0f);
  const float h = __uint_as_float(sgn | ((unsigned)(e - 896) << 23) | ((whi & 0xfffffu) << 3) | (wlo >> 29));
  const unsigned R = wlo & 0x1fffffffu;  // l = R 2^(e - 1075)
  if (R == 0u) return make_float2(h, 0.0f);
  const int n = 31 - __clz((int)R);      // leading one of R, 0 .. 28
  const int el = n + e - 948;            // biased float exponent of l
  if (el < 1) return make_float2(h, 0.0f);
  const unsigned mant = (n >= 23 ? (R >> (n - 23)) : (R << (23 - n))) & 0x7fffffu;
  return make_float2(h, __uint_as_float(sgn | ((unsigned)el << 23) | mant));
}
// v truncated to a float (the h of d2dw_bits): |v| - |h| < 2^-23 |v|, sign kept
__device__ __forceinline__ float d2f_trunc(double v) { return d2dw_bits(v).x; }

// v 2^m by the exponent field (v normal and the result in range)
__device__ __forceinline__ double ldexp_bits(double v, int m) {
  return v == 0.0 ? 0.0 : __longlong_as_double(__double_as_longlong(v) + ((long long)m << 52));
}

// 2^(j/16), j = 0..15, as the nearest float pairs
static __constant__ float2 kExp2Sixteenth[16] = {
    {0x1p+0f, 0.0f},                       {0x1.0b5586p+0f, 0x1.9f3122p-25f},  {0x1.172b84p+0f, -0x1.c15742p-27f},
    {0x1.2387a6p+0f, 0x1.ceac48p-25f},     {0x1.306fep+0f, 0x1.4636e2p-25f},   {0x1.3dea64p+0f, 0x1.824684p-25f},
    {0x1.4bfdaep+0f, -0x1.593abcp-25f},    {0x1.5ab07ep+0f, -0x1.5bd5ecp-27f}, {0x1.6a09e6p+0f, 0x1.9fcef4p-26f},
    {0x1.7a1148p+0f, -0x1.829fd0p-25f},    {0x1.8ace54p+0f, 0x1.15506ep-27f},  {0x1.9c4918p+0f, 0x1.51f848p-27f},
    {0x1.ae89fap+0f, -0x1.a94b14p-26f},    {0x1.c199bep+0f, -0x1.3d56b2p-27f}, {0x1.d5818ep+0f, -0x1.822dbcp-27f},
    {0x1.ea4afap+0f, 0x1.52486cp-27f}};

// exp(a) for a double word a, |a| < 170, as a double word and a power of two:
// exp(a) = 2^m (h + l).  Cody-Waite reduction a = n ln2/16 + r with ln2/16 split into
// C1 + C2 + C3 (12, 12 and 24 significant bits, so n C1 and n C2 are exact for |n| <
// 2^12, that is |a| < 177, and a.h - n C1 is exact by Sterbenz's lemma), |r| <= ~ln2/32;
// exp(r) - 1 by its Taylor series to r^6 (truncation < 2^-50), the three highest terms in
// FP32; then the table entry 2^(j/16), j = n mod 16, m = floor(n / 16).  Relative error
// < 2^-45.
// The constants are the float pairs nearest ln2/16, 16/ln2, 2^(j/16), 1/6, 1/24,
// 1/120 and 1/720.
__device__ __forceinline__ float2 dw_exp(float2 a, int& m) {
  constexpr float kC1 = 0x1.62ep-5f, kC2 = 0x1.0cp-19f, kC3 = -0x1.05c61p-33f, kInv = 0x1.715476p+4f;
  const float nf = rintf(__fmul_rn(a.x, kInv));
  const int n = (int)nf;
  const float t = __fsub_rn(a.x, __fmul_rn(nf, kC1));
  float2 r = dw_addf(make_float2(t, 0.0f), a.y);
  r = dw_addf(r, -__fmul_rn(nf, kC2));
  r = dw_addf(r, -__fmul_rn(nf, kC3));
  const float tail = __fmaf_rn(__fmaf_rn(r.x, 0x1.6c16c2p-10f, 0x1.111112p-7f), r.x, 0x1.555556p-5f);
  float2 p = dw_add(make_float2(0x1.555556p-3f, -0x1.555556p-28f), dw_mulf(r, tail));  // 1/6 + r tail
  p = dw_addf(dw_mul(r, p), 0.5f);                                                     // 1/2 + r p
  const float2 em1 = dw_add(r, dw_mul(r, dw_mul(r, p)));                               // exp(r) - 1
  const int j = n & 15;
  m = n >> 4;  // floor(n / 16)
  const float2 T = kExp2Sixteenth[j];
  return dw_add(T, dw_mul(T, em1));
}
// exp of a double word, as a double (the FP64 exponential outside |a| < 170, where the
// reduction above stops being exact; NaN propagates)
__device__ __forceinline__ double dw_exp_d(float2 a) {
  if (!(fabsf(a.x) < 170.0f)) return exp(f2d_bits(a.x) + f2d_bits(a.y));
  int m;
  const float2 v = dw_exp(a, m);
  return ldexp_bits(dw2d(v), m);
}

}  // namespace pta
