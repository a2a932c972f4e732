// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi), giving a ~48-bit significand on the FP32
// pipes (GB300 issues FP32 at 64x the FP64 rate).  Built from the classical
// error-free transformations: Knuth's two-sum, Dekker's fast-two-sum and the
// FMA-based two-product (a*b = p + e exactly with e = fma(a, b, -p)).
// Every operation uses explicit round-to-nearest intrinsics so the compiler
// cannot contract or reassociate the compensation terms.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "common.cuh"

namespace fde {

struct df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __device__ explicit df(double x);
  __device__ explicit operator double() const;
  __device__ explicit df(int v) : hi((float)v), lo(0.f) {}
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df(s, e);
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// x + y: two-sum of the leading parts, trailing parts added to the error
__device__ __forceinline__ df operator+(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s.hi, e);
}
__device__ __forceinline__ df operator-(df x) { return df(-x.hi, -x.lo); }
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }
__device__ __forceinline__ df operator*(df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ df& operator+=(df& x, df y) {
  x = x + y;
  return x;
}
// a*b + c*d with both products error-free before the single normalisation
__device__ __forceinline__ df dot2(df a, df b, df c, df d) {
  const float p1 = __fmul_rn(a.hi, b.hi);
  const float e1 = __fmaf_rn(a.hi, b.hi, -p1);
  const float p2 = __fmul_rn(c.hi, d.hi);
  const float e2 = __fmaf_rn(c.hi, d.hi, -p2);
  df s = two_sum(p1, p2);
  float t = __fadd_rn(s.lo, __fadd_rn(e1, e2));
  t = __fmaf_rn(a.hi, b.lo, t);
  t = __fmaf_rn(a.lo, b.hi, t);
  t = __fmaf_rn(c.hi, d.lo, t);
  t = __fmaf_rn(c.lo, d.hi, t);
  return fast_two_sum(s.hi, t);
}

// c + a b: the product error-free (two-product) before one normalisation
__device__ __forceinline__ df df_fma(df a, df b, df c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const df s = two_sum(c.hi, p);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(c.lo, e)));
}

// double -> hi + lo with integer operations only (no FP64 instruction): hi
// keeps the leading 24 significand bits (truncated), lo the next 24 bits
// (rounded).  |hi + lo - x| <= 2^-47 |x| for 2^-73 <= |x| <= 2^100, where lo
// is a normal float; below that lo (then below 2^-97) is dropped and below
// 2^-100 the value flushes to 0, so the error stays under 2^-97 absolutely
// (the callers' data are vectors of norm ~1 and fields of order 1).  Larger
// values and infinities become +-inf and NaN stays NaN, so non-finite data
// stay visible downstream.
__device__ __forceinline__ df df_from_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 63);
  const int E = (int)((b >> 52) & 0x7FF) - 1023;
  if (E > 100) {
    const bool nan = E == 1024 && (b & 0xFFFFFFFFFFFFFull);
    return df(__uint_as_float((sign << 31) | 0x7F800000u | (nan ? 0x400000u : 0u)), 0.f);
  }
  if (E < -100) return df(0.f, 0.f);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;  // 52 bits
  const unsigned hm = (unsigned)(m >> 29);               // top 23 stored bits
  const unsigned hb = (sign << 31) | ((unsigned)(E + 127) << 23) | hm;
  const unsigned rest = (unsigned)(m & 0x1FFFFFFFull);   // low 29 bits
  float lo = 0.f;
  if (rest) {
    // rest * 2^(E - 52); __uint2float_rn rounds 29 -> 24 bits
    const float r = __uint2float_rn(rest);
    const int ebits = (int)((__float_as_uint(r) >> 23) & 0xFF) + (E - 52);
    if (ebits > 0)
      lo = __uint_as_float((sign << 31) | ((unsigned)ebits << 23) |
                           (__float_as_uint(r) & 0x7FFFFF));
  }
  return fast_two_sum(__uint_as_float(hb), lo);
}
// float -> double with integer operations only (GB300 runs FP64 conversions
// at the FP64 rate, 1/64 of FP32): exact for every float, infinities and NaN
// included
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  const unsigned e = (u >> 23) & 0xFF;
  unsigned long long m = u & 0x7FFFFF;
  if (e == 255) return __longlong_as_double((long long)(sign | (0x7FFull << 52) | (m << 29)));
  if (e == 0) {
    if (!m) return __longlong_as_double((long long)sign);
    // subnormal: m 2^-149 with the leading bit at position p
    const int p = 31 - __clz((int)m);
    m = (m << (52 - p)) & 0xFFFFFFFFFFFFFull;
    return __longlong_as_double(
        (long long)(sign | ((unsigned long long)(p - 149 + 1023) << 52) | m));
  }
  return __longlong_as_double(
      (long long)(sign | ((unsigned long long)(e - 127 + 1023) << 52) | (m << 29)));
}
// double -> float, round to nearest even, with integer operations only:
// overflow gives +-inf, results below the normal range are rounded into
// FP32 subnormals (or 0), NaN stays NaN
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const int E = (int)((b >> 52) & 0x7FF) - 1023;
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (E == 1024) return __uint_as_float(sign | 0x7F800000u | (m ? 0x400000u : 0u));
  if (E > 127) return __uint_as_float(sign | 0x7F800000u);
  if (E >= -126) {
    unsigned keep = (unsigned)(m >> 29);
    const unsigned rem = (unsigned)(m & 0x1FFFFFFFull), half = 1u << 28;
    // a carry out of the significand moves into the exponent (up to inf)
    unsigned bits = ((unsigned)(E + 127) << 23) + keep;
    if (rem > half || (rem == half && (keep & 1u))) ++bits;
    return __uint_as_float(sign | bits);
  }
  if (E < -150) return __uint_as_float(sign);
  // subnormal result: the 53-bit significand shifted right by -E - 126 + 29
  const unsigned long long full = m | (1ull << 52);
  const int sh = 29 + (-126 - E);  // 30 .. 53
  const unsigned long long keep = full >> sh;
  const unsigned long long rem = full & ((1ull << sh) - 1), half = 1ull << (sh - 1);
  unsigned bits = (unsigned)keep;
  if (rem > half || (rem == half && (keep & 1ull))) ++bits;
  return __uint_as_float(sign | bits);
}
// element conversions of the FFT passes and the V-cycle's input and output:
// FP32 <-> FP64 through the integer routines above, everything else by value
template <typename To, typename From>
__device__ __forceinline__ To cvt(From v) {
  return To(v);
}
template <>
__device__ __forceinline__ float cvt<float, double>(double v) {
  return d2f_bits(v);
}
template <>
__device__ __forceinline__ double cvt<double, float>(float v) {
  return f2d_bits(v);
}
// double-float <-> FP32: the leading part (|lo| <= ulp(hi) / 2, so hi is
// hi + lo rounded to FP32 but at an exact tie), and an exact widening
template <>
__device__ __forceinline__ float cvt<float, df>(df v) {
  return v.hi;
}
template <>
__device__ __forceinline__ df cvt<df, float>(float v) {
  return df(v, 0.f);
}

__device__ inline df::df(double x) { *this = df_from_bits(x); }
__device__ inline df::operator double() const { return __dadd_rn(f2d_bits(hi), f2d_bits(lo)); }

template <>
__device__ __forceinline__ cx<df> cmul<df>(cx<df> a, cx<df> b) {
  return {dot2(a.re, b.re, -a.im, b.im), dot2(a.re, b.im, a.im, b.re)};
}
template <>
__device__ __forceinline__ cx<df> cmulc<df>(cx<df> a, cx<df> b) {
  return {dot2(a.re, b.re, a.im, b.im), dot2(a.im, b.re, -a.re, b.im)};
}

}  // namespace fde
