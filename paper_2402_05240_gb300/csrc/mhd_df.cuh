// mhd_df.cuh -- double-float ("df") numbers: a value is the unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi)/2, giving a 48-bit significand
// computed entirely on the FP32 pipes.
//
// On this GPU the FP32 FMA rate is 58 times the FP64 rate, so the FP64-accurate
// step can run its reconstruction, Riemann solver and edge fields in df while
// the state, the pressure recovery and the update accumulation stay in
// double.  Arithmetic is built from the error-free transformations TwoSum
// (Knuth, TAOCP vol. 2), FastTwoSum and TwoProduct with a fused multiply-add
// (Dekker 1971), combined as in the double-word algorithms analysed by Joldes,
// Muller and Popescu (ACM TOMS 2017): "sloppy" addition (absolute error of
// order u^2 (|x| + |y|), u = 2^-24), multiplication, division and square root
// by one correction step.  The range is that of float (about 1e-38 .. 3e38).
#pragma once

#include <cuda_runtime.h>

namespace mhd {

// keep the float/double overloads visible next to the df ones below
using ::fabs;
using ::fmax;
using ::fmin;

// Conversions between double and df.  On this GPU the float<->double
// conversion instructions issue at the FP64 rate, so both directions are done
// on the bit patterns with integer and FP32 instructions; only the final
// hi + lo of df -> double is an FP64 addition.

// exact float -> double of a finite float, subnormals flushed to (signed) zero;
// Inf and NaN keep their class
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned s = u & 0x80000000u;
  const unsigned m = u & 0x7fffffu;
  const unsigned ed = e == 0u ? 0u : (e == 0xffu ? 0x7ffu : e + 896u);  // rebias 127 -> 1023
  const unsigned mh = e == 0u ? 0u : (m >> 3);
  const unsigned ml = e == 0u ? 0u : (m << 29);
  const unsigned long long b = ((unsigned long long)(s | (ed << 20) | mh) << 32) | ml;
  return __longlong_as_double((long long)b);
}

// double -> float, rounded to nearest even, on the bit pattern (integer
// instructions only): exact IEEE rounding for results in the normal float
// range; results below 2^-126 flush to a signed zero, overflow gives an
// infinity and NaN stays NaN.
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const unsigned eb = (hw >> 20) & 0x7ffu;
  const unsigned s = hw & 0x80000000u;
  const unsigned m = ((hw & 0xfffffu) << 3) | (lw >> 29);  // kept 23 bits
  const unsigned r = lw & 0x1fffffffu;                     // dropped 29 bits
  unsigned v = ((eb - 896u) << 23) | m;
  // a carry out of the significand raises the exponent (to infinity at the top)
  v += (r > 0x10000000u || (r == 0x10000000u && (m & 1u))) ? 1u : 0u;
  v = eb < 897u ? 0u : v;
  const unsigned nan = (eb == 0x7ffu && ((hw & 0xfffffu) | lw)) ? 0x7fc00000u : 0x7f800000u;
  v = eb > 1150u ? nan : v;
  return __uint_as_float(s | v);
}

struct df;
__device__ __forceinline__ df df_from_double(double x);

struct __align__(8) df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ df(double x);
  __device__ __forceinline__ df(float x) : hi(x), lo(0.0f) {}
  __device__ __forceinline__ df(int x) : hi((float)x), lo(0.0f) {}
  __device__ __forceinline__ explicit operator double() const { return f2d_bits(hi) + f2d_bits(lo); }
};

// double -> df, integer and FP32 instructions only (no branch: a cold path
// with conversion instructions would be if-converted and still occupy the
// FP64 pipe).  For 2^-80 <= |x| < 2^128: hi = x with its significand cut to
// 24 bits (exact), lo = the remaining 29 bits rounded to 23 bits, via the
// 2^23 magic-number conversion, times 2^(e-46); |lo| < ulp(hi) and
// |x - (hi + lo)| <= 2^-47 |x|.  For 2^-126 <= |x| < 2^-80, lo = 0 (absolute
// error below 2^-103); smaller |x| gives a signed zero, |x| >= 2^128 an
// infinity and NaN a NaN.
__device__ __forceinline__ df df_from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const unsigned eb = (hw >> 20) & 0x7ffu;  // biased exponent
  const unsigned s = hw & 0x80000000u;
  const unsigned sig = ((hw & 0xfffffu) << 3) | (lw >> 29);  // top 23 stored significand bits
  unsigned hb = s | ((eb - 896u) << 23) | sig;
  hb = eb < 897u ? s : hb;
  const unsigned big = s | 0x7f800000u | ((eb == 0x7ffu && ((hw & 0xfffffu) | lw)) ? 0x400000u : 0u);
  hb = eb > 1150u ? big : hb;
  const unsigned r = lw & 0x1fffffffu;  // remainder: r * 2^(E-52), E = eb - 1023
  // (r + 32) >> 6 <= 2^23: ORed into the significand of 2^23 it gives 2^23 + q
  // exactly (q = 2^23 carries into the exponent, giving 2^24 = 2^23 + q too)
  const float q = __uint_as_float(0x4b000000u | ((r + 32u) >> 6)) - 8388608.0f;
  const bool has_lo = eb >= 943u && eb <= 1150u;
  const float sc = __uint_as_float(has_lo ? (eb - 942u) << 23 : 0u);  // 2^(E-46), or 0
  return df(__uint_as_float(hb), __uint_as_float(__float_as_uint(q * sc) ^ s));
}

__device__ __forceinline__ df::df(double x) : df(df_from_double(x)) {}

// s + e = a + b exactly (no ordering assumed)
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float v = s - a;
  const float e = (a - (s - v)) + (b - v);
  return df(s, e);
}
// s + e = a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = a + b;
  return df(s, b - (s - a));
}
// p + e = a * b exactly
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = a * b;
  return df(p, fmaf(a, b, -p));
}

__device__ __forceinline__ df operator+(df x, df y) {
  const df s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ df operator-(df x) { return df(-x.hi, -x.lo); }
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }
__device__ __forceinline__ df operator*(df x, df y) {
  df p = two_prod(x.hi, y.hi);
  float l = fmaf(x.hi, y.lo, p.lo);
  l = fmaf(x.lo, y.hi, l);
  return fast_two_sum(p.hi, l);
}
__device__ __forceinline__ df operator/(df x, df y) {
  // below 2^-100 the reciprocal of the leading float would overflow for
  // subnormal divisors: scale both operands by 2^100 (exact)
  const float sc = fabsf(y.hi) < 7.888609052210118e-31f ? 1.2676506002282294e30f : 1.0f;
  x = df(x.hi * sc, x.lo * sc);
  y = df(y.hi * sc, y.lo * sc);
  const float r = __frcp_rn(y.hi);
  const float q1 = x.hi * r;
  // remainder x - q1 y, formed with an exact product
  const df p = two_prod(q1, y.hi);
  const float rem = ((x.hi - p.hi) - p.lo + x.lo) - q1 * y.lo;
  const float q2 = rem * r;
  return fast_two_sum(q1, q2);
}
__device__ __forceinline__ df& operator+=(df& x, df y) { return x = x + y; }
__device__ __forceinline__ df& operator-=(df& x, df y) { return x = x - y; }
__device__ __forceinline__ df& operator*=(df& x, df y) { return x = x * y; }

__device__ __forceinline__ bool operator<(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(df a, df b) { return b < a; }
__device__ __forceinline__ bool operator<=(df a, df b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(df a, df b) { return !(a < b); }
__device__ __forceinline__ bool operator==(df a, df b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(df a, df b) { return !(a == b); }

__device__ __forceinline__ df fabs(df a) { return a.hi < 0.0f ? -a : a; }
__device__ __forceinline__ df fmin(df a, df b) { return b < a ? b : a; }
__device__ __forceinline__ df fmax(df a, df b) { return a < b ? b : a; }

// square root: s = sqrt(hi), one correction (x - s^2) / (2 s)
__device__ __forceinline__ df df_sqrt(df x) {
  if (!(x.hi > 0.0f)) return df(0.0f, 0.0f);
  const float s = sqrtf(x.hi);
  const df p = two_prod(s, s);
  const float c = ((x.hi - p.hi) - p.lo + x.lo) * (0.5f / s);
  return fast_two_sum(s, c);
}

// 1/sqrt(x): r = rsqrt(hi), one Newton step r + r (1 - x r^2) / 2 in df;
// the residual is formed as (x r) r, which stays near 1, so r^2 never
// overflows for tiny x
__device__ __forceinline__ df df_rsqrt(df x) {
  const float r = rsqrtf(x.hi);
  const df rr(r, 0.0f);
  const df e = df(1.0f) - (x * rr) * rr;
  return rr + df(0.5f * r, 0.0f) * e;
}

}  // namespace mhd
