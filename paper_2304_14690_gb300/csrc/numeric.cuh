// Conversions between FP64 and FP32 (pairs) done with integer operations on the IEEE-754
// encodings, so that the FP64 pipe (about 1/60 of the FP32 rate on this GPU) is left to the
// arithmetic that needs it. Each routine falls back to the hardware conversion outside the
// FP32 normal range (zero, subnormal, huge, inf, nan), where it is not on a hot path.
#pragma once

#include <cuda_runtime.h>

namespace pc {

// Out-of-line slow paths, so that the compiler cannot if-convert them into every call (their
// FP64 conversions would then run predicated for all elements on the slow FP64 pipe).
static __device__ __noinline__ double f2d_slow(float f) { return (double)f; }
static __device__ __noinline__ float2 split_slow(double v) {
  float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}
static __device__ __noinline__ float d2f_slow(double v) { return (float)v; }

// Exact float -> double.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return f2d_slow(f);
  const unsigned long long b = ((unsigned long long)(u >> 31) << 63) |
                               ((unsigned long long)(e - 127u + 1023u) << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)b);
}

// Split v into an unevaluated pair hi + lo with |v - hi - lo| < 2^-46 |v|: hi keeps the leading
// 24 significand bits of v (truncation), lo the leading 24 bits of the 29-bit remainder.
__device__ __forceinline__ void split_f64(double v, float &hi, float &lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  if (e < -74 || e > 127) {
    const float2 r = split_slow(v);
    hi = r.x;
    lo = r.y;
    return;
  }
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const unsigned long long mant = b & 0xfffffffffffffULL;
  hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)(mant >> 29));
  const unsigned rm = (unsigned)(mant & 0x1fffffffULL);   // remainder in units of 2^(e-52)
  if (rm == 0u) {
    lo = 0.0f;
    return;
  }
  const int lz = __clz(rm);                 // >= 3
  const int p = 31 - lz;                    // position of the leading one
  // 23 bits after the leading one (truncated); 64-bit shift so lz = 31 is well defined
  const unsigned frac = (unsigned)((((unsigned long long)rm) << (lz + 1)) >> 9) & 0x7fffffu;
  const int be = p + e - 52 + 127;          // biased exponent of lo, >= 1 for e >= -74
  lo = __uint_as_float(sign | ((unsigned)be << 23) | frac);
}

// double -> float, rounding toward zero (the hi part of split_f64).
__device__ __forceinline__ float d2f_rz_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  if (e < -126 || e > 127) return d2f_slow(v);
  return __uint_as_float(((unsigned)(b >> 63) << 31) | ((unsigned)(e + 127) << 23) |
                         (unsigned)((b & 0xfffffffffffffULL) >> 29));
}

// An FP64 value as an unevaluated FP32 pair (hi, lo).
__device__ __forceinline__ float2 as_pair(double v) {
  float hi, lo;
  split_f64(v, hi, lo);
  return make_float2(hi, lo);
}
__device__ __forceinline__ float2 as_pair(float v) { return make_float2(v, 0.0f); }

// Compensated dot product in FP32 arithmetic: (w.x + w.y) . (u.x + u.y) accumulated as an
// unevaluated pair; products by TwoProduct (fma), sums by TwoSum.
struct DF { float hi, lo; };
__device__ __forceinline__ void df_acc(DF &s, float2 w, float2 u) {
  float p = w.x * u.x;
  float e = fmaf(w.x, u.x, -p);
  e = fmaf(w.x, u.y, e);
  e = fmaf(w.y, u.x, e);
  float t = s.hi + p;
  float z = t - s.hi;
  float err = (s.hi - (t - z)) + (p - z);
  s.hi = t;
  s.lo += err + e;
}
__device__ __forceinline__ double df_value(DF s) { return f2d_bits(s.hi) + f2d_bits(s.lo); }

}  // namespace pc
