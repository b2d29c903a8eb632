// Float-pair ("double-float") arithmetic for float64 transforms without the
// FP64 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2:
// 48 significand bits, the float exponent range.  The operations are the
// classical error-free transformations built from float additions and fused
// multiply-adds (Dekker 1971; Knuth's TwoSum; Joldes, Muller and Popescu,
// "Tight and rigorous error bounds for basic building blocks of double-word
// arithmetic", ACM TOMS 2017):
//   two_sum(a, b)       s + e = a + b exactly              (6 float ops)
//   fast_two_sum(a, b)  the same when |a| >= |b|           (3 float ops)
//   a + b               two_sum of the high parts, the low parts added to the
//                       error, renormalised: |error| <= 2^-47 (|a| + |b|)
//                       (no relative bound under cancellation, but the
//                       normwise bound an FFT's error analysis needs)
//   a * b               exact product of the high parts by FMA, the cross
//                       terms added by FMA, renormalised (relative error
//                       below 2^-46)
// GB300 runs FP32 at about 64 times its FP64 rate, so a float64 FFT in this
// arithmetic (about ten float operations per float64 operation) is faster
// than on the FP64 pipe.  Accuracy: about 2^-47 per operation instead of
// 2^-53, which keeps a transform inside the float64 accuracy bar
// (5e-15 log2 N relative L2); inputs beyond the float exponent range
// (|x| above 2^127 or below 2^-100) are not representable.
#pragma once

#include <cuda_runtime.h>

namespace tf {

struct dd {
  float hi, lo;
  __host__ __device__ constexpr dd() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  // nearest float and the nearest float of the remainder
  __host__ __device__ constexpr explicit dd(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ constexpr dd(int v) : hi((float)v), lo(0.f) {}
};

struct __align__(16) cdd {
  dd x, y;
};

__device__ __forceinline__ dd dd_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dd(s, e);
}
__device__ __forceinline__ dd dd_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dd(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dd operator+(dd a, dd b) {
  const dd s = dd_two_sum(a.hi, b.hi);
  return dd_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__device__ __forceinline__ dd operator*(dd a, dd b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dd_fast_two_sum(p, e);
}
__device__ __forceinline__ bool operator!=(dd a, dd b) { return a.hi != b.hi || a.lo != b.lo; }

// float64 -> float pair by integer operations (no FP64 instruction): hi
// holds the top 24 significand bits of v (truncated), lo the remaining 29
// bits rounded to a float (relative error of the pair below 2^-47).  Values
// whose pair would leave the normal float range (|v| < 2^-74, |v| >= 2^127,
// zero, subnormal, infinite or NaN) take the float64 conversion.
__device__ __forceinline__ dd dd_from_double(double v) {
  const int whi = __double2hiint(v);
  const unsigned wlo = (unsigned)__double2loint(v);
  const int ex = (whi >> 20) & 0x7FF;
  if (ex < 949 || ex > 1150) {
    const float h = __double2float_rn(v);
    return dd(h, isfinite(h) ? __double2float_rn(v - (double)h) : 0.f);
  }
  const unsigned sign = (unsigned)whi & 0x80000000u;
  const unsigned m_hi = (((unsigned)whi & 0xFFFFFu) << 3) | (wlo >> 29);  // top 23 explicit bits
  const float h = __uint_as_float(sign | ((unsigned)(ex - 896) << 23) | m_hi);
  // remainder r * 2^(ex - 1075), r < 2^29; the scale is a normal float power of two
  const float scale = __uint_as_float((unsigned)(ex - 1075 + 127) << 23);
  const float l = __int2float_rn((int)(wlo & 0x1FFFFFFFu)) * scale;
  return dd_fast_two_sum(h, __uint_as_float(__float_as_uint(l) | sign));  // |lo| <= ulp(hi) / 2
}
// float -> float64 by integer operations (exact; a subnormal float, which only
// a low part can be, becomes zero: below 2^-126, far under the pair's error)
__device__ __forceinline__ double dd_widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned sign = u & 0x80000000u;
  if (e == 0) return __hiloint2double((int)sign, 0);
  const unsigned de = (e == 0xFFu) ? 0x7FFu : e + 896u;
  const unsigned m = u & 0x7FFFFFu;
  return __hiloint2double((int)(sign | (de << 20) | (m >> 3)), (int)(m << 29));
}
// float pair -> float64: one float64 addition of the exactly widened parts
__device__ __forceinline__ double dd_to_double(dd a) { return dd_widen(a.hi) + dd_widen(a.lo); }

__device__ __forceinline__ cdd cdd_from(double2 v) { return cdd{dd_from_double(v.x), dd_from_double(v.y)}; }
__device__ __forceinline__ double2 cdd_to(cdd v) { return make_double2(dd_to_double(v.x), dd_to_double(v.y)); }

}  // namespace tf
