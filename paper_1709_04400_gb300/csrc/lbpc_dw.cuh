// Double-word ("DF64") arithmetic on pairs of binary32 numbers.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2, which carries a
// 48-bit significand (relative precision about 2^-48 = 3.6e-15) in the binary32 exponent range. On
// GB300 the FP32 pipes issue 64 times as many operations per clock as the FP64 pipe, so a coupled
// step evaluated in double-word arithmetic runs several times faster than the same step in binary64.
// It still tracks a binary64 result to about 1e-14 per operation.
//
// The building blocks are the classical error-free transformations:
//   TwoSum     s + e = a + b exactly, any a, b (Knuth, TAOCP vol. 2, 4.2.2; Moller 1965)
//   Fast2Sum   s + e = a + b exactly when exponent(a) >= exponent(b) (Dekker 1971)
//   2Prod      p + e = a * b exactly, with one fused multiply-add
// and the double-word algorithms analysed by Joldes, Muller and Popescu, "Tight and rigorous error
// bounds for basic building blocks of double-word arithmetic", ACM TOMS 44(2), 2017:
//   addition   TwoSum of the high words plus the low words, without the final renormalisation of
//              their "sloppy" DW + DW: error below a few 2^-48 (|x| + |y|), i.e. bounded relative to
//              the operands as binary64 rounding is, not relative to a cancelling result
//   product    DW x DW with FMA (their DWTimesDW2): relative error below 5 * 2^-48
//   division   binary32 quotient corrected once by the exactly computed remainder (Dekker 1971)
//   sqrt       binary32 root corrected once by the exactly computed residual (Karp & Markstein 1997)
//   rsqrt      reciprocal of the correctly rounded binary32 root, one Newton step on 1 - x r^2
// Every operation uses the round-to-nearest intrinsics (__fadd_rn, __fmul_rn, __fmaf_rn), which the
// compiler neither contracts nor reorders, so the error-free transformations stay exact.
#pragma once

#include <cuda_runtime.h>

namespace lbpc {

struct __align__(8) dw {
  float hi, lo;
  dw() = default;
  __host__ __device__ constexpr dw(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr explicit dw(float f) : hi(f), lo(0.0f) {}
  __host__ __device__ constexpr explicit dw(int i) : hi((float)i), lo(0.0f) {}  // exact for |i| < 2^24
  // nearest binary32 and the nearest binary32 of the remainder, which is exact in binary64
  __host__ __device__ constexpr explicit dw(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// the binary32 / binary64 overloads stay visible beside the double-word ones below
using ::fmax;
using ::isfinite;
using ::rsqrt;
using ::sqrt;

template <class S> struct is_dw_t { static constexpr bool value = false; };
template <> struct is_dw_t<dw> { static constexpr bool value = true; };

__device__ __forceinline__ dw dw_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
  return dw(s, e);
}

__device__ __forceinline__ dw dw_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dw(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dw dw_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return dw(p, __fmaf_rn(a, b, -p));
}

// Renormalise a pair so that |lo| <= ulp(hi)/2 (TwoSum, exact for any hi, lo).
__device__ __forceinline__ dw dw_norm(dw x) { return dw_two_sum(x.hi, x.lo); }

// Addition without the final renormalisation: TwoSum of the high words plus the low words. The pair
// it returns may have |lo| a few ulp(hi) (after cancellation, more); its absolute error, like that of
// the normalised "sloppy" sum, stays within a few 2^-48 (|x| + |y|). Products take such pairs as they
// are; division, roots, comparisons and checks renormalise first.
__device__ __forceinline__ dw operator+(dw x, dw y) {
  const dw s = dw_two_sum(x.hi, y.hi);
  return dw(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dw operator-(dw x) { return dw(-x.hi, -x.lo); }
__device__ __forceinline__ dw operator-(dw x, dw y) { return x + (-y); }

// Product: 2Prod of the high words plus the cross terms, renormalised (Fast2Sum). The renormalisation
// is kept here: leaving products unnormalised as well was measured to lose accuracy (5e-10 against
// a binary64 evaluation after 200 coupled steps, against 3e-13 with it).
__device__ __forceinline__ dw operator*(dw x, dw y) {
  const dw c = dw_two_prod(x.hi, y.hi);
  const float t = __fmaf_rn(x.lo, y.hi, __fmul_rn(x.hi, y.lo));
  return dw_fast_two_sum(c.hi, __fadd_rn(c.lo, t));
}

// x * c for a binary32 constant c (2, 3, 0.5, ...). A power of two scales both words exactly;
// otherwise 2Prod of the high word plus c x.lo (DW x FP). The power-of-two test folds away once the
// constant is inlined.
__device__ __forceinline__ dw operator*(dw x, float c) {
  if ((__float_as_uint(c) & 0x007fffffu) == 0u && c != 0.0f) return dw(__fmul_rn(x.hi, c), __fmul_rn(x.lo, c));
  const dw p = dw_two_prod(x.hi, c);
  return dw_fast_two_sum(p.hi, __fmaf_rn(x.lo, c, p.lo));
}
__device__ __forceinline__ dw operator*(float c, dw x) { return x * c; }
__device__ __forceinline__ dw operator*(dw x, int c) { return x * (float)c; }  // |c| < 2^24

__device__ __forceinline__ dw operator/(dw x, dw y) {
  x = dw_norm(x);
  y = dw_norm(y);
  const float r = __frcp_rn(y.hi);
  const float q1 = __fmul_rn(x.hi, r);
  // remainder x - q1 y: q1 y.hi exactly by 2Prod, q1 y.lo to binary32 precision
  const dw p = dw_two_prod(q1, y.hi);
  const float d = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p.hi), p.lo), __fsub_rn(x.lo, __fmul_rn(q1, y.lo)));
  return dw_fast_two_sum(q1, __fmul_rn(d, r));
}

__device__ __forceinline__ dw& operator+=(dw& a, dw b) { return a = a + b; }
__device__ __forceinline__ dw& operator-=(dw& a, dw b) { return a = a - b; }
__device__ __forceinline__ dw& operator*=(dw& a, dw b) { return a = a * b; }

// comparisons of normalised pairs: the sign of the difference
__device__ __forceinline__ bool dw_lt(dw a, dw b) {
  a = dw_norm(a);
  b = dw_norm(b);
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ bool dw_le(dw a, dw b) {
  a = dw_norm(a);
  b = dw_norm(b);
  return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo);
}
__device__ __forceinline__ bool operator<(dw a, dw b) { return dw_lt(a, b); }
__device__ __forceinline__ bool operator>(dw a, dw b) { return dw_lt(b, a); }
__device__ __forceinline__ bool operator<=(dw a, dw b) { return dw_le(a, b); }
__device__ __forceinline__ bool operator>=(dw a, dw b) { return dw_le(b, a); }

__device__ __forceinline__ bool isfinite(dw a) { return ::isfinite(a.hi) && ::isfinite(a.lo); }

// larger of a and b; a NaN operand yields the other one, as fmax does
__device__ __forceinline__ dw fmax(dw a, dw b) {
  if (::isnan(a.hi) || ::isnan(a.lo)) return b;
  if (::isnan(b.hi) || ::isnan(b.lo)) return a;
  return a < b ? dw_norm(b) : dw_norm(a);
}

__device__ __forceinline__ dw sqrt(dw x) {
  x = dw_norm(x);
  if (!(x.hi > 0.0f)) return dw(::sqrtf(x.hi), 0.0f);  // zero, negative (NaN) or NaN
  const float s = __fsqrt_rn(x.hi);
  const dw p = dw_two_prod(s, s);
  const float d = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p.hi), p.lo), x.lo);  // x - s^2
  return dw_fast_two_sum(s, __fmul_rn(d, __fmul_rn(0.5f, __frcp_rn(s))));
}

__device__ __forceinline__ dw rsqrt(dw x) {
  x = dw_norm(x);
  const float r = __frcp_rn(__fsqrt_rn(x.hi));
  const dw e = dw(1) - x * dw_two_prod(r, r);  // 1 - x r^2, small; both words count (e is not normalised)
  return dw_fast_two_sum(r, __fmul_rn(__fmul_rn(0.5f, r), __fadd_rn(e.hi, e.lo)));
}

// read-only load of a plane value in any arithmetic type
template <class T> __device__ __forceinline__ T ldgv(const T* p) { return __ldg(p); }
template <> __device__ __forceinline__ dw ldgv<dw>(const dw* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return dw(v.x, v.y);
}

}  // namespace lbpc
