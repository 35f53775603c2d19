// Double-float ("df") arithmetic on the FP32 pipe, shared by the double-float filter
// (df.cu) and the double-float dense products (dense.cu).  A value is the unevaluated sum
// hi + lo of two FP32 numbers.  The transforms below are exact only as written: the
// __fadd_rn / __fsub_rn / __fmul_rn intrinsics and their packed FP32x2 forms are never
// contracted into an FMA, so the compiler cannot fuse a product into a later sum.
#pragma once

#include "arb_internal.h"

namespace arb {
namespace {

__device__ __forceinline__ df2 df_from(double x) {
  const float h = __double2float_rn(x);
  return df2{h, __double2float_rn(x - static_cast<double>(h))};
}
// s + e = a + b exactly when |a| >= |b|
__device__ __forceinline__ df2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df2{s, __fsub_rn(b, __fsub_rn(s, a))};
}
// p + e = a.hi * b.hi exactly (e from one FMA), then the cross terms a.hi b.lo + a.lo b.hi
__device__ __forceinline__ df2 df_mul(df2 a, df2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// two double-float values (a lane's two columns): hi parts and lo parts as pairs
struct dfp {
  float2 hi, lo;
};
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ dfp neg(const dfp& a) { return dfp{neg2(a.hi), neg2(a.lo)}; }
__device__ __forceinline__ dfp dfp_of(df2 a, df2 b) { return dfp{make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)}; }
// b - a, exactly rounded, as one packed FMA with the constant -1 (no separate negation)
__device__ __forceinline__ float2 sub2(float2 b, float2 a) { return __ffma2_rn(a, make_float2(-1.f, -1.f), b); }
__device__ __forceinline__ dfp fast_two_sum2(float2 a, float2 b) {
  const float2 s = __fadd2_rn(a, b);
  return dfp{s, sub2(b, sub2(s, a))};
}

// Compensated accumulation (Ogita, Rump & Oishi's Dot2) of c * v into (S, E), for both
// columns at once: S collects the rounded sums of the leading products, E the exact
// rounding errors of those sums (Knuth's two-sum) and of the products (one FMA each) plus
// the cross terms, so S + E carries the dot product as if computed with twice the working
// precision.  nc = -c is passed in so that every subtraction is an FMA with -1 or with
// the negated multiplier: 12 packed instructions per term for two columns.
__device__ __forceinline__ void dot2p(float2& S, float2& E, const dfp& c, const dfp& nc, const dfp& v) {
  const float2 p = __fmul2_rn(c.hi, v.hi);
  float2 en = __ffma2_rn(nc.hi, v.hi, p);  // -(exact rounding error of p)
  en = __ffma2_rn(nc.hi, v.lo, en);
  en = __ffma2_rn(nc.lo, v.hi, en);
  const float2 s = __fadd2_rn(S, p);
  const float2 bb = sub2(s, S);
  const float2 t = __fadd2_rn(sub2(S, sub2(s, bb)), sub2(p, bb));
  S = s;
  E = __fadd2_rn(E, sub2(t, en));
}

// (hi, lo) of a double with hi + lo = x up to 2^-48 |x|, by integer operations on its bits
// (no FP64 instruction): hi keeps the leading 24 significand bits (truncated), lo the next
// bits rounded to 24.  Below |x| ~ 2^-75 lo leaves FP32's normal range and is dropped (hi
// alone, 2^-24 relative), below 2^-126 both are zero - far below any entry of the blocks
// the solver forms; infinities stay infinite and NaNs become NaNs or infinities.
__device__ __forceinline__ void split_f64(double x, float& hi, float& lo) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned sign = static_cast<unsigned>(b >> 63) << 31;
  const int e = static_cast<int>((b >> 52) & 0x7ff);
  const int fe = e - 1023 + 127;
  const unsigned mhi = static_cast<unsigned>((b >> 29) & 0x7fffff);
  if (fe <= 0) {
    hi = 0.f;
    lo = 0.f;
    return;
  }
  if (fe >= 255) {
    hi = __uint_as_float(sign | 0x7f800000u | (e == 0x7ff ? mhi : 0u));
    lo = 0.f;
    return;
  }
  hi = __uint_as_float(sign | (static_cast<unsigned>(fe) << 23) | mhi);
  const unsigned low = static_cast<unsigned>(b & 0x1fffffffull);  // value low * 2^(e - 1075)
  const unsigned lb = __float_as_uint(__uint2float_rn(low));      // exact power-of-two scaling below
  const int le = static_cast<int>(lb >> 23) + e - 1075;          // biased exponent of lo
  lo = (low == 0u || le <= 0) ? 0.f : __uint_as_float(sign | (static_cast<unsigned>(le) << 23) | (lb & 0x7fffffu));
}

}  // namespace
}  // namespace arb
