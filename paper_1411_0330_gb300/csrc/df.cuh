// df.cuh -- double-float arithmetic: a value is the unevaluated sum h + l of
// two FP32 numbers with |l| <= ulp(h) / 2, 48 significant bits (unit roundoff
// about 2^-48 = 3.6e-15).  The operations are the error-free transformations
// of Knuth (TwoSum, 1969), Dekker (FastTwoSum, 1971) and the FMA form of
// TwoProduct, combined as in Dekker's double-length arithmetic:
//   a + b:  (s, e) = TwoSum(a.h, b.h); e += a.l + b.l; FastTwoSum(s, e)
//   a * b:  p = a.h b.h; e = fma(a.h, b.h, -p) + a.h b.l + a.l b.h; FastTwoSum(p, e)
// The addition's error is bounded by a small multiple of 2^-48 (|a| + |b|),
// which is what the normwise error analysis of an FFT asks for.  Every step
// uses the _rn intrinsics, so the compiler neither contracts nor reassociates
// them.  On GB300 the FP32 pipes issue 64 times the FP64 rate, so a
// double-float operation costs a fraction of a native FP64 one.
#pragma once

#include "common.cuh"

namespace lsh {

struct __align__(8) DF {
  float h, l;
  DF() = default;
  __host__ __device__ constexpr DF(float hi, float lo) : h(hi), l(lo) {}
  __host__ __device__ constexpr DF(double d) : h((float)d), l((float)(d - (double)(float)d)) {}
  __host__ __device__ constexpr DF(int i) : DF((double)i) {}
};

struct __align__(16) DF2 {
  DF x, y;
};
template <> struct cplx_of<DF> { typedef DF2 type; };

template <typename T> struct is_df { static constexpr bool value = false; };
template <> struct is_df<DF> { static constexpr bool value = true; };

// s + e with |e| <= ulp(s) / 2 when |a| >= |b| (or a = 0)
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return DF(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ DF operator+(DF a, DF b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bv = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bv)), __fsub_rn(b.h, bv));
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  return df_fast_two_sum(s, e);
}
__device__ __forceinline__ DF operator-(DF a) { return DF(-a.h, -a.l); }
__device__ __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }
__device__ __forceinline__ DF operator*(DF a, DF b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ DF& operator+=(DF& a, DF b) { return a = a + b; }
__device__ __forceinline__ DF& operator-=(DF& a, DF b) { return a = a - b; }
__device__ __forceinline__ DF& operator*=(DF& a, DF b) { return a = a * b; }

// exact scalings by powers of two
__device__ __forceinline__ DF df_scale2(DF a, float p2) { return DF(__fmul_rn(a.h, p2), __fmul_rn(a.l, p2)); }

// double -> double-float with integer operations only (the FP64 pipe is the
// scarce unit): h = d with its significand cut to 24 bits, l = the remaining
// 29 bits rounded to FP32 (together within 2^-48 |d|).  |d| < 2^-126 maps to
// 0, the low part of |d| < 2^-74 to 0 (below 2^-98 in absolute terms).
__device__ __forceinline__ DF df_split(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const int ef = e - 896;  // FP32 exponent field: e - 1023 + 127
  const unsigned sign = hi & 0x80000000u;
  if (ef <= 0) return DF(0.f, 0.f);
  if (ef >= 255) return DF(__uint_as_float(sign | 0x7f800000u), 0.f);
  const float h = __uint_as_float(sign | ((unsigned)ef << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
  float l = 0.f;
  if (e >= 949) l = __fmul_rn(__uint2float_rn(lo & 0x1fffffffu), __uint_as_float((unsigned)(e - 948) << 23));
  return DF(h, sign ? -l : l);
}

// conversions through the FP64 pipe (one FP64 operation each)
__device__ __forceinline__ DF df_from(double d) {
  const float h = __double2float_rn(d);
  return DF(h, __double2float_rn(d - (double)h));
}
__device__ __forceinline__ double df_to(DF a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ DF2 df2_from(double2 d) {
  DF2 r;
  r.x = df_from(d.x);
  r.y = df_from(d.y);
  return r;
}

}  // namespace lsh
