// lbve_df32.cuh -- float32 pairs ("double-float") for the LBVE_DF32 storage
// precision: a value is hi + lo with |lo| <= ulp(hi)/2, stored as two float32
// (8 bytes, as float64) and computed with error-free float32 transformations
// (Knuth's two-sum, Dekker's product through fmaf), about 48 significant bits.
// GB300 issues a float64 instruction once every 64 cycles per warp; these
// operations run on the float32 pipe, which issues every cycle.
//   add: two-sum of the high parts, the low parts added to its error, a fast
//        two-sum to renormalise (11 float32 operations; error ~2^-48 of the
//        larger operand);
//   mul: exact product of the high parts by fmaf plus the cross terms, left
//        unrenormalised: |lo| stays within about 1.5 ulp(hi), which the
//        two-sum of the next addition absorbs (4 operations instead of 7;
//        10 % off the step on the batched mix);
//   div: a float32 quotient from one reciprocal, refined by one correction step.
#pragma once
#include <cuda_runtime.h>

namespace lbve {

struct df32 {
  float hi, lo;
  __host__ __device__ constexpr df32() : hi(0.f), lo(0.f) {}
  // exact split of a float64 constant (folded at compile time for literals)
  __host__ __device__ constexpr df32(double x)
      : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ constexpr df32(int x) : hi((float)x), lo(0.f) {}
  __host__ __device__ constexpr df32(float h, float l) : hi(h), lo(l) {}
};

__device__ __forceinline__ df32 df_renorm(float s, float e) {
  const float h = s + e;
  return df32(h, e - (h - s));
}

__device__ __forceinline__ df32 operator+(df32 a, df32 b) {
  const float s = a.hi + b.hi, bv = s - a.hi;
  const float e = ((a.hi - (s - bv)) + (b.hi - bv)) + (a.lo + b.lo);
  return df_renorm(s, e);
}
__device__ __forceinline__ df32 operator-(df32 a) { return df32(-a.hi, -a.lo); }
__device__ __forceinline__ df32 operator-(df32 a, df32 b) { return a + (-b); }
__device__ __forceinline__ df32 operator*(df32 a, df32 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df32(p, e);
}
__device__ __forceinline__ df32 operator/(df32 a, df32 b) {
  // one correctly rounded reciprocal serves both quotients; the correction
  // takes the first quotient's extra rounding (about 47 bits in all)
  const float rb = 1.f / b.hi;
  const float q = a.hi * rb;
  const float p = b.hi * q;  // b * q exactly as a pair (b.hi q + b.lo q)
  const df32 bq(p, fmaf(b.lo, q, fmaf(b.hi, q, -p)));
  const df32 r = a - bq;  // remainder
  return df_renorm(q, r.hi * rb);
}
__device__ __forceinline__ df32& operator+=(df32& a, df32 b) { return a = a + b; }

// float64 value of a pair (one float64 addition; used off the hot path)
__device__ __forceinline__ double df_to_f64(df32 a) { return (double)a.hi + (double)a.lo; }

}  // namespace lbve
