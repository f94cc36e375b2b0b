// Double-float arithmetic: a value as the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi)/2, so 48 significand bits on the FP32 pipes
// (the FP64 rate of this part is 1/64 of its FP32 rate).  The operations are
// the error-free transformations of Knuth (two-sum), Dekker (fast two-sum)
// and the FMA form of the exact product, combined as in the accurate
// double-double addition and multiplication of Hida, Li and Bailey (2001):
// relative error of an operation about 2^-46 or better.  Device code only
// computes with these; conversions from and to FP64 happen at the edges.
#pragma once
#include <cmath>

#include "common.cuh"

namespace pwh {

struct df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr df(double d)
      : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ constexpr df(float f) : hi(f), lo(0.f) {}
  __host__ __device__ constexpr df(int i) : hi((float)i), lo(0.f) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// rounded FP32 operations that the compiler may not contract into FMAs
__host__ __device__ __forceinline__ float df_add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
__host__ __device__ __forceinline__ float df_sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
__host__ __device__ __forceinline__ float df_mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
__host__ __device__ __forceinline__ float df_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}

// s + e = a + b exactly (Knuth)
__host__ __device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = df_add(a, b);
  const float bb = df_sub(s, a);
  e = df_add(df_sub(a, df_sub(s, bb)), df_sub(b, bb));
}
// s + e = a + b exactly when |a| >= |b| (Dekker)
__host__ __device__ __forceinline__ void df_fast_two_sum(float a, float b, float& s, float& e) {
  s = df_add(a, b);
  e = df_sub(b, df_sub(s, a));
}

__host__ __device__ __forceinline__ df operator+(df a, df b) {
  float s, e, t, f;
  df_two_sum(a.hi, b.hi, s, e);
  df_two_sum(a.lo, b.lo, t, f);
  e = df_add(e, t);
  df_fast_two_sum(s, e, s, e);
  e = df_add(e, f);
  df_fast_two_sum(s, e, s, e);
  return df(s, e);
}
__host__ __device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__host__ __device__ __forceinline__ df operator*(df a, df b) {
  const float p = df_mul(a.hi, b.hi);
  float e = df_fma(a.hi, b.hi, -p);  // exact low part of a.hi b.hi
  e = df_fma(a.hi, b.lo, e);
  e = df_fma(a.lo, b.hi, e);
  float s;
  df_fast_two_sum(p, e, s, e);
  return df(s, e);
}
__host__ __device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }
__host__ __device__ __forceinline__ df& operator*=(df& a, df b) { return a = a * b; }

struct dfc {
  df x, y;
};
template <> struct cplx<df> { using t = dfc; };

// FP64 -> double-float, the nearest pair (hi the FP32 rounding of the value,
// lo that of the remainder)
__device__ __forceinline__ df df_from(double d) {
  const float h = __double2float_rn(d);
  return df(h, __double2float_rn(d - (double)h));
}

}  // namespace pwh
