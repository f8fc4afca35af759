// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi)/2, giving about 48 significant bits.  Built from the error-free
// transformations of floating-point arithmetic:
//   TwoSum (Knuth): s + e = a + b exactly, any a, b;
//   Fast2Sum (Dekker): s + e = a + b exactly when |a| >= |b|;
//   TwoProd via FMA: p + e = a b exactly (e = fma(a, b, -p)).
// The _rn intrinsics keep the compiler from contracting or reassociating these sequences.
// On GB300 the FP32 pipe issues 64x the FP64 pipe's FMAs, so an FP64-accurate contraction in
// df64 (about 27 FP32 instructions per FMA) can outrun native FP64.
#pragma once
#include <cuda_runtime.h>

namespace nhmf {

struct __align__(8) df64 {
  float hi, lo;
  __device__ __forceinline__ df64() {}
  __device__ __forceinline__ df64(float h, float l) : hi(h), lo(l) {}
  // nearest df64 to an FP64 value: hi = fl32(d), lo = fl32(d - hi)
  __device__ __forceinline__ explicit df64(double d) {
    hi = __double2float_rn(d);
    lo = __double2float_rn(d - (double)hi);
  }
  __device__ __forceinline__ explicit df64(int i) : hi(float(i)), lo(0.f) {}
};

__device__ __forceinline__ double to_double(df64 a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

__device__ __forceinline__ float fast_two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
  return s;
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  float e1, e2, e3, e4;
  float s = two_sum(a.hi, b.hi, e1);
  const float t = two_sum(a.lo, b.lo, e2);
  e1 = __fadd_rn(e1, t);
  s = fast_two_sum(s, e1, e3);
  e3 = __fadd_rn(e3, e2);
  s = fast_two_sum(s, e3, e4);
  return df64(s, e4);
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float l;
  const float s = fast_two_sum(p, e, l);
  return df64(s, l);
}

using ::fma;  // keep the FP64/FP32 overloads visible next to the df64 one
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) { return a * b + c; }
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) {
  a = a + b;
  return a;
}

}  // namespace nhmf
