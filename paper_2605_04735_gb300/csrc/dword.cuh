// Double-word ("double-float") arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significand
// bits.  GB300 runs FP32 at 64 times its FP64 rate, so an operator evaluated
// in double-word arithmetic (7 to 11 FP32 operations per operation) is
// several times faster than the same operator in FP64, at an error of about
// 2^-48 instead of 2^-53 per operation.
//
// Building blocks (error-free transformations, all in round-to-nearest):
//   two_sum       Knuth's TwoSum: s + e == a + b exactly, no ordering needed;
//   fast_two_sum  Dekker's Fast2Sum: exact when exponent(a) >= exponent(b);
//   the product error a*b - round(a*b) from one FMA.
// The sum adds the two high parts exactly and the low parts (with the
// rounding error) in FP32, then renormalises: its absolute error stays
// within a few 2^-48 (|x| + |y|), which is what an operator sum needs.
// Every operation uses the __f*_rn intrinsics, which the compiler never
// contracts into an FMA or reorders.
#pragma once

#include <cuda_runtime.h>

namespace topo {

struct Dw {
  float hi, lo;
  Dw() = default;
  __host__ __device__ explicit constexpr Dw(float h, float l = 0.0f) : hi(h), lo(l) {}
};

__device__ __forceinline__ Dw two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return Dw(s, e);
}

__device__ __forceinline__ Dw fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return Dw(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ Dw operator+(Dw x, Dw y) {
  const Dw s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ Dw operator-(Dw x) { return Dw(-x.hi, -x.lo); }

__device__ __forceinline__ Dw operator-(Dw x, Dw y) { return x + (-y); }

__device__ __forceinline__ Dw& operator+=(Dw& x, Dw y) { return x = x + y; }

__device__ __forceinline__ Dw operator*(Dw x, Dw y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);  // exact rounding error of the product
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ Dw fmadd(Dw a, Dw b, Dw c) { return a * b + c; }

// split a double into hi + lo (exact up to the 48 bits the pair holds)
__host__ __device__ __forceinline__ Dw dw_from(double v) {
  const float h = (float)v;
  return Dw(h, (float)(v - (double)h));
}

__device__ __forceinline__ double dw_to(Dw v) { return (double)v.hi + (double)v.lo; }

// warp shuffle of both words
__device__ __forceinline__ Dw shfl_up1(Dw v) {
  return Dw(__shfl_up_sync(0xffffffffu, v.hi, 1), __shfl_up_sync(0xffffffffu, v.lo, 1));
}

}  // namespace topo
