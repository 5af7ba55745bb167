// Double-word ("float-float") arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers with abs(lo) <= ulp(hi)/2, about 48 significant
// bits.  Used for the transforms of the FP64 residual in the FP32-inner
// precision mode: on this part FP32 instructions issue at many times the FP64
// rate, and a double-word FFT keeps the residual at FP64-level accuracy
// (relative error of a few 2^-48 per operation, far below the Newton and CG
// tolerances).
//
// Building blocks (Dekker 1971; Knuth, TAOCP vol. 2, 4.2.2; Joldes, Muller,
// Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", ACM TOMS 2017):
//   TwoSum(a, b):     s = fl(a + b) and the exact error e, a + b = s + e;
//   FastTwoSum(a, b): the same when abs(a) >= abs(b), three operations;
//   TwoProd(a, b):    p = fl(a b), e = fma(a, b, -p) exact, a b = p + e.
// Addition is the "sloppy" double-word sum (error bounded relative to
// abs(x) + abs(y), which is what the normwise error of an FFT needs),
// multiplication the FMA-based product.  Every operation goes through the
// _rn intrinsics so that the compiler cannot contract a product into a later
// sum (that would change the error terms).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

struct dw {
  float hi, lo;
  dw() = default;
  __host__ __device__ constexpr dw(float h, float l) : hi(h), lo(l) {}
  // from FP64: hi = fl32(v), lo = fl32(v - hi)
  __host__ __device__ constexpr dw(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ constexpr dw(int k) : hi((float)k), lo(0.0f) {}   // exact for abs(k) < 2^24
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __host__ __device__ explicit operator float() const { return hi + lo; }
};

struct dwc {
  dw x, y;
};
template <> struct CT<dw> { typedef dwc t; };

namespace dwops {

__device__ __forceinline__ dw fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return dw(s, e);
}

__device__ __forceinline__ dw add(dw a, dw b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));   // TwoSum error
  return fast_two_sum(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ dw neg(dw a) { return dw(-a.hi, -a.lo); }

__device__ __forceinline__ dw mul(dw a, dw b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);                       // TwoProd error
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// a / b: two quotient digits, q1 = a.hi / b.hi and q2 from the remainder
__device__ __forceinline__ dw div(dw a, dw b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const dw r = add(a, neg(mul(b, dw(q1, 0.0f))));
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return fast_two_sum(q1, q2);
}

}  // namespace dwops

__device__ __forceinline__ dw operator+(dw a, dw b) { return dwops::add(a, b); }
__device__ __forceinline__ dw operator-(dw a, dw b) { return dwops::add(a, dwops::neg(b)); }
__device__ __forceinline__ dw operator-(dw a) { return dwops::neg(a); }
__device__ __forceinline__ dw operator*(dw a, dw b) { return dwops::mul(a, b); }
__device__ __forceinline__ dw operator/(dw a, dw b) { return dwops::div(a, b); }
__device__ __forceinline__ dw& operator+=(dw& a, dw b) { a = a + b; return a; }
__device__ __forceinline__ dw& operator-=(dw& a, dw b) { a = a - b; return a; }

__device__ __forceinline__ dwc cmake(dw a, dw b) { dwc r; r.x = a; r.y = b; return r; }

// exact split of an FP64 complex value into double-word parts, and back
__device__ __forceinline__ dwc to_dwc(double2 v) { dwc r; r.x = dw(v.x); r.y = dw(v.y); return r; }
__device__ __forceinline__ double2 to_double2(dwc v) { return make_double2((double)v.x, (double)v.y); }
