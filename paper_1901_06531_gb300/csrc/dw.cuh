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
  float e = __fmaf_rn(a.lo, b.lo, 0.0f);   // kept: for squares it has one sign (no bias in sums of squares)
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  e = __fadd_rn(e, __fmaf_rn(a.hi, b.hi, -p));               // TwoProd error
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

// Compensated sum of double-word terms and products with one normalisation
// at the end (Ogita, Rump, Oishi, "Accurate sum and dot product", SIAM J.
// Sci. Comput. 2005, algorithm Dot2, on the high parts): the running head s
// is updated by TwoSum, so the head is exact up to the error e, which
// gathers the TwoSum and TwoProd errors and the low-part terms in one FP32
// word.  Each error added to e is of order 2^-24 of the term, so its own
// rounding is of order 2^-48: the accuracy of a chain of double-word
// operations, in about 12 FP32 operations per product term instead of 20.
struct DwAcc {
  float s, e;
  __device__ __forceinline__ DwAcc() : s(0.0f), e(0.0f) {}
  __device__ __forceinline__ explicit DwAcc(dw a) : s(a.hi), e(a.lo) {}
  __device__ __forceinline__ void head(float p, float pe) {   // s += p (TwoSum), pe joins the error
    const float t = __fadd_rn(s, p);
    const float bb = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    s = t;
    e = __fadd_rn(e, __fadd_rn(err, pe));
  }
  __device__ __forceinline__ void add(dw a) { head(a.hi, a.lo); }
  // += a b
  __device__ __forceinline__ void fma(dw a, dw b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float pe = __fmaf_rn(a.hi, b.hi, -p);   // TwoProd error
    pe = __fmaf_rn(a.hi, b.lo, pe);
    pe = __fmaf_rn(a.lo, b.hi, pe);
    pe = __fmaf_rn(a.lo, b.lo, pe);          // kept: one sign for squares, as in mul
    head(p, pe);
  }
  __device__ __forceinline__ dw value() const { return dwops::fast_two_sum(s, e); }
};

__device__ __forceinline__ dwc cmake(dw a, dw b) { dwc r; r.x = a; r.y = b; return r; }

#ifndef MF_NO_F32X2
// Complex double-word add and subtract with the real and imaginary parts in
// the two lanes of packed FP32 instructions (add.f32x2, sub.f32x2): the same
// operations in the same order as dwops::add on each part, so the results
// are those of the scalar form bit for bit.
namespace dwpk {
typedef unsigned long long u64;
__device__ __forceinline__ u64 pk(float a, float b) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk(u64 r, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r)); }
__device__ __forceinline__ u64 add(u64 a, u64 b) {
  u64 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 sub(u64 a, u64 b) {
  u64 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
// (a + b) or (a - b) per part; NEG: subtract
template <bool NEG>
__device__ __forceinline__ dwc addsub(dwc a, dwc b) {
  const u64 A = pk(a.x.hi, a.y.hi), B = pk(b.x.hi, b.y.hi);
  const u64 s = NEG ? sub(A, B) : add(A, B);
  const u64 bb = sub(s, A);
  // TwoSum error: (a.hi - (s - bb)) + (b.hi - bb), with b.hi negated for NEG
  const u64 e0 = sub(A, sub(s, bb));
  const u64 e = NEG ? sub(e0, add(B, bb)) : add(e0, sub(B, bb));
  const u64 L = NEG ? sub(pk(a.x.lo, a.y.lo), pk(b.x.lo, b.y.lo)) : add(pk(a.x.lo, a.y.lo), pk(b.x.lo, b.y.lo));
  const u64 t = add(e, L);
  const u64 s2 = add(s, t);
  const u64 e2 = sub(t, sub(s2, s));
  dwc r;
  upk(s2, r.x.hi, r.y.hi);
  upk(e2, r.x.lo, r.y.lo);
  return r;
}
}  // namespace dwpk
__device__ __forceinline__ dwc cadd(dwc a, dwc b) { return dwpk::addsub<false>(a, b); }
__device__ __forceinline__ dwc csub(dwc a, dwc b) { return dwpk::addsub<true>(a, b); }
#endif

// Complex products with the TwoProd errors of both real products gathered
// before one TwoSum (fewer operations than four double-word products and
// two double-word sums).  a b (SIGN = -1) or a conj(b) pieces are formed by
// the callers below.
__device__ __forceinline__ dw dot2(dw a, dw b, dw c, dw d, bool minus) {
  // a b - c d (minus) or a b + c d
  const float p1 = __fmul_rn(a.hi, b.hi);
  const float e1 = __fmaf_rn(a.hi, b.hi, -p1);
  float p2 = __fmul_rn(c.hi, d.hi);
  float e2 = __fmaf_rn(c.hi, d.hi, -p2);
  if (minus) { p2 = -p2; e2 = -e2; }
  const float s = __fadd_rn(p1, p2);
  const float bb = __fsub_rn(s, p1);
  float e = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bb)), __fsub_rn(p2, bb));
  e = __fadd_rn(e, __fadd_rn(e1, e2));
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  e = minus ? __fmaf_rn(-c.hi, d.lo, e) : __fmaf_rn(c.hi, d.lo, e);
  e = minus ? __fmaf_rn(-c.lo, d.hi, e) : __fmaf_rn(c.lo, d.hi, e);
  return dwops::fast_two_sum(s, e);
}
__device__ __forceinline__ dwc cmul(dwc a, dwc b) {
  dwc r;
  r.x = dot2(a.x, b.x, a.y, b.y, true);
  r.y = dot2(a.x, b.y, a.y, b.x, false);
  return r;
}
// a * conj(b)
__device__ __forceinline__ dwc cmulc(dwc a, dwc b) {
  dwc r;
  r.x = dot2(a.x, b.x, a.y, b.y, false);
  r.y = dot2(a.y, b.x, a.x, b.y, true);
  return r;
}

// FP64 <-> double word by bit manipulation (no FP64 instruction on the way
// in, one FP64 addition on the way out: FP64 and its conversions run on the
// slow FP64 pipe of this part).
//
// In: hi = the FP64 value truncated to 24 significant bits (exact in FP32),
// lo = the remaining 29 bits rounded to the nearest 24 (so that the error,
// at most 2^-48 relative, has no bias: averages over many voxels keep FP64
// accuracy).  Magnitudes below 2^-74 contribute no lo part; below 2^-126
// the value becomes zero; beyond the FP32 range it becomes an infinity, and
// infinities and NaNs pass through (so a non-finite P is still seen).
__device__ __forceinline__ dw dw_split(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const unsigned sign = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7ffu);
  const unsigned m23 = ((hw & 0xfffffu) << 3) | (lw >> 29);
  if (e >= 897 && e <= 1150) {
    const float hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | m23);
    float lo = 0.0f;
    const unsigned ml = lw & 0x1fffffffu;
    if (ml != 0u && e >= 949) {
      lo = __fmul_rn(__uint2float_rn(ml), __uint_as_float((unsigned)(e - 948) << 23));
      if (sign) lo = -lo;
    }
    return dwops::fast_two_sum(hi, lo);   // normalise: abs(lo) <= ulp(hi)/2
  }
  if (e < 897) return dw(sign ? -0.0f : 0.0f, 0.0f);
  const unsigned nan = (e == 2047 && ((hw & 0xfffffu) | lw)) ? 0x400000u : 0u;
  return dw(__uint_as_float(sign | 0x7f800000u | nan), 0.0f);
}

// An FP32 value as FP64, exactly (subnormal FP32 values flush to zero).
__device__ __forceinline__ double f32_as_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e8 = (u >> 23) & 0xffu;
  const unsigned sign = u & 0x80000000u;
  if (e8 == 0u) return __hiloint2double((int)sign, 0);
  if (e8 == 255u)
    return __hiloint2double((int)(sign | 0x7ff00000u | ((u & 0x7fffffu) ? 0x80000u : 0u)), 0);
  return __hiloint2double((int)(sign | ((e8 + 896u) << 20) | ((u >> 3) & 0xfffffu)), (int)(u << 29));
}

__device__ __forceinline__ double dw_join(dw a) { return f32_as_f64(a.hi) + f32_as_f64(a.lo); }

__device__ __forceinline__ dwc to_dwc(double2 v) { dwc r; r.x = dw_split(v.x); r.y = dw_split(v.y); return r; }
__device__ __forceinline__ double2 to_double2(dwc v) { return make_double2(dw_join(v.x), dw_join(v.y)); }
