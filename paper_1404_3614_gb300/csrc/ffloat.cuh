// Float-float arithmetic: a real number held as the unevaluated sum hi + lo of two FP32
// numbers, about 48 significant bits. Built from error-free transformations of FP32
// operations: TwoSum (Knuth, TAOCP vol. 2, 4.2.2), FastTwoSum and the exact product error of
// T. J. Dekker ("A floating-point technique for extending the available precision", Numer.
// Math. 18, 1971), here by one FMA. Every step uses the round-to-nearest intrinsics, which
// the compiler neither contracts nor reorders.
//
// The sums and products do not renormalise their result (|lo| <= ulp(hi) / 2 is not kept):
// hi is the FP32 sum or product of the high parts, exactly, and lo gathers its exact
// rounding error with the low-part terms. This saves the FastTwoSum of every operation
// (addition 8 FP32 operations instead of 11, product 4 instead of 7). The low part then
// grows with each unnormalised operation and its own rounding with it, so the transform
// passes renormalise every value they store between stages (st_norm): within one radix
// stage, a few operations deep, the error stays a small multiple of 2^-48 of the operands'
// magnitudes, the measure that bounds a transform's error (an FP64 operation's is 2^-53).
// The division, whose quotient estimate needs hi to dominate, renormalises its operands.
//
// Use: the FP64 residual of the mixed-precision refinement. The transform passes are
// templated on the arithmetic type; with ffloat they run on the FP32 pipes, whose issue
// rate on this GPU is more than sixty times the FP64 one, while every value in memory outside
// the passes stays FP64.
#pragma once
#include <cuda_runtime.h>

namespace homb {
// The type and its operators live in a namespace of their own, found by argument-dependent
// lookup: an fma(ffloat, ffloat, ffloat) declared in homb itself would hide the FP32 / FP64
// fma of the templated passes.
namespace ffa {

struct __align__(8) ffloat {
  float hi, lo;
  ffloat() = default;
  __host__ __device__ constexpr ffloat(float h, float l) : hi(h), lo(l) {}
  // nearest float-float of a double: hi = fl32(x), lo = fl32(x - hi) (x - hi is exact)
  __host__ __device__ explicit constexpr ffloat(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

struct __align__(16) ffloat2 {
  ffloat x, y;
};

// s + e = a + b exactly, for |a| >= |b| (or a = 0)
__device__ __forceinline__ ffloat ff_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return ffloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// s + e = a + b exactly, any order of magnitude
__device__ __forceinline__ ffloat ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ffloat(s, e);
}

// a + b: the high parts by TwoSum, the low parts added to its error (not renormalised);
// absolute error below about 2 * 2^-24 (|a.lo| + |b.lo| + |s.lo|), i.e. a few 2^-48 (|a| + |b|)
__device__ __forceinline__ ffloat operator+(ffloat a, ffloat b) {
  const ffloat s = ff_two_sum(a.hi, b.hi);
  return ffloat(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ffloat operator-(ffloat a) { return ffloat(-a.hi, -a.lo); }
__device__ __forceinline__ ffloat operator-(ffloat a, ffloat b) { return a + (-b); }

// a * b: hi * hi with its exact error by FMA, the cross terms folded into the error (the
// lo * lo term, below 2^-48 |a b|, is dropped)
__device__ __forceinline__ ffloat operator*(ffloat a, ffloat b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ffloat(p, e);
}

// a * b + c: the product's high part and c's by TwoSum, the product error, the cross terms
// and c's low part added to the TwoSum error
__device__ __forceinline__ ffloat fma(ffloat a, ffloat b, ffloat c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  const ffloat s = ff_two_sum(p, c.hi);
  return ffloat(s.hi, __fadd_rn(s.lo, __fadd_rn(pe, c.lo)));
}

// the same value with |lo| <= ulp(hi) / 2
__device__ __forceinline__ ffloat ff_norm(ffloat a) { return ff_two_sum(a.hi, a.lo); }

// a / b by one correction step of long division on renormalised operands: q1 = fl(a.hi /
// b.hi), the remainder a - q1 b in float-float, q2 = fl(rem / b.hi)
__device__ __forceinline__ ffloat operator/(ffloat a, ffloat b) {
  a = ff_norm(a);
  b = ff_norm(b);
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const ffloat rem = a - b * ffloat(q1, 0.f);
  const float q2 = __fdiv_rn(__fadd_rn(rem.hi, rem.lo), b.hi);
  return ff_fast_two_sum(q1, q2);
}

__device__ __forceinline__ ffloat& operator+=(ffloat& a, ffloat b) { return a = a + b; }
// equality of the values (the pairs need not be normalised)
__device__ __forceinline__ bool operator==(ffloat a, ffloat b) {
  const ffloat d = ff_norm(a - b);
  return d.hi == 0.f;
}

}  // namespace ffa

using ffa::ffloat;
using ffa::ffloat2;

template <typename T> struct is_ff { static constexpr bool value = false; };
template <> struct is_ff<ffloat> { static constexpr bool value = true; };

// conversions of FP64 data at the edges of a float-float pass
__device__ __forceinline__ ffloat ff_from(double x) {
  const float h = __double2float_rn(x);
  return ffloat(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ ffloat2 ff2_from(double2 v) {
  ffloat2 r;
  r.x = ff_from(v.x);
  r.y = ff_from(v.y);
  return r;
}
__device__ __forceinline__ double2 ff2_to(ffloat2 v) { return make_double2((double)v.x, (double)v.y); }

}  // namespace homb
