// Float-float arithmetic: a real number held as the unevaluated sum hi + lo of two FP32
// numbers, |lo| <= ulp(hi) / 2, about 48 significant bits. Built from error-free
// transformations of FP32 operations: TwoSum (Knuth, TAOCP vol. 2, 4.2.2), FastTwoSum and
// the splitting product of T. J. Dekker ("A floating-point technique for extending the
// available precision", Numer. Math. 18, 1971), the exact product error by one FMA. Every
// step uses the round-to-nearest intrinsics, which the compiler neither contracts nor
// reorders.
//
// Use: the FP64 residual of the mixed-precision refinement. The transform passes are
// templated on the arithmetic type; with ffloat they run on the FP32 pipes, whose issue
// rate on this GPU is more than sixty times the FP64 one, at about 2^-47 relative error per
// operation (FP64: 2^-53), while every value in memory outside the passes stays FP64.
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

// a + b: the high parts by TwoSum, the low parts added to its error, renormalised; absolute
// error below about 3 * 2^-48 (|a| + |b|), as an FP64 addition's is below 2^-53 |a + b|
__device__ __forceinline__ ffloat operator+(ffloat a, ffloat b) {
  const ffloat s = ff_two_sum(a.hi, b.hi);
  return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ffloat operator-(ffloat a) { return ffloat(-a.hi, -a.lo); }
__device__ __forceinline__ ffloat operator-(ffloat a, ffloat b) { return a + (-b); }

// a * b: hi * hi with its exact error by FMA, the cross terms folded into the error
__device__ __forceinline__ ffloat operator*(ffloat a, ffloat b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}

// a * b + c with one renormalisation: the product's high part and c's by TwoSum, the
// product error, the cross terms and c's low part added to the TwoSum error
__device__ __forceinline__ ffloat fma(ffloat a, ffloat b, ffloat c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  const ffloat s = ff_two_sum(p, c.hi);
  return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(pe, c.lo)));
}

// a / b by one correction step of long division: q1 = fl(a.hi / b.hi), the remainder
// a - q1 b in float-float, q2 = fl(rem / b.hi)
__device__ __forceinline__ ffloat operator/(ffloat a, ffloat b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const ffloat rem = a - b * ffloat(q1, 0.f);
  const float q2 = __fdiv_rn(rem.hi, b.hi);
  return ff_fast_two_sum(q1, q2);
}

__device__ __forceinline__ ffloat& operator+=(ffloat& a, ffloat b) { return a = a + b; }
__device__ __forceinline__ bool operator==(ffloat a, ffloat b) { return a.hi == b.hi && a.lo == b.lo; }

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
