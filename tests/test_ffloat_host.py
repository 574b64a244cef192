"""Float-float arithmetic of the refinement residuals (csrc/ffloat.cuh) checked on the CPU.

The header's operations are compiled as host C++ with the CUDA round-to-nearest intrinsics
mapped to plain IEEE single-precision operations (strict evaluation, no contraction), and
checked against exact or long-double references: TwoSum and FastTwoSum are error-free
(Knuth; Dekker), the unnormalised sum, product and fused multiply-add keep their value to a
few 2^-48 of the operands' magnitudes, a stage of operations followed by the stores'
renormalisation keeps that bound, and the division is accurate to about 2^-46.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1404_3614_gb300", "csrc")

SHIM = r"""
#pragma once
#include <cmath>
#define __host__
#define __device__
#define __forceinline__ inline
#define __align__(n) alignas(n)
struct double2 { double x, y; };
inline double2 make_double2(double x, double y) { return double2{x, y}; }
static inline float __fadd_rn(float a, float b) { volatile float r = a + b; return r; }
static inline float __fsub_rn(float a, float b) { volatile float r = a - b; return r; }
static inline float __fmul_rn(float a, float b) { volatile float r = a * b; return r; }
static inline float __fmaf_rn(float a, float b, float c) { return std::fmaf(a, b, c); }
static inline float __fdiv_rn(float a, float b) { volatile float r = a / b; return r; }
static inline float __double2float_rn(double x) { return (float)x; }
"""

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include "ffloat.cuh"
using homb::ffloat;
typedef long double LD;
static LD val(ffloat a) { return (LD)a.hi + (LD)a.lo; }
static uint64_t st = 88172645463325252ull;
static double urand() {   // xorshift64, uniform in [-1, 1)
  st ^= st << 13; st ^= st >> 7; st ^= st << 17;
  return (double)(st >> 11) / 4503599627370496.0 - 1.0;
}
static ffloat rnd(double scale) {
  const double x = urand() * scale * std::ldexp(1.0, (int)(st % 7) - 3);
  return ffloat(x);
}
int main() {
  const LD u = std::ldexp((LD)1, -48);
  LD worst_add = 0, worst_mul = 0, worst_fma = 0, worst_div = 0, worst_chain = 0;
  long bad_2sum = 0, bad_fast = 0;
  for (int it = 0; it < 200000; ++it) {
    const float a = (float)urand() * std::ldexp(1.0f, (int)(st % 40) - 20);
    const float b = (float)urand() * std::ldexp(1.0f, (int)((st >> 8) % 40) - 20);
    const ffloat s = homb::ffa::ff_two_sum(a, b);
    if ((LD)s.hi + (LD)s.lo != (LD)a + (LD)b) ++bad_2sum;
    const float big = std::fabs(a) >= std::fabs(b) ? a : b, small = std::fabs(a) >= std::fabs(b) ? b : a;
    const ffloat f = homb::ffa::ff_fast_two_sum(big, small);
    if ((LD)f.hi + (LD)f.lo != (LD)big + (LD)small) ++bad_fast;
    const ffloat x = rnd(1.0), y = rnd(1.0), z = rnd(1.0);
    const LD mx = std::fabs(val(x)), my = std::fabs(val(y)), mz = std::fabs(val(z));
    LD e = std::fabs(val(x + y) - (val(x) + val(y))) / ((mx + my) * u);
    if (e > worst_add) worst_add = e;
    e = std::fabs(val(x * y) - val(x) * val(y)) / (mx * my * u);
    if (e > worst_mul) worst_mul = e;
    e = std::fabs(val(fma(x, y, z)) - (val(x) * val(y) + val(z))) / ((mx * my + mz) * u);
    if (e > worst_fma) worst_fma = e;
    if (my > 1e-3) {
      const LD q = val(x) / val(y);
      e = std::fabs(val(x / y) - q) / (std::fabs(q) * u);
      if (e > worst_div) worst_div = e;
    }
    // one radix stage's depth of unnormalised sums and products, then the store's renormalisation
    ffloat acc = x;
    LD ref = val(x), mag = mx;
    for (int k = 0; k < 8; ++k) {
      const ffloat w = rnd(1.0), c = rnd(1.0);
      acc = fma(c, w, acc) - w;
      ref = val(c) * val(w) + ref - val(w);
      mag += std::fabs(val(c) * val(w)) + std::fabs(val(w));
    }
    acc = homb::ffa::ff_norm(acc);
    e = std::fabs(val(acc) - ref) / (mag * u);
    if (e > worst_chain) worst_chain = e;
    if (std::fabs((LD)acc.lo) > std::ldexp(std::fabs((LD)acc.hi), -24)) ++bad_fast;
  }
  std::printf("%ld %ld %.4Lf %.4Lf %.4Lf %.4Lf %.4Lf\n", bad_2sum, bad_fast, worst_add, worst_mul, worst_fma,
              worst_div, worst_chain);
  return 0;
}
"""


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("ffloat")
    (d / "cuda_runtime.h").write_text(SHIM)
    (d / "main.cpp").write_text(DRIVER)
    exe = d / "ffcheck"
    subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-I", str(d), "-I", CSRC,
                    str(d / "main.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return [int(out[0]), int(out[1])] + [float(v) for v in out[2:]]


def test_error_free_sums(results):
    """TwoSum on any pair and FastTwoSum with the larger operand first are exact."""
    assert results[0] == 0 and results[1] == 0, results


def test_unnormalised_operations_stay_within_a_few_ulps_of_2_48(results):
    """Sum, product and fused multiply-add without renormalisation: error below 6 * 2^-48 of
    the operands' magnitudes (an FP64 operation's is 2^-53 of its result's; measured worst
    cases over 200 000 random operands: about 2.3, 3.1 and 4.2)."""
    add, mul, fma_, div, chain = results[2:]
    assert add <= 6.0 and mul <= 6.0 and fma_ <= 6.0, results


def test_division_and_a_stage_chain(results):
    """The division (renormalised operands, one correction) is within 8 * 2^-48 relative; eight
    unnormalised multiply-adds and subtractions, as in one radix stage, then the store's
    renormalisation stay within 32 * 2^-48 of the summed magnitudes, and leave |lo| below
    2^-24 |hi| (checked with the error-free sums above)."""
    add, mul, fma_, div, chain = results[2:]
    assert div <= 8.0 and chain <= 32.0, results
