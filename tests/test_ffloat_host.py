"""Float-float arithmetic of the refinement residuals (csrc/ffloat.cuh) checked on the CPU.

The header's operations are compiled as host C++ with the CUDA round-to-nearest intrinsics
mapped to plain IEEE single-precision operations (strict evaluation, no contraction), and
checked against exact or long-double references: TwoSum and FastTwoSum are error-free
(Knuth; Dekker), the unnormalised sum, product and fused multiply-add keep their value to a
few 2^-48 of the operands' magnitudes, a stage of operations followed by the stores'
renormalisation keeps that bound, and the division is accurate to about 2^-46.

The warp-level register FFTs of csrc/slab.cuh (the float-float passes at length 225) run as
15 host threads, one per lane of a lane group, with the warp barrier as a thread barrier.

The block-level FFT engine of csrc/common.cuh is compiled the same way, as one thread that
runs every butterfly of a stage in turn (its loops stride by the block size, and the barriers
become no-ops), and its float-float transforms are checked against the DFT's definition
summed in long double: the compile-time register schedules (radix 15, 9, 5, 3) at the double
grid's lengths, with and without the zero band's pruned first and last stages, and the
runtime plan (a generic prime radix).
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


FFT_SHIM_EXTRA = r"""
struct float2 { float x, y; };
inline float2 make_float2(float x, float y) { return float2{x, y}; }
struct HostDim { unsigned x, y, z; };
static HostDim threadIdx{0, 0, 0}, blockDim{1, 1, 1}, blockIdx{0, 0, 0}, gridDim{1, 1, 1};
inline void __syncthreads() {}
inline double __shfl_down_sync(unsigned, double v, int) { return v; }
inline unsigned __umulhi(unsigned a, unsigned b) { return (unsigned)(((unsigned long long)a * b) >> 32); }
"""

FFT_DRIVER = r"""
#include <cstdio>
#include <cmath>
#include <vector>
#include "common.cuh"
using namespace homb;
typedef long double LD;
static const LD PI = 3.141592653589793238462643383279502884L;
static uint64_t st = 0x9E3779B97F4A7C15ull;
static double urand() { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return (double)(st >> 11) / 4503599627370496.0 - 1.0; }
static ffloat split(LD v) { const float h = (float)v; return ffloat(h, (float)(v - (LD)h)); }
static LD val(ffloat a) { return (LD)a.hi + (LD)a.lo; }

// max |X - DFT(x)| / max |DFT(x)| over G pencils; band: the inputs of the zero band (positions
// 4M/15 .. 11M/15 - 1, the lane rows 4..10 of the radix-15 layout) are zero, and with trunc only
// the outputs outside it are compared
template <int M>
static double check(int dir, int prune, bool band, bool trunc) {
  const int G = 3;
  std::vector<ffloat2> W(M), a(G * M), b(G * M);
  for (int j = 0; j < M; ++j) W[j] = ffloat2{split(std::cos(-2 * PI * j / M)), split(std::sin(-2 * PI * j / M))};
  std::vector<LD> xr(G * M), xi(G * M);
  const int lo = 4 * M / 15, hi = 11 * M / 15;
  for (int i = 0; i < G * M; ++i) {
    const int p = i % M;
    const bool zero = band && p >= lo && p < hi;
    const double re = zero ? 0.0 : urand(), im = zero ? 0.0 : urand();
    a[i] = ffloat2{ffloat(re), ffloat(im)};
    xr[i] = val(a[i].x); xi[i] = val(a[i].y);
  }
  ffloat2* res = cfft<ffloat, M>(a.data(), b.data(), G, W.data(), dir, prune);
  double worst = 0, scale = 0;
  std::vector<LD> Xr(M), Xi(M);
  for (int g = 0; g < G; ++g) {
    for (int k = 0; k < M; ++k) {
      LD sr = 0, si = 0;
      for (int n = 0; n < M; ++n) {
        const LD ang = dir * 2 * PI * (LD)((long long)n * k % M) / M;
        const LD c = std::cos(ang), s = std::sin(ang);
        sr += xr[g * M + n] * c - xi[g * M + n] * s;
        si += xr[g * M + n] * s + xi[g * M + n] * c;
      }
      Xr[k] = sr; Xi[k] = si;
      scale = std::fmax(scale, (double)std::sqrt(sr * sr + si * si));
    }
    for (int k = 0; k < M; ++k) {
      if (trunc && k >= lo && k < hi) continue;
      const ffloat2 v = res[g * M + k];
      const LD er = val(v.x) - Xr[k], ei = val(v.y) - Xi[k];
      worst = std::fmax(worst, (double)std::sqrt(er * er + ei * ei));
    }
  }
  return worst / scale;
}


// a chain like the operator's: inverse transform, pointwise coefficient (values 1 and 1/100),
// forward transform, repeated three times, against the same chain in long double
template <int M>
static double check_chain() {
  const int G = 2;
  std::vector<ffloat2> W(M), a(G * M), b(G * M);
  for (int j = 0; j < M; ++j) W[j] = ffloat2{split(std::cos(-2 * PI * j / M)), split(std::sin(-2 * PI * j / M))};
  std::vector<LD> xr(G * M), xi(G * M), c(M);
  for (int j = 0; j < M; ++j) c[j] = (j % 7) < 3 ? 1.0L : 0.01L;
  for (int i = 0; i < G * M; ++i) {
    a[i] = ffloat2{ffloat(urand()), ffloat(urand())};
    xr[i] = val(a[i].x); xi[i] = val(a[i].y);
  }
  ffloat2* cur = a.data();
  ffloat2* oth = b.data();
  for (int rep = 0; rep < 3; ++rep) {
    for (int dir : {+1, -1}) {
      ffloat2* res = cfft<ffloat, M>(cur, oth, G, W.data(), dir, 0);
      oth = res == cur ? oth : cur;
      cur = res;
      std::vector<LD> yr(G * M), yi(G * M);
      for (int g = 0; g < G; ++g)
        for (int k = 0; k < M; ++k) {
          LD sr = 0, si = 0;
          for (int n = 0; n < M; ++n) {
            const LD ang = dir * 2 * PI * (LD)((long long)n * k % M) / M;
            sr += xr[g * M + n] * std::cos(ang) - xi[g * M + n] * std::sin(ang);
            si += xr[g * M + n] * std::sin(ang) + xi[g * M + n] * std::cos(ang);
          }
          yr[g * M + k] = sr / (dir > 0 ? 1 : M); yi[g * M + k] = si / (dir > 0 ? 1 : M);
        }
      xr = yr; xi = yi;
      for (int i = 0; i < G * M; ++i) {   // the coefficient after the inverse, 1/M after the forward
        const ffloat s = dir > 0 ? split(c[i % M]) : split(1.0L / M);
        const LD sv = dir > 0 ? c[i % M] : 1.0L;
        cur[i].x = cur[i].x * s;
        cur[i].y = cur[i].y * s;
        if (dir > 0) { xr[i] *= sv; xi[i] *= sv; }
      }
    }
  }
  double worst = 0, scale = 0;
  for (int i = 0; i < G * M; ++i) {
    scale = std::fmax(scale, (double)std::sqrt(xr[i] * xr[i] + xi[i] * xi[i]));
    const LD er = val(cur[i].x) - xr[i], ei = val(cur[i].y) - xi[i];
    worst = std::fmax(worst, (double)std::sqrt(er * er + ei * ei));
  }
  return worst / scale;
}

static double check_plan(int M, int dir) {
  FftPlan plan{};
  plan.M = M;
  int m = M;
  for (int r : {5, 3, 7, 11, 13}) while (m % r == 0) { plan.radix[plan.nrad++] = r; m /= r; }
  if (m > 1) plan.radix[plan.nrad++] = m;   // one generic prime radix
  const int G = 2;
  std::vector<ffloat2> W(M), a(G * M), b(G * M);
  for (int j = 0; j < M; ++j) W[j] = ffloat2{split(std::cos(-2 * PI * j / M)), split(std::sin(-2 * PI * j / M))};
  std::vector<LD> xr(G * M), xi(G * M);
  for (int i = 0; i < G * M; ++i) {
    a[i] = ffloat2{ffloat(urand()), ffloat(urand())};
    xr[i] = val(a[i].x); xi[i] = val(a[i].y);
  }
  ffloat2* res = fft_pencils<ffloat>(a.data(), b.data(), G, M, plan, W.data(), dir);
  double worst = 0, scale = 0;
  for (int g = 0; g < G; ++g)
    for (int k = 0; k < M; ++k) {
      LD sr = 0, si = 0;
      for (int n = 0; n < M; ++n) {
        const LD ang = dir * 2 * PI * (LD)((long long)n * k % M) / M;
        sr += xr[g * M + n] * std::cos(ang) - xi[g * M + n] * std::sin(ang);
        si += xr[g * M + n] * std::sin(ang) + xi[g * M + n] * std::cos(ang);
      }
      scale = std::fmax(scale, (double)std::sqrt(sr * sr + si * si));
      const LD er = val(res[g * M + k].x) - sr, ei = val(res[g * M + k].y) - si;
      worst = std::fmax(worst, (double)std::sqrt(er * er + ei * ei));
    }
  return worst / scale;
}

int main() {
  std::printf("%.3e %.3e %.3e %.3e %.3e %.3e %.3e %.3e %.3e %.3e %.3e %.3e\n",
              check<225>(-1, 0, false, false), check<225>(+1, 0, false, false),
              check<225>(+1, 4, true, false), check<225>(-1, 8, false, true),
              check<45>(-1, 0, false, false), check<81>(+1, 0, false, false),
              check<125>(-1, 0, false, false), check<405>(+1, 0, false, false),
              check_plan(17 * 3, -1), check_plan(7 * 5, +1), check_chain<45>(), check_chain<225>());
  return 0;
}
"""


@pytest.fixture(scope="module")
def fft_errors(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("ffloat_fft")
    (d / "cuda_runtime.h").write_text(SHIM + FFT_SHIM_EXTRA)
    (d / "main.cpp").write_text(FFT_DRIVER)
    exe = d / "fftcheck"
    subprocess.run([cxx, "-std=c++17", "-O1", "-ffp-contract=off", "-fno-fast-math", "-I", str(d), "-I", CSRC,
                    str(d / "main.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return [float(v) for v in out]


def test_register_schedules_at_225(fft_errors):
    """Length 225 in two radix-15 stages (prime-factor 3 x 5 in registers), forward and inverse,
    and with the zero band: the padded inverse's pruned first stage (bit 4) and the truncating
    forward's pruned last stage (bit 8): within 5e-14 of the DFT's scale (measured about 1e-14;
    FP64 transforms reach about 1e-15, FP32 about 1e-6)."""
    assert max(fft_errors[:4]) < 5e-14, fft_errors


def test_register_schedules_at_the_other_double_grid_lengths(fft_errors):
    """45 = 15 x 3, 81 = 9 x 9, 125 = 25 x 5, 405 = 15 x 9 x 3 (the batched kernel's float-float
    energy and coefficient transforms): within 5e-14."""
    assert max(fft_errors[4:8]) < 5e-14, fft_errors


def test_runtime_plan_with_a_generic_prime_radix(fft_errors):
    """The runtime plan (radices 5, 3, 7 and a generic prime 17 from shared memory): within 5e-14."""
    assert max(fft_errors[8:10]) < 5e-14, fft_errors


def test_operator_like_chain_keeps_the_error_at_one_transforms(fft_errors):
    """Three rounds of inverse transform, pointwise coefficient (1 and 1/100) and forward
    transform at lengths 45 and 225 stay within 4e-14 (measured 1.4e-14 and 2.1e-14). Without
    the renormalisation at the stage stores the same chain reaches 4.8e-14 and 6.3e-14: the
    unnormalised low parts grow along the chain."""
    assert max(fft_errors[10:12]) < 4e-14, fft_errors


WARP_NAMES = ("dft_reg_zin", "dft_reg_zout", "pencil_fft_inplace", "pencil_fft_fwd_trunc", "pencil_fft_pad_inv")


def extract_warp_functions():
    """The register-FFT device functions of slab.cuh, cut out by name (template line to the
    matching closing brace): the rest of that header is the GPU-only slab kernel."""
    src = open(os.path.join(CSRC, "slab.cuh")).read()
    out = []
    for name in WARP_NAMES:
        head = "template <typename T, int R>\n__device__ __forceinline__ void " + name + "("
        i = src.index(head)
        j = src.index("{", i)
        depth = 0
        for k in range(j, len(src)):
            if src[k] == "{":
                depth += 1
            elif src[k] == "}":
                depth -= 1
                if depth == 0:
                    break
        out.append(src[i:k + 1])
    return "\n\n".join(out)


WARP_DRIVER = r"""
#include <barrier>
#include <cstdio>
#include <cmath>
#include <thread>
#include <vector>
#include "common.cuh"
namespace homb {
#include "warpfft.inc"
}
using namespace homb;
typedef long double LD;
static const LD PI = 3.141592653589793238462643383279502884L;
static uint64_t st = 0xD1B54A32D192ED03ull;
static double urand() { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return (double)(st >> 11) / 4503599627370496.0 - 1.0; }
static ffloat split(LD v) { const float h = (float)v; return ffloat(h, (float)(v - (LD)h)); }
static LD val(ffloat a) { return (LD)a.hi + (LD)a.lo; }
constexpr int R = 15, M = R * R;

// mode 0: full transform; 1: padded inverse (zero band inputs zero, not read); 2: truncating
// forward (the band's outputs not compared)
static double run(int dir, int mode) {
  std::vector<ffloat2> p(M), Wt(M);
  for (int t = 0; t < M; ++t) {
    const int k = t / R, l = t - k * R;
    const LD ang = -2 * PI * (LD)(l * k) / M;
    Wt[t] = ffloat2{split(std::cos(ang)), split(std::sin(ang))};
  }
  std::vector<LD> xr(M), xi(M);
  for (int n = 0; n < M; ++n) {
    const bool zero = mode == 1 && ZeroBand<R>::in(n / R);
    p[n] = zero ? ffloat2{ffloat(0.f, 0.f), ffloat(0.f, 0.f)} : ffloat2{ffloat(urand()), ffloat(urand())};
    xr[n] = val(p[n].x); xi[n] = val(p[n].y);
  }
  std::barrier<> bar(R);
  g_bar = &bar;
  std::vector<std::thread> lanes;
  for (int l = 0; l < R; ++l)
    lanes.emplace_back([&, l] {
      if (mode == 1) pencil_fft_pad_inv<ffloat, R>(p.data(), l, Wt.data(), true);
      else if (mode == 2) pencil_fft_fwd_trunc<ffloat, R>(p.data(), l, Wt.data(), true);
      else pencil_fft_inplace<ffloat, R>(p.data(), l, Wt.data(), dir, true);
    });
  for (auto& t : lanes) t.join();
  double worst = 0, scale = 0;
  for (int k = 0; k < M; ++k) {
    LD sr = 0, si = 0;
    for (int n = 0; n < M; ++n) {
      const LD ang = dir * 2 * PI * (LD)((long long)n * k % M) / M;
      sr += xr[n] * std::cos(ang) - xi[n] * std::sin(ang);
      si += xr[n] * std::sin(ang) + xi[n] * std::cos(ang);
    }
    scale = std::fmax(scale, (double)std::sqrt(sr * sr + si * si));
    if (mode == 2 && ZeroBand<R>::in(k / R)) continue;
    const LD er = val(p[k].x) - sr, ei = val(p[k].y) - si;
    worst = std::fmax(worst, (double)std::sqrt(er * er + ei * ei));
  }
  return worst / scale;
}

int main() {
  std::printf("%.3e %.3e %.3e %.3e\n", run(-1, 0), run(+1, 0), run(+1, 1), run(-1, 2));
  return 0;
}
"""

WARP_SHIM_EXTRA = r"""
#include <barrier>
inline std::barrier<>* g_bar = nullptr;
inline void __syncwarp() { g_bar->arrive_and_wait(); }
"""


@pytest.fixture(scope="module")
def warp_errors(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("ffloat_warp")
    (d / "cuda_runtime.h").write_text(SHIM + FFT_SHIM_EXTRA + WARP_SHIM_EXTRA)
    (d / "warpfft.inc").write_text(extract_warp_functions())
    (d / "main.cpp").write_text(WARP_DRIVER)
    exe = d / "warpcheck"
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-ffp-contract=off", "-fno-fast-math", "-pthread", "-I", str(d),
                        "-I", CSRC, str(d / "main.cpp"), "-o", str(exe)], capture_output=True, text=True)
    if r.returncode != 0 and "barrier" in r.stderr:
        pytest.skip("no C++20 std::barrier")
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return [float(v) for v in out]


def test_warp_register_ffts_at_225(warp_errors):
    """The lane-group FFT of length 225 = 15 x 15 (two register radix-15 stages, twiddles, the
    exchange through the pencil), forward and inverse, its padded inverse (the zero band's input
    rows not read) and its truncating forward (the band's output rows not computed): within
    5e-14 of the DFT's scale, as the block-level engine."""
    assert max(warp_errors) < 5e-14, warp_errors
