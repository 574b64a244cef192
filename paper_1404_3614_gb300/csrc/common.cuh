// Shared device helpers: complex arithmetic, the shared-memory FFT engine,
// deterministic block reductions and the launch-argument structures.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace homb {

template <typename T> struct cplx_t;
template <> struct cplx_t<double> { using type = double2; };
template <> struct cplx_t<float> { using type = float2; };
}  // namespace homb
#include "ffloat.cuh"
namespace homb {
template <> struct cplx_t<ffloat> { using type = ffloat2; };
template <typename T> using cpx = typename cplx_t<T>::type;

template <typename T> __device__ __forceinline__ cpx<T> mk(T x, T y) { cpx<T> r; r.x = x; r.y = y; return r; }
template <typename T> __device__ __forceinline__ cpx<T> add(cpx<T> a, cpx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cpx<T> sub(cpx<T> a, cpx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ cpx<T> scl(cpx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
template <typename T> __device__ __forceinline__ cpx<T> conj_(cpx<T> a) { return mk<T>(a.x, -a.y); }
// a * b
template <typename T> __device__ __forceinline__ cpx<T> mul(cpx<T> a, cpx<T> b) {
  return mk<T>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * (b or conj b)
template <typename T> __device__ __forceinline__ cpx<T> mulc(cpx<T> a, cpx<T> b, bool conjb) {
  T by = conjb ? -b.y : b.y;
  return mk<T>(fma(a.x, b.x, -a.y * by), fma(a.x, by, a.y * b.x));
}
// A value as stored between transform stages: float-float pairs renormalised there (their
// sums and products do not renormalise, and a low part left to grow through a whole chain
// of stages would make the rounding error grow with the square of its depth); FP32 and FP64
// values pass unchanged.
template <typename T> __device__ __forceinline__ cpx<T> st_norm(cpx<T> v) {
  if constexpr (is_ff<T>::value) {
    cpx<T> r;
    r.x = ff_norm(v.x);
    r.y = ff_norm(v.y);
    return r;
  } else {
    return v;
  }
}
// i * a  (s = +1) or -i * a (s = -1)
template <typename T> __device__ __forceinline__ cpx<T> rot(cpx<T> a, int s) {
  return s > 0 ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

constexpr int kMaxRadices = 24;

// Division by a runtime divisor d >= 1 for numerators n < 2^31 with one high multiply:
// q = (umulhi(n, m) + n) >> s, s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1
// (the round-up method of Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994).
struct FastDiv {
  uint32_t d, m, s;
  __host__ __device__ FastDiv() : d(1), m(1), s(0) {}
  __host__ __device__ explicit FastDiv(uint32_t dd) : d(dd ? dd : 1) {
    uint32_t sh = 0;
    while ((1ull << sh) < d) ++sh;
    s = sh;
    m = (uint32_t)((((uint64_t)1 << 32) * (((uint64_t)1 << sh) - d)) / d + 1);
  }
  __device__ __forceinline__ int div(int n) const {
    return (int)((__umulhi((uint32_t)n, m) + (uint32_t)n) >> s);
  }
};

// Compile-time factorisation of a transform length. big = false: radices 5 then 3 (the
// runtime plan's order); big = true: composite radices done in registers (15, 25, 9,
// then 5 and 3), fewer shared-memory stages for the same length.
__host__ __device__ constexpr int cf_radix(int M, int stage, bool big = false) {
  int m = M, idx = 0;
  const int rs_small[5] = {5, 3, 7, 11, 13};
  const int rs_big[5] = {15, 25, 9, 5, 3};
  for (int i = 0; i < 5; ++i) {
    const int r = big ? rs_big[i] : rs_small[i];
    while (m > 1 && m % r == 0) {
      if (idx == stage) return r;
      m /= r;
      ++idx;
    }
  }
  return 0;
}
__host__ __device__ constexpr int cf_nstages(int M, bool big = false) {
  int n = 0;
  while (cf_radix(M, n, big) != 0) ++n;
  return n;
}
__host__ __device__ constexpr int cf_ns(int M, int stage, bool big = false) {
  int p = 1;
  for (int i = 0; i < stage; ++i) p *= cf_radix(M, i, big);
  return p;
}

// Factorised plan of one odd transform length M (Stockham autosort, mixed radix).
struct FftPlan {
  int M;
  int nrad;
  int radix[kMaxRadices];
  int sched;   // compile-time lengths in the batched kernel: 0 precision default,
               // 1 radices 5 and 3, 2 composite register radices 15, 25, 9
};

// ---------------------------------------------------------------------------------
// Small DFT butterflies. dir = -1: forward (w = exp(-2 pi i / r)); dir = +1: inverse.
// The constants are cos/sin of 2 pi/3, 2 pi/5, 4 pi/5.
// ---------------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ void dft3(cpx<T>* v, int dir) {
  const T h = T(0.5);
  const T s3 = T(0.86602540378443864676372317075294);
  cpx<T> t1 = add<T>(v[1], v[2]);
  cpx<T> t2 = mk<T>(fma(-h, t1.x, v[0].x), fma(-h, t1.y, v[0].y));
  cpx<T> t3 = scl<T>(sub<T>(v[1], v[2]), s3);
  v[0] = add<T>(v[0], t1);
  // forward: V1 = t2 - i t3, V2 = t2 + i t3
  cpx<T> it3 = rot<T>(t3, dir > 0 ? 1 : -1);
  v[1] = add<T>(t2, it3);
  v[2] = sub<T>(t2, it3);
}

template <typename T> __device__ __forceinline__ void dft5(cpx<T>* v, int dir) {
  const T c1 = T(0.30901699437494742410229341718282);    // cos(2 pi/5)
  const T c2 = T(-0.80901699437494742410229341718282);   // cos(4 pi/5)
  const T s1 = T(0.95105651629515357211643933337938);    // sin(2 pi/5)
  const T s2 = T(0.58778525229247312916870595463907);    // sin(4 pi/5)
  cpx<T> a1 = add<T>(v[1], v[4]), b1 = sub<T>(v[1], v[4]);
  cpx<T> a2 = add<T>(v[2], v[3]), b2 = sub<T>(v[2], v[3]);
  cpx<T> m1 = mk<T>(fma(c1, a1.x, fma(c2, a2.x, v[0].x)), fma(c1, a1.y, fma(c2, a2.y, v[0].y)));
  cpx<T> m2 = mk<T>(fma(c2, a1.x, fma(c1, a2.x, v[0].x)), fma(c2, a1.y, fma(c1, a2.y, v[0].y)));
  cpx<T> n1 = mk<T>(fma(s1, b1.x, s2 * b2.x), fma(s1, b1.y, s2 * b2.y));
  cpx<T> n2 = mk<T>(fma(s2, b1.x, -s1 * b2.x), fma(s2, b1.y, -s1 * b2.y));
  v[0] = add<T>(v[0], add<T>(a1, a2));
  int s = dir > 0 ? 1 : -1;     // forward: V1 = m1 - i n1
  cpx<T> in1 = rot<T>(n1, s), in2 = rot<T>(n2, s);
  v[1] = add<T>(m1, in1);
  v[4] = sub<T>(m1, in1);
  v[2] = add<T>(m2, in2);
  v[3] = sub<T>(m2, in2);
}

// Compile-time cos / sin of 2 pi p / q from their Taylor series (argument reduced to
// [-pi, pi]); used only for the twiddle constants inside the register DFTs.
__host__ __device__ constexpr double ct_sin_red(double x) {
  double term = x, sum = x;
  for (int n = 1; n < 30; ++n) {
    term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double ct_cos_red(double x) {
  double term = 1.0, sum = 1.0;
  for (int n = 1; n < 30; ++n) {
    term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
    sum += term;
  }
  return sum;
}
// angle 2 pi p / q reduced to (-pi, pi]
__host__ __device__ constexpr double ct_angle(int p, int q) {
  int r = p % q;
  if (r < 0) r += q;
  if (2 * r > q) r -= q;
  return 6.283185307179586476925286766559 * (double)r / (double)q;
}
__host__ __device__ constexpr double ct_cos2pi(int p, int q) { return ct_cos_red(ct_angle(p, q)); }
__host__ __device__ constexpr double ct_sin2pi(int p, int q) { return ct_sin_red(ct_angle(p, q)); }

__host__ __device__ constexpr int ct_first_factor(int R) {
  return R % 3 == 0 ? 3 : (R % 5 == 0 ? 5 : R);
}

// Register DFT of compile-time length R (a product of 3s and 5s): Cooley-Tukey with
// R = R1 * R2, inner DFTs over n1 for each n2, constant twiddles w_R^{n2 k1}, outer
// DFTs over n2; output index k1 + R1 k2. dir = -1 forward, +1 inverse.
template <typename T, int R>
__device__ __forceinline__ void dft_reg(cpx<T>* v, int dir);

template <typename T, int R1, int R2>
__device__ __forceinline__ void dft_ct(cpx<T>* v, int dir) {
  constexpr int R = R1 * R2;
  cpx<T> t[R];
#pragma unroll
  for (int n2 = 0; n2 < R2; ++n2) {
    cpx<T> a[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) a[n1] = v[R2 * n1 + n2];
    dft_reg<T, R1>(a, dir);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      if (n2 * k1 == 0) {
        t[n2 * R1 + k1] = a[k1];
      } else {
        const T c = T(ct_cos2pi(n2 * k1, R)), sn = T(ct_sin2pi(n2 * k1, R));
        const T s = dir > 0 ? sn : -sn;    // w = exp(dir * 2 pi i n2 k1 / R)
        t[n2 * R1 + k1] = mk<T>(fma(a[k1].x, c, -a[k1].y * s), fma(a[k1].x, s, a[k1].y * c));
      }
    }
  }
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    cpx<T> b[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) b[n2] = t[n2 * R1 + k1];
    dft_reg<T, R2>(b, dir);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = b[k2];
  }
}

// Length 15 by the prime-factor (Good-Thomas) map, 15 = 3 * 5 with coprime factors:
// input n = (5 n1 + 3 n2) mod 15, output k = (10 k1 + 6 k2) mod 15, so that
// w_15^(n k) = w_3^(n1 k1) w_5^(n2 k2) and no twiddle multiplications are needed.
template <typename T>
__device__ __forceinline__ void dft15_pfa(cpx<T>* v, int dir) {
  cpx<T> t[15];
#pragma unroll
  for (int n2 = 0; n2 < 5; ++n2) {
    cpx<T> a[3];
#pragma unroll
    for (int n1 = 0; n1 < 3; ++n1) a[n1] = v[(5 * n1 + 3 * n2) % 15];
    dft3<T>(a, dir);
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) t[n2 * 3 + k1] = a[k1];
  }
#pragma unroll
  for (int k1 = 0; k1 < 3; ++k1) {
    cpx<T> b[5];
#pragma unroll
    for (int n2 = 0; n2 < 5; ++n2) b[n2] = t[n2 * 3 + k1];
    dft5<T>(b, dir);
#pragma unroll
    for (int k2 = 0; k2 < 5; ++k2) v[(10 * k1 + 6 * k2) % 15] = b[k2];
  }
}

template <typename T, int R>
__device__ __forceinline__ void dft_reg(cpx<T>* v, int dir) {
  if constexpr (R == 3) {
    dft3<T>(v, dir);
  } else if constexpr (R == 5) {
    dft5<T>(v, dir);
  } else if constexpr (R == 15) {
    dft15_pfa<T>(v, dir);
  } else {
    constexpr int R1 = ct_first_factor(R);
    dft_ct<T, R1, R / R1>(v, dir);
  }
}

// Known zeros of the warp FFTs' transforms of length M = R*R. A zero-padded inverse transform has
// at most N <= (M+1)/2 nonzero inputs: at positions p <= (M-3)/4 and p >= (3M+3)/4 (the y rows
// of the padded slab, the Hermitian x extension, Nh <= (M+3)/4); a truncating forward one
// keeps only the outputs at those positions. In the lane layout p = l + R n of the register
// FFTs, the rows n in [lo, hi] hold only such positions for every lane l: they are never read
// as inputs (inverse) and never computed or stored as outputs (forward).
template <int R> struct ZeroBand {
  static constexpr int M = R * R;
  static constexpr int lo = ((M + 3) / 4 + R - 1) / R;
  static constexpr int hi = ((3 * M - 3) / 4 - (R - 1)) / R;
  static constexpr bool in(int n) { return n >= lo && n <= hi; }
};
static_assert(ZeroBand<15>::lo == 4 && ZeroBand<15>::hi == 10, "zero band of the length-225 transforms");

// DFT3 of (a0, a1, a2) with compile-time zero inputs (Z0, Z1, Z2), same convention as dft3:
// y_k = sum_n a_n w^(n k), w = exp(dir 2 pi i / 3). Inputs marked zero are not read.
template <typename T, bool Z0, bool Z1, bool Z2>
__device__ __forceinline__ void dft3_z(const cpx<T>* a, cpx<T>* y, int dir) {
  const T h = T(0.5);
  const T s3 = (dir > 0 ? T(1) : T(-1)) * T(0.86602540378443864676372317075294);
  if constexpr (!Z0 && Z1 && Z2) {
    y[0] = a[0];
    y[1] = a[0];
    y[2] = a[0];
  } else if constexpr (Z0 && !Z1 && Z2) {   // y1 = w a1, y2 = w^2 a1
    const cpx<T> b = a[1];
    const T mx = -h * b.x, my = -h * b.y;
    y[0] = b;
    y[1] = mk<T>(fma(-s3, b.y, mx), fma(s3, b.x, my));
    y[2] = mk<T>(fma(s3, b.y, mx), fma(-s3, b.x, my));
  } else if constexpr (!Z0 && !Z1 && Z2) {   // y1 = a0 + w a1, y2 = a0 + w^2 a1
    const cpx<T> m = mk<T>(fma(-h, a[1].x, a[0].x), fma(-h, a[1].y, a[0].y));
    y[0] = add<T>(a[0], a[1]);
    y[1] = mk<T>(fma(-s3, a[1].y, m.x), fma(s3, a[1].x, m.y));
    y[2] = mk<T>(fma(s3, a[1].y, m.x), fma(-s3, a[1].x, m.y));
  } else if constexpr (!Z0 && Z1 && !Z2) {   // y1 = a0 + w^2 a2, y2 = a0 + w a2
    const cpx<T> m = mk<T>(fma(-h, a[2].x, a[0].x), fma(-h, a[2].y, a[0].y));
    y[0] = add<T>(a[0], a[2]);
    y[1] = mk<T>(fma(s3, a[2].y, m.x), fma(-s3, a[2].x, m.y));
    y[2] = mk<T>(fma(-s3, a[2].y, m.x), fma(s3, a[2].x, m.y));
  } else if constexpr (Z0 && !Z1 && !Z2) {   // y1 = w a1 + w^2 a2, y2 = w^2 a1 + w a2
    const cpx<T> t = add<T>(a[1], a[2]), dd = sub<T>(a[1], a[2]);
    const T mx = -h * t.x, my = -h * t.y;
    y[0] = t;
    y[1] = mk<T>(fma(-s3, dd.y, mx), fma(s3, dd.x, my));
    y[2] = mk<T>(fma(s3, dd.y, mx), fma(-s3, dd.x, my));
  } else {
    y[0] = a[0];
    y[1] = a[1];
    y[2] = a[2];
    dft3<T>(y, dir);
  }
}

// DFT5 of b computing only the outputs in the compile-time mask KEEP (bit k: output k); the
// others are left unchanged. Same convention as dft5.
template <typename T, int KEEP>
__device__ __forceinline__ void dft5_keep(cpx<T>* v, int dir) {
  const T c1 = T(0.30901699437494742410229341718282);    // cos(2 pi/5)
  const T c2 = T(-0.80901699437494742410229341718282);   // cos(4 pi/5)
  const T s1 = T(0.95105651629515357211643933337938);    // sin(2 pi/5)
  const T s2 = T(0.58778525229247312916870595463907);    // sin(4 pi/5)
  const cpx<T> a1 = add<T>(v[1], v[4]), b1 = sub<T>(v[1], v[4]);
  const cpx<T> a2 = add<T>(v[2], v[3]), b2 = sub<T>(v[2], v[3]);
  const int s = dir > 0 ? 1 : -1;
  cpx<T> o[5];
  if constexpr ((KEEP & 0x12) != 0) {   // outputs 1, 4
    const cpx<T> m1 = mk<T>(fma(c1, a1.x, fma(c2, a2.x, v[0].x)), fma(c1, a1.y, fma(c2, a2.y, v[0].y)));
    const cpx<T> n1 = mk<T>(fma(s1, b1.x, s2 * b2.x), fma(s1, b1.y, s2 * b2.y));
    const cpx<T> in1 = rot<T>(n1, s);
    o[1] = add<T>(m1, in1);
    o[4] = sub<T>(m1, in1);
  }
  if constexpr ((KEEP & 0x0c) != 0) {   // outputs 2, 3
    const cpx<T> m2 = mk<T>(fma(c2, a1.x, fma(c1, a2.x, v[0].x)), fma(c2, a1.y, fma(c1, a2.y, v[0].y)));
    const cpx<T> n2 = mk<T>(fma(s2, b1.x, -s1 * b2.x), fma(s2, b1.y, -s1 * b2.y));
    const cpx<T> in2 = rot<T>(n2, s);
    o[2] = add<T>(m2, in2);
    o[3] = sub<T>(m2, in2);
  }
  if constexpr ((KEEP & 1) != 0) v[0] = add<T>(v[0], add<T>(a1, a2));
#pragma unroll
  for (int k = 1; k < 5; ++k)
    if ((KEEP >> k) & 1) v[k] = o[k];
}

// Length-15 DFT (prime-factor map as dft15_pfa) with the inputs of the zero band (4..10) known
// to be zero: they are not read, and the first-layer DFT3s take their reduced forms.
template <typename T>
__device__ __forceinline__ void dft15_zin(cpx<T>* v, int dir) {
  cpx<T> t[15];
  {
    const cpx<T> a[3] = {v[0], v[0], v[0]};   // n2 = 0: inputs 0, 5, 10
    dft3_z<T, false, true, true>(a, t + 0, dir);
  }
  {
    const cpx<T> a[3] = {v[3], v[3], v[13]};   // n2 = 1: inputs 3, 8, 13
    dft3_z<T, false, true, false>(a, t + 3, dir);
  }
  {
    const cpx<T> a[3] = {v[1], v[11], v[1]};   // n2 = 2: inputs 6, 11, 1
    dft3_z<T, true, false, false>(a, t + 6, dir);
  }
  {
    const cpx<T> a[3] = {v[14], v[14], v[14]};   // n2 = 3: inputs 9, 14, 4
    dft3_z<T, true, false, true>(a, t + 9, dir);
  }
  {
    const cpx<T> a[3] = {v[12], v[2], v[2]};   // n2 = 4: inputs 12, 2, 7
    dft3_z<T, false, false, true>(a, t + 12, dir);
  }
#pragma unroll
  for (int k1 = 0; k1 < 3; ++k1) {
    cpx<T> b[5];
#pragma unroll
    for (int n2 = 0; n2 < 5; ++n2) b[n2] = t[n2 * 3 + k1];
    dft5<T>(b, dir);
#pragma unroll
    for (int k2 = 0; k2 < 5; ++k2) v[(10 * k1 + 6 * k2) % 15] = b[k2];
  }
}

// Length-15 DFT (prime-factor map) computing only the outputs outside the zero band (0..3,
// 11..14); the band's outputs are left undefined.
template <typename T>
__device__ __forceinline__ void dft15_zout(cpx<T>* v, int dir) {
  cpx<T> t[15];
#pragma unroll
  for (int n2 = 0; n2 < 5; ++n2) {
    cpx<T> a[3];
#pragma unroll
    for (int n1 = 0; n1 < 3; ++n1) a[n1] = v[(5 * n1 + 3 * n2) % 15];
    dft3<T>(a, dir);
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) t[n2 * 3 + k1] = a[k1];
  }
  // outputs k = (10 k1 + 6 k2) mod 15 outside 4..10: k1 = 0: k2 in {0, 2, 3} (0, 12, 3);
  // k1 = 1: k2 in {1, 3} (1, 13); k1 = 2: k2 in {1, 2, 4} (11, 2, 14)
  cpx<T> b[5];
#pragma unroll
  for (int n2 = 0; n2 < 5; ++n2) b[n2] = t[n2 * 3 + 0];
  dft5_keep<T, 0x0d>(b, dir);
  v[0] = b[0];
  v[12] = b[2];
  v[3] = b[3];
#pragma unroll
  for (int n2 = 0; n2 < 5; ++n2) b[n2] = t[n2 * 3 + 1];
  dft5_keep<T, 0x0a>(b, dir);
  v[1] = b[1];
  v[13] = b[3];
#pragma unroll
  for (int n2 = 0; n2 < 5; ++n2) b[n2] = t[n2 * 3 + 2];
  dft5_keep<T, 0x16>(b, dir);
  v[11] = b[1];
  v[2] = b[2];
  v[14] = b[4];
}

// Generic compile-time radix R from registers, roots from the length-M table W.
template <typename T, int R>
__device__ __forceinline__ void dftR(cpx<T>* v, const cpx<T>* W, int M, int dir) {
  cpx<T> o[R];
  const int step = M / R;
#pragma unroll
  for (int s = 0; s < R; ++s) {
    cpx<T> acc = v[0];
#pragma unroll
    for (int q = 1; q < R; ++q) acc = add<T>(acc, mulc<T>(v[q], W[((q * s) % R) * step], dir > 0));
    o[s] = acc;
  }
#pragma unroll
  for (int s = 0; s < R; ++s) v[s] = o[s];
}

// One Stockham stage for butterfly j of one pencil (src/dst of length M).
template <typename T, int R>
__device__ __forceinline__ void stage_bfly(const cpx<T>* __restrict__ src, cpx<T>* __restrict__ dst,
                                           int j, int Ns, int M, const cpx<T>* W, int dir) {
  const int nb = M / R;
  const int k = j % Ns;
  cpx<T> v[R];
#pragma unroll
  for (int q = 0; q < R; ++q) v[q] = src[j + q * nb];
  const int tstep = k * (M / (Ns * R));
  if (k) {
#pragma unroll
    for (int q = 1; q < R; ++q) v[q] = mulc<T>(v[q], W[q * tstep], dir > 0);
  }
  if (R == 3) dft3<T>(v, dir);
  else if (R == 5) dft5<T>(v, dir);
  else dftR<T, R>(v, W, M, dir);
  const int base = (j / Ns) * Ns * R + k;
#pragma unroll
  for (int q = 0; q < R; ++q) dst[base + q * Ns] = st_norm<T>(v[q]);
}

// Runtime radix (2 or a prime above 13) straight from shared memory: output s of butterfly j,
// O(R) per output, so that a large prime radix spreads over R threads.
template <typename T>
__device__ void stage_out_generic(const cpx<T>* __restrict__ src, cpx<T>* __restrict__ dst,
                                  int j, int s, int Ns, int M, int R, const cpx<T>* W, int dir) {
  const int nb = M / R;
  const int k = j % Ns;
  const int tstep = k * (M / (Ns * R));
  const int step = M / R;
  const int base = (j / Ns) * Ns * R + k;
  cpx<T> acc = src[j];
  int ws = 0;   // (q * s) mod R, advanced incrementally
  for (int q = 1; q < R; ++q) {
    ws += s;
    if (ws >= R) ws -= R;
    const cpx<T> vq = mulc<T>(src[j + q * nb], W[q * tstep], dir > 0);
    acc = add<T>(acc, mulc<T>(vq, W[ws * step], dir > 0));
  }
  dst[base + s * Ns] = st_norm<T>(acc);
}

// G pencils of length M at a + g*ld (ping-pong with b, same strides). The CTA runs
// all stages; returns the buffer holding the result. Ends with __syncthreads().
template <typename T>
__device__ cpx<T>* fft_pencils(cpx<T>* a, cpx<T>* b, int G, int ld, const FftPlan& plan,
                               const cpx<T>* W, int dir) {
  const int M = plan.M;
  int Ns = 1;
  cpx<T>* src = a;
  cpx<T>* dst = b;
  for (int s = 0; s < plan.nrad; ++s) {
    const int R = plan.radix[s];
    const int nb = M / R;
    if (R == 3 || R == 5 || R == 7 || R == 11 || R == 13) {
      const int total = G * nb;
      for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int g = t / nb;
        const int j = t - g * nb;
        const cpx<T>* sp = src + (size_t)g * ld;
        cpx<T>* dp = dst + (size_t)g * ld;
        switch (R) {
          case 3: stage_bfly<T, 3>(sp, dp, j, Ns, M, W, dir); break;
          case 5: stage_bfly<T, 5>(sp, dp, j, Ns, M, W, dir); break;
          case 7: stage_bfly<T, 7>(sp, dp, j, Ns, M, W, dir); break;
          case 11: stage_bfly<T, 11>(sp, dp, j, Ns, M, W, dir); break;
          default: stage_bfly<T, 13>(sp, dp, j, Ns, M, W, dir); break;
        }
      }
    } else {
      const int per = nb * R;
      const int total = G * per;
      for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int g = t / per;
        const int rem = t - g * per;
        const int j = rem / R;
        const int so = rem - j * R;
        stage_out_generic<T>(src + (size_t)g * ld, dst + (size_t)g * ld, j, so, Ns, M, R, W, dir);
      }
    }
    __syncthreads();
    cpx<T>* t = src; src = dst; dst = t;
    Ns *= R;
  }
  return src;
}

// ---------------------------------------------------------------------------------
// Compile-time length M (product of radices 3 and 5): every divisor is a constant.
// ---------------------------------------------------------------------------------
template <typename T, int M, int R, int Ns>
__device__ __forceinline__ void cbfly(const cpx<T>* __restrict__ src, cpx<T>* __restrict__ dst, int j,
                                      const cpx<T>* W, int dir) {
  constexpr int nb = M / R;
  const int k = j % Ns;
  cpx<T> v[R];
#pragma unroll
  for (int q = 0; q < R; ++q) v[q] = src[j + q * nb];
  if (Ns > 1) {
    constexpr int step = M / (Ns * R);
#pragma unroll
    for (int q = 1; q < R; ++q) v[q] = mulc<T>(v[q], W[q * k * step], dir > 0);
  }
  dft_reg<T, R>(v, dir);
  const int base = (j / Ns) * Ns * R + k;
#pragma unroll
  for (int q = 0; q < R; ++q) dst[base + q * Ns] = st_norm<T>(v[q]);
}

// Radix-3 butterflies of a first stage whose middle inputs are all zero (a zero-padded
// spectrum), and of a last stage whose middle outputs are not needed (a truncated one).
template <typename T>
__device__ __forceinline__ void dft3_mid_in0(cpx<T>* v, int dir) {   // v[1] == 0
  const T h = T(0.5);
  const T s3 = T(0.86602540378443864676372317075294);
  const cpx<T> a = v[0], c = v[2];
  const cpx<T> t2 = mk<T>(fma(-h, c.x, a.x), fma(-h, c.y, a.y));
  const cpx<T> it3 = rot<T>(mk<T>(-s3 * c.x, -s3 * c.y), dir > 0 ? 1 : -1);
  v[0] = add<T>(a, c);
  v[1] = add<T>(t2, it3);
  v[2] = sub<T>(t2, it3);
}
template <typename T>
__device__ __forceinline__ void dft3_skip_out1(cpx<T>* v, int dir) {   // v[1] left undefined
  const T h = T(0.5);
  const T s3 = T(0.86602540378443864676372317075294);
  const cpx<T> t1 = add<T>(v[1], v[2]);
  const cpx<T> t2 = mk<T>(fma(-h, t1.x, v[0].x), fma(-h, t1.y, v[0].y));
  const cpx<T> it3 = rot<T>(scl<T>(sub<T>(v[1], v[2]), s3), dir > 0 ? 1 : -1);
  v[0] = add<T>(v[0], t1);
  v[2] = sub<T>(t2, it3);
}

// prune bit 1: the first stage (radix 3, stride nb = M/3) reads only inputs j and j + 2 nb
// (the inputs j + nb are zero padding); bit 2: the last stage (radix 3) writes only outputs
// base and base + 2 Ns (the outputs base + Ns are truncated away); bits 4 and 8: the same for
// a radix-15 first / last stage and its zero band (q = 4..10 of the 15 inputs / outputs,
// positions 4 M/15 .. 11 M/15 - 1). The caller checks that the padding / truncation covers
// those positions.
template <typename T, int M, int S, bool BIG>
__device__ __forceinline__ cpx<T>* cfft_from(cpx<T>* a, cpx<T>* b, int G, const cpx<T>* W, int dir,
                                             int prune = 0) {
  if constexpr (S >= cf_nstages(M, BIG)) {
    return a;
  } else {
    constexpr int R = cf_radix(M, S, BIG);
    constexpr int Ns = cf_ns(M, S, BIG);
    constexpr int nb = M / R;
    constexpr bool last = S + 1 == cf_nstages(M, BIG);
    if constexpr (R == 3 && S == 0 && !last) {
      if (prune & 1) {
        for (int t = threadIdx.x; t < G * nb; t += blockDim.x) {
          const int g = t / nb;
          const int j = t - g * nb;
          const cpx<T>* src = a + g * M;
          cpx<T> v[3] = {src[j], mk<T>(T(0), T(0)), src[j + 2 * nb]};
          dft3_mid_in0<T>(v, dir);
          cpx<T>* dst = b + g * M;
#pragma unroll
          for (int q = 0; q < 3; ++q) dst[3 * j + q] = st_norm<T>(v[q]);   // Ns = 1: base = 3 j
        }
        __syncthreads();
        return cfft_from<T, M, S + 1, BIG>(b, a, G, W, dir, prune);
      }
    }
    if constexpr (R == 15 && S == 0 && !last) {
      if (prune & 4) {   // radix-15 first stage: inputs j + nb q, q in the zero band, are zero
        for (int t = threadIdx.x; t < G * nb; t += blockDim.x) {
          const int g = t / nb;
          const int j = t - g * nb;
          const cpx<T>* src = a + g * M;
          cpx<T> v[15];
#pragma unroll
          for (int q = 0; q < 15; ++q)
            if (!ZeroBand<15>::in(q)) v[q] = src[j + q * nb];
          dft15_zin<T>(v, dir);
          cpx<T>* dst = b + g * M;
#pragma unroll
          for (int q = 0; q < 15; ++q) dst[15 * j + q] = st_norm<T>(v[q]);   // Ns = 1: base = 15 j
        }
        __syncthreads();
        return cfft_from<T, M, S + 1, BIG>(b, a, G, W, dir, prune);
      }
    }
    if constexpr (R == 15 && last && S > 0) {
      if (prune & 8) {   // radix-15 last stage: outputs base + Ns q, q in the zero band, not needed
        for (int t = threadIdx.x; t < G * nb; t += blockDim.x) {
          const int g = t / nb;
          const int j = t - g * nb;
          const cpx<T>* src = a + g * M;
          const int k = j % Ns;
          cpx<T> v[15];
#pragma unroll
          for (int q = 0; q < 15; ++q) v[q] = src[j + q * nb];
          if (k) {
            constexpr int step = M / (Ns * R);
#pragma unroll
            for (int q = 1; q < 15; ++q) v[q] = mulc<T>(v[q], W[q * k * step], dir > 0);
          }
          dft15_zout<T>(v, dir);
          cpx<T>* dst = b + g * M;
          const int base = (j / Ns) * Ns * R + k;
#pragma unroll
          for (int q = 0; q < 15; ++q)
            if (!ZeroBand<15>::in(q)) dst[base + q * Ns] = st_norm<T>(v[q]);
        }
        __syncthreads();
        return b;
      }
    }
    if constexpr (R == 3 && last && S > 0) {
      if (prune & 2) {
        for (int t = threadIdx.x; t < G * nb; t += blockDim.x) {
          const int g = t / nb;
          const int j = t - g * nb;
          const cpx<T>* src = a + g * M;
          const int k = j % Ns;
          cpx<T> v[3] = {src[j], src[j + nb], src[j + 2 * nb]};
          if (k) {
            constexpr int step = M / (Ns * R);
            v[1] = mulc<T>(v[1], W[k * step], dir > 0);
            v[2] = mulc<T>(v[2], W[2 * k * step], dir > 0);
          }
          dft3_skip_out1<T>(v, dir);
          cpx<T>* dst = b + g * M;
          const int base = (j / Ns) * Ns * R + k;
          dst[base] = st_norm<T>(v[0]);
          dst[base + 2 * Ns] = st_norm<T>(v[2]);
        }
        __syncthreads();
        return b;
      }
    }
    for (int t = threadIdx.x; t < G * nb; t += blockDim.x) {
      const int g = t / nb;
      const int j = t - g * nb;
      cbfly<T, M, R, Ns>(a + g * M, b + g * M, j, W, dir);
    }
    __syncthreads();
    return cfft_from<T, M, S + 1, BIG>(b, a, G, W, dir, prune);
  }
}

// G contiguous pencils of compile-time length M (stride M), ping-pong between a and b.
// FP32 and float-float use the composite register radices (fewer shared-memory passes, and
// no twiddle products inside a prime-factor radix 15); FP64 keeps
// radices 3 and 5, which need the fewest FP64 operations, except at M = 225 = 15 * 15, where
// the radix-15 stages with the zero band pruned (bits 4 and 8) need fewer.
constexpr int kBandM64 = 225;
template <typename T, int M>
__device__ __forceinline__ cpx<T>* cfft(cpx<T>* a, cpx<T>* b, int G, const cpx<T>* W, int dir, int prune = 0) {
  return cfft_from<T, M, 0, (sizeof(T) == 4 || is_ff<T>::value || M == kBandM64)>(a, b, G, W, dir, prune);
}

// Prune bits valid for a length-M transform whose spectrum is nonzero (inverse) or needed
// (forward) only at [0, lo) and (M - lo, M): the middle third of a radix-3 first / last
// stage, [M/3, 2M/3), must lie inside [lo, M - lo].
__host__ __device__ inline bool prune3_ok(int M, int lo) {
  return M % 3 == 0 && M / 3 >= lo && 2 * (M / 3) - 1 <= M - lo;
}

// Deterministic block sum of one double per thread (fixed tree order).
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) s += red[w];
  }
  return s;  // valid in thread 0 only
}

// Frequency of storage index i in FFT order for odd length n.
__device__ __forceinline__ int sfreq(int i, int n) { return i <= (n - 1) / 2 ? i : i - n; }
// The Nyquist frequency k = -n/2 of an even axis: the conforming spaces E_N, J_N of general
// grids exclude it (Def. FD_proj_E: G^E_{N,0}, G^J_{N,0} vanish there), so every N-grid
// field keeps it at zero. Never true on odd axes.
__device__ __forceinline__ bool nyquist(int k, int n) { return (n & 1) == 0 && k == -(n >> 1); }

// Per-side CG scalars (device memory), one slot per right-hand side.
struct CgScalars {
  double rr[3];
  double pq[3];
  double alpha[3];
  double beta[3];
  double tol2[3];    // stop when r.r <= tol2 (per right-hand side)
  double rr_min[3];  // smallest r.r seen (divergence guard of the FP32 inner solves)
  int min_iter[3];   // iteration of the last new minimum of r.r (stagnation guard)
  int active[3];     // 1 while the solve runs
  int iters[3];
  int status[3];     // 0 converged, 1 running / max_iter, 2 stopped by a guard, -2 breakdown
  int guard;         // 1: an FP32 inner solve; breakdown and divergence stop it (status 2)
  int fault;         // 1: a bounded device wait of an operator pass gave up
};

}  // namespace homb
