// Operator pass kernels, templated on the precision T and on the transform length MT
// of the pass (MT = 0: runtime length and plan; otherwise a compile-time 3/5-smooth
// length, so that every index divisor in the FFT is a constant). Included by
// passes_f64.cu / passes_f32.cu, which instantiate the launchers for one precision.
//
// Operator (Lemma double-grid, Eq. MBA_GA, structure of Eq. linear_system_primal):
//   C u = Gamma P_N F_M (A_M/|M|) F_M^{-1} Pad(u),  M = 2N-1,
// applied to half-spectrum fields as a chain of passes: inverse transforms along z and y
// with zero padding (k_pencil), a row pass along x (k_xpass: Hermitian-half c2r, pointwise
// coefficient, r2c), the forward y transform with truncation (k_pencil) and the forward z
// transform with truncation, Gamma and the CG partial sums (k_final).
#pragma once
#include <atomic>

#include "attr.cuh"
#include "kernels.cuh"

namespace homb {

constexpr int kPassThreads = 256;
#ifndef HOMB_PASS_SMEM_KB
#define HOMB_PASS_SMEM_KB 48
#endif
constexpr size_t kPassSmemBudget = HOMB_PASS_SMEM_KB * 1024;
constexpr size_t kPassSmemMax = 220 * 1024;

// compile-time lengths with specialised kernels (every M = 2N-1 of the paper's workloads)
#define HOMB_FOR_EACH_M(X) X(45) X(81) X(125) X(225) X(405)

template <typename T>
__device__ __forceinline__ void stage_twiddles(cpx<T>* Ws, const void* W, int M) {
  const cpx<T>* w = reinterpret_cast<const cpx<T>*>(W);
  for (int t = threadIdx.x; t < M; t += blockDim.x) Ws[t] = w[t];
}

template <typename T, int MT>
__device__ __forceinline__ cpx<T>* fft_any(cpx<T>* a, cpx<T>* b, int G, const FftPlan& plan,
                                           const cpx<T>* W, int dir, int prune = 0) {
  if constexpr (MT > 0) return cfft<T, MT>(a, b, G, W, dir, prune);
  else return fft_pencils<T>(a, b, G, plan.M, plan, W, dir);
}

// FP32 and float-float pencils of length 225 = 15 * 15 are transformed by warp-level
// in-register FFTs in place (slab.cuh), with no ping-pong buffer (measured faster there; at 81
// the shared-memory Stockham passes stay ahead). Float-float's long dependent chains of FP32
// operations need the warp FFT's 30 busy lanes of 32: a block-level radix-15 stage keeps
// only M / 15 threads a pencil busy.
template <typename T, int MT> constexpr int warp_fft_r() {
  return (sizeof(T) == 4 || is_ff<T>::value) && MT == 225 ? 15 : 0;
}
template <typename T> inline bool warp_fft_len(int M) { return (sizeof(T) == 4 || is_ff<T>::value) && M == 225; }
// the float-float row pass at 225 runs the warp FFTs too (the FP32 row pass keeps its
// shared-memory stages: the fused slab pass replaces it in 3D)
template <typename T, int MT> constexpr int xpass_warp_r() { return is_ff<T>::value ? warp_fft_r<T, MT>() : 0; }
template <typename T> inline bool xpass_warp_len(int M) { return is_ff<T>::value && M == 225; }

template <typename T, int R>
__device__ __forceinline__ void pencil_fft_inplace(cpx<T>* p, int l, const cpx<T>* Wt, int dir, bool on);
template <typename T, int R>
__device__ __forceinline__ void pencil_fft_pad_inv(cpx<T>* p, int l, const cpx<T>* Wt, bool on);
template <typename T, int R>
__device__ __forceinline__ void pencil_fft_fwd_trunc(cpx<T>* p, int l, const cpx<T>* Wt, bool on);

// twiddles w_M^(l k) at [k][l] for the warp FFT of length R * R
template <typename T, int R>
__device__ __forceinline__ void stage_twiddles_kl(cpx<T>* Wt, const void* W) {
  const cpx<T>* w = reinterpret_cast<const cpx<T>*>(W);
  for (int t = threadIdx.x; t < R * R; t += blockDim.x) {
    const int k = t / R;
    Wt[t] = w[(t - k * R) * k];
  }
}


// G contiguous pencils (stride R*R) in place, R lanes per pencil; ends with __syncthreads.
// mode 1: zero-padded inverse transforms (at most (M+1)/2 nonzero inputs: the zero band of
// the lane layout is not read); mode 2: truncating forward transforms (at most (M+1)/2
// outputs kept: the band's outputs are neither computed nor stored); 0: full transforms.
// true when Nlog frequencies stored around 0 of a length-M pencil (positions 0..half and the
// top Nlog - 1 - half) leave the zero band of the warp FFT's lane layout, positions
// (M+3)/4 .. (3M-3)/4, empty
__host__ __device__ inline bool zero_band_free(int M, int Nlog) {
  const int half = (Nlog - 1) / 2, top = Nlog - 1 - half;
  return half < (M + 3) / 4 && M - top > (3 * M - 3) / 4;
}

template <typename T, int R>
__device__ __forceinline__ void fft_warp_all(cpx<T>* A, int G, const cpx<T>* Wt, int dir, int mode = 0) {
  constexpr int PW = 32 / R;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane / R, l = lane - sub * R;
  const bool act = sub < PW;
  const int slots = (blockDim.x >> 5) * PW;
  for (int g0 = 0; g0 < G; g0 += slots) {
    if (g0 + warp * PW >= G) break;   // warps with no pencil left skip the arithmetic on zeros
    const int g = g0 + warp * PW + sub;
    const bool on = act && g < G;
    cpx<T>* p = A + (size_t)(on ? g : 0) * (R * R);
    if (mode == 1 && dir > 0) pencil_fft_pad_inv<T, R>(p, l, Wt, on);
    else if (mode == 2 && dir < 0) pencil_fft_fwd_trunc<T, R>(p, l, Wt, on);
    else pencil_fft_inplace<T, R>(p, l, Wt, dir, on);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------
// pencil pass along y or z (one component slab per CTA, XC contiguous positions)
// ---------------------------------------------------------------------------------
template <typename T, int MT>
__global__ void __launch_bounds__(kPassThreads) k_pencil(PencilArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int M = MT > 0 ? MT : a.plan.M;
  cpx<T>* Ws = reinterpret_cast<cpx<T>*>(smem);
  cpx<T>* A = Ws + M;
  cpx<T>* B = A + (size_t)a.XC * M;
  const int s = blockIdx.y;
  const int x0 = blockIdx.x * a.XC;
  const int rhs = s / a.slabs_per_rhs;
  if (a.cg != nullptr && !a.cg->active[rhs]) return;
  const int comp = (s / a.slabs_per_comp) % a.C;
  const int XC = min(a.XC, a.X - x0);
  constexpr int WR = warp_fft_r<T, MT>();
  if constexpr (WR > 0) stage_twiddles_kl<T, WR>(Ws, a.W);
  else stage_twiddles<T>(Ws, a.W, M);
  const bool pad = a.dir > 0 && a.Pin != M;
  if (pad) {
    for (int t = threadIdx.x; t < XC * M; t += blockDim.x) A[t] = mk<T>(T(0), T(0));
    __syncthreads();
  }
  cpx<T>* pin = const_cast<cpx<T>*>(reinterpret_cast<const cpx<T>*>(a.in)) + (long long)s * a.in_slab;
  const T beta = a.prologue == 1 ? T(a.cg->beta[rhs]) : T(0);
  const int half = (a.Nlog - 1) / 2;
  // FP32 on long pencils: four independent loads per thread in flight before their
  // shared-memory stores (the stores may alias the loads for the compiler, which would
  // otherwise serialise them); FP64 is bound by its arithmetic pipe and short FP32 pencils
  // by occupancy: they keep one load (and their registers)
  constexpr int U = sizeof(T) == 4 && (MT == 0 || MT >= 125) ? 4 : 1;
  const int nload = a.Pin * a.XC;
  for (int t0 = threadIdx.x; t0 < nload; t0 += U * blockDim.x) {
    cpx<T> v[U], r[U];
    long long gi[U];
    int p[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = t0 + u * (int)blockDim.x;
      p[u] = -1;
      if (t < nload) {
        const int pp = a.fd_XC.div(t);
        const int xx = t - pp * a.XC;
        if (xx < XC) {
          p[u] = pp;
          gi[u] = (long long)pp * a.X + x0 + xx;
          if constexpr (is_ff<T>::value) {
            v[u] = a.in64 ? ff2_from(reinterpret_cast<const double2*>(pin)[gi[u]]) : pin[gi[u]];
          } else {
            v[u] = pin[gi[u]];
          }
          if (a.prologue == 1) r[u] = reinterpret_cast<const cpx<T>*>(a.aux)[(long long)s * a.in_slab + gi[u]];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (p[u] < 0) continue;
      const int xx = (int)(gi[u] - (long long)p[u] * a.X - x0);
      cpx<T> w = v[u];
      if (a.prologue == 1) {
        w = mk<T>(fma(beta, w.x, r[u].x), fma(beta, w.y, r[u].y));
        pin[gi[u]] = w;
      } else if (a.prologue == 2) {
        if (comp == rhs && p[u] == 0 && x0 + xx == 0) w.x += T(1);
      }
      const int pos = pad ? (p[u] <= half ? p[u] : p[u] - a.Nlog + M) : p[u];
      A[xx * M + pos] = w;
    }
  }
  __syncthreads();
  cpx<T>* res;
  if constexpr (WR > 0) {
    // padded inverse / truncating forward: M >= 2 Nlog - 1, so the zero band holds no data
    const bool band = zero_band_free(M, a.Nlog);
    fft_warp_all<T, WR>(A, XC, Ws, a.dir, pad && band ? 1 : (a.dir < 0 && a.Pout != M && band ? 2 : 0));
    res = A;
  } else {
    const bool trunc_ = a.dir < 0 && a.Pout != M;
    const bool zb = zero_band_free(M, a.Nlog);
    const int prune = (pad && prune3_ok(M, half + 1) ? 1 : 0) | (trunc_ && prune3_ok(M, half + 1) ? 2 : 0) |
                      (pad && zb ? 4 : 0) | (trunc_ && zb ? 8 : 0);
    res = fft_any<T, MT>(A, B, XC, a.plan, Ws, a.dir, prune);
  }
  cpx<T>* out = reinterpret_cast<cpx<T>*>(a.out) + (long long)s * a.out_slab;
  const bool trunc = a.dir < 0 && a.Pout != M;
  for (int t = threadIdx.x; t < a.Pout * a.XC; t += blockDim.x) {
    const int i = a.fd_XC.div(t);
    const int xx = t - i * a.XC;
    if (xx >= XC) continue;
    const int pos = trunc ? (i <= half ? i : i - a.Nlog + M) : i;
    // the Nyquist row of an even axis is not computed by a pruned last stage: zero it
    out[(long long)i * a.X + x0 + xx] = trunc && nyquist(i - a.Nlog, a.Nlog) ? mk<T>(T(0), T(0)) : res[xx * M + pos];
  }
}

// ---------------------------------------------------------------------------------
// final forward pass + truncation + projection (+ CG partial p.q or FP64 residual)
// ---------------------------------------------------------------------------------
template <typename T, int MT>
__global__ void __launch_bounds__(kPassThreads) k_final(FinalArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int M = MT > 0 ? MT : a.M;
  const int C = a.C;
  cpx<T>* Ws = reinterpret_cast<cpx<T>*>(smem);
  constexpr int WR = warp_fft_r<T, MT>();
  cpx<T>* A = Ws + M;
  cpx<T>* B = A + (size_t)C * a.XC * M;   // ping-pong half (not allocated for the warp FFT)
  double* red = reinterpret_cast<double*>(WR > 0 ? B : B + (size_t)C * a.XC * M);
  const int rhs = blockIdx.y;
  if (a.cg != nullptr && !a.cg->active[rhs]) return;
  const int x0 = blockIdx.x * a.XC;
  const int XC = min(a.XC, a.X - x0);
  if constexpr (WR > 0) stage_twiddles_kl<T, WR>(Ws, a.W);
  else stage_twiddles<T>(Ws, a.W, M);
  const cpx<T>* in = reinterpret_cast<const cpx<T>*>(a.in) + (long long)rhs * C * a.in_comp;
  const int per = M * a.XC;
  // FP32 on long pencils: four independent read-only loads per thread in flight before their
  // shared-memory stores; FP64 and short FP32 pencils keep one
  constexpr int U = sizeof(T) == 4 && (MT == 0 || MT >= 125) ? 4 : 1;
  for (int t0 = threadIdx.x; t0 < C * per; t0 += U * blockDim.x) {
    cpx<T> v[U];
    int dst[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = t0 + u * (int)blockDim.x;
      dst[u] = -1;
      if (t < C * per) {
        const int g = a.fd_per.div(t);
        const int rem = t - g * per;
        const int p = a.fd_XC.div(rem);
        const int xx = rem - p * a.XC;
        if (xx < XC) {
          dst[u] = (g * XC + xx) * M + p;
          const cpx<T>* src = in + (long long)g * a.in_comp + (long long)p * a.X + x0 + xx;
          if constexpr (is_ff<T>::value) v[u] = *src;
          else v[u] = __ldg(src);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (dst[u] >= 0) A[dst[u]] = v[u];
  }
  __syncthreads();
  cpx<T>* res;
  if constexpr (WR > 0) {
    fft_warp_all<T, WR>(A, C * XC, Ws, -1, a.Nlog < M && zero_band_free(M, a.Nlog) ? 2 : 0);
    res = A;
  } else {
    res = fft_any<T, MT>(A, B, C * XC, a.plan, Ws, -1,
                         (prune3_ok(M, (a.Nlog - 1) / 2 + 1) ? 2 : 0) |
                             (a.Nlog < M && zero_band_free(M, a.Nlog) ? 8 : 0));
  }
  cpx<T>* out = reinterpret_cast<cpx<T>*>(a.out) + (long long)rhs * C * a.out_comp;
  const cpx<T>* pdir = (a.cg && a.aux) ? reinterpret_cast<const cpx<T>*>(a.aux) + (long long)rhs * C * a.out_comp
                                       : nullptr;
  const cpx<T>* bsub = a.bsub ? reinterpret_cast<const cpx<T>*>(a.bsub) + (long long)rhs * C * a.out_comp
                              : nullptr;
  const int half = (a.Nlog - 1) / 2;
  // float-float: the reciprocal cell lengths once per thread, so that xi = k / Y is one
  // float-float product per component (k is exact in FP32)
  T invYf[3];
  if constexpr (is_ff<T>::value) {
#pragma unroll
    for (int c = 0; c < 3; ++c) invYf[c] = T(a.invY[c]);
  }
  double acc = 0.0;
  // FP32: the p.Cp terms of up to 8 points in FP32, their sums in FP64 (FP64 instructions
  // issue at a small fraction of the FP32 rate)
  float run = 0.f;
  int cnt = 0;
  for (int t = threadIdx.x; t < a.Nlog * a.XC; t += blockDim.x) {
    const int i = a.fd_XC.div(t);
    const int xx = t - i * a.XC;
    if (xx >= XC) continue;
    const int kl = i <= half ? i : i - a.Nlog;
    const int pos = kl < 0 ? kl + M : kl;
    const int x = x0 + xx;
    int kx, ky, kz;
    if (a.d == 3) {
      const int iy = a.fd_Nh.div(x);
      kx = x - iy * a.Nh;
      ky = sfreq(iy, a.Ny);
      kz = kl;
    } else {
      kx = x;
      ky = kl;
      kz = 0;
    }
    const long long oi = (long long)i * a.X + x;
    // FP32: the CG direction p is fetched first, so that its latency overlaps the projection
    // (issued after the stores below, the loads would wait for them); FP64, bound by its
    // arithmetic pipe, keeps its registers and loads p after the stores
    cpx<T> pv[3];
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
        pv[c] = pdir && c < C ? __ldg(pdir + (long long)c * a.out_comp + oi) : mk<T>(T(0), T(0));
    }
    cpx<T> u[3];
    // Nyquist rows of even axes are not computed by a pruned last stage: write zeros there
    const bool nyq = nyquist(kl, a.Nlog) || (a.d == 3 && nyquist(ky, a.Ny));
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = c < C && !nyq ? res[(c * XC + xx) * M + pos] : mk<T>(T(0), T(0));
    if (a.project) {
      T xi[3];
      if constexpr (is_ff<T>::value) {
        xi[0] = T((float)kx, 0.f) * invYf[0];
        xi[1] = T((float)ky, 0.f) * invYf[1];
        xi[2] = T((float)kz, 0.f) * invYf[2];
      } else {
        xi[0] = T(kx * a.invY[0]);
        xi[1] = T(ky * a.invY[1]);
        xi[2] = T(kz * a.invY[2]);
      }
      T n2 = T(0);
      cpx<T> dot = mk<T>(T(0), T(0));
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (c < C) {
          n2 = fma(xi[c], xi[c], n2);
          dot = mk<T>(fma(xi[c], u[c].x, dot.x), fma(xi[c], u[c].y, dot.y));
        }
      if (n2 == T(0)) {
#pragma unroll
        for (int c = 0; c < 3; ++c) u[c] = mk<T>(T(0), T(0));
      } else {
        const T inv = T(1) / n2;
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (c < C) {
            const cpx<T> ge = mk<T>(xi[c] * dot.x * inv, xi[c] * dot.y * inv);
            u[c] = a.project == 1 ? ge : sub<T>(u[c], ge);
          }
      }
    }
    if constexpr (is_ff<T>::value) {
      // float-float passes write FP64: C u, or the residual b - C u with b in FP64 (no CG
      // direction: the launcher rejects aux)
      const double2* b64 = reinterpret_cast<const double2*>(bsub);
      double2* o64 = reinterpret_cast<double2*>(out);
      double sq = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (c < C) {
          double2 w = ff2_to(u[c]);
          if (b64) {
            const double2 bb = b64[(long long)c * a.out_comp + oi];
            w = make_double2(bb.x - w.x, bb.y - w.y);
            sq += w.x * w.x + w.y * w.y;
          }
          o64[(long long)c * a.out_comp + oi] = w;
        }
      if (b64) acc += (kx == 0 ? 1.0 : 2.0) * sq;
      continue;
    }
    if (bsub) {
      double sq = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (c < C) {
          u[c] = sub<T>(bsub[(long long)c * a.out_comp + oi], u[c]);
          sq += (double)u[c].x * (double)u[c].x + (double)u[c].y * (double)u[c].y;
        }
      acc += (kx == 0 ? 1.0 : 2.0) * sq;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < C) out[(long long)c * a.out_comp + oi] = u[c];
    if (pdir) {
      if constexpr (sizeof(T) == 4) {
        float sq = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (c < C) sq = fmaf(pv[c].x, u[c].x, fmaf(pv[c].y, u[c].y, sq));
        run = fmaf(kx == 0 ? 1.f : 2.f, sq, run);
        if (++cnt == 8) {
          acc += (double)run;
          run = 0.f;
          cnt = 0;
        }
      } else {
        double sq = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (c < C) {
            pv[c] = pdir[(long long)c * a.out_comp + oi];
            sq += (double)pv[c].x * (double)u[c].x + (double)pv[c].y * (double)u[c].y;
          }
        acc += (kx == 0 ? 1.0 : 2.0) * sq;
      }
    }
  }
  acc += (double)run;
  if (a.partial) {
    const double sum = block_sum(acc, red);
    if (threadIdx.x == 0) a.partial[rhs * a.partial_ld + blockIdx.x] = sum;
  }
}

}  // namespace homb
#include "zpipe.cuh"
namespace homb {

// ---------------------------------------------------------------------------------
// row pass along x: Hermitian-half rows, two real rows packed per complex FFT
// ---------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void apply_coef(const T* coef, long long gi, long long cstride, int ncomp,
                                           int d, const T* u, T* v, T scale) {
  if (ncomp == 1) {
    const T a = coef[gi] * scale;
    for (int c = 0; c < d; ++c) v[c] = a * u[c];
  } else if (d == 2) {
    const T a11 = coef[gi] * scale, a22 = coef[gi + cstride] * scale, a12 = coef[gi + 2 * cstride] * scale;
    v[0] = fma(a11, u[0], a12 * u[1]);
    v[1] = fma(a12, u[0], a22 * u[1]);
  } else {
    const T a11 = coef[gi] * scale, a22 = coef[gi + cstride] * scale, a33 = coef[gi + 2 * cstride] * scale;
    const T a23 = coef[gi + 3 * cstride] * scale, a13 = coef[gi + 4 * cstride] * scale,
            a12 = coef[gi + 5 * cstride] * scale;
    v[0] = fma(a11, u[0], fma(a12, u[1], a13 * u[2]));
    v[1] = fma(a12, u[0], fma(a22, u[1], a23 * u[2]));
    v[2] = fma(a13, u[0], fma(a23, u[1], a33 * u[2]));
  }
}

// mode-0 row pass with warp-owned register FFTs (float-float at M = R * R): the pair
// pencils Z = X_a + i X_b are formed straight from the global rows (Z(k) and Z(M - k) from
// X_a(k), X_b(k): no staging copy), transformed in place, multiplied by the coefficient,
// transformed back and split. A: [npair][M] after the twiddles Ws [R][R].
template <typename T, int R>
__device__ __forceinline__ void xpass_warp(const XArgs& a, cpx<T>* Ws, cpx<T>* A, int p0, int YB, int rhs) {
  constexpr int M = R * R;
  const int rpp = a.fd_rpp.d;
  const int nrow = YB * rpp;
  const int npair = (nrow + 1) / 2;
  const int Nin = a.Nin;
  const cpx<T>* in = reinterpret_cast<const cpx<T>*>(a.in);
  auto row_off = [&](int row) -> long long {
    const int yy = a.fd_rpp.div(row);
    return (long long)(rhs * a.C + row - yy * rpp) * a.comp_stride + (long long)(p0 + yy) * Nin;
  };
  stage_twiddles_kl<T, R>(Ws, a.W);
  const bool bin = zero_band_free(M, 2 * Nin - 1);
  for (int t = threadIdx.x; t < npair * Nin; t += blockDim.x) {
    const int pp = a.fd_Nin.div(t);
    const int k = t - pp * Nin;
    const int r0 = 2 * pp;
    cpx<T> xa = in[row_off(r0) + k];
    cpx<T> xb = r0 + 1 < nrow ? in[row_off(r0 + 1) + k] : mk<T>(T(0), T(0));
    if (k == 0) {
      xa.y = T(0);
      xb.y = T(0);
    }
    cpx<T>* z = A + (size_t)pp * M;
    z[k] = mk<T>(xa.x - xb.y, xa.y + xb.x);                    // X_a(k) + i X_b(k)
    if (k > 0) z[M - k] = mk<T>(xa.x + xb.y, xb.x - xa.y);     // conj(X_a(k)) + i conj(X_b(k))
  }
  // the positions between the two ends that the inverse reads: zero (with the zero band,
  // the lane rows ZeroBand<R>::lo..hi, positions R lo .. R hi + R - 1, are not read)
  const int gap = M - 2 * Nin + 1;
  for (int t = threadIdx.x; t < npair * gap; t += blockDim.x) {
    const int pp = t / gap;
    const int k = Nin + (t - pp * gap);
    if (!(bin && k >= R * ZeroBand<R>::lo && k < R * (ZeroBand<R>::hi + 1))) A[(size_t)pp * M + k] = mk<T>(T(0), T(0));
  }
  __syncthreads();
  fft_warp_all<T, R>(A, npair, Ws, +1, bin ? 1 : 0);
  const T* coef = reinterpret_cast<const T*>(a.coef);
  const long long cstride = (long long)a.planes * M;
  const int C = a.C;
  const T scale = T(a.scale);
  for (int t = threadIdx.x; t < YB * M; t += blockDim.x) {
    const int yy = t / M;
    const int x = t - yy * M;
    T u[3], v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < C) {
        const int row = yy * C + c;
        const cpx<T> z = A[(row >> 1) * M + x];
        u[c] = (row & 1) ? z.y : z.x;
      }
    apply_coef<T>(coef, (long long)(p0 + yy) * M + x, cstride, a.ncomp, C, u, v, scale);
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < C) {
        const int row = yy * C + c;
        if (row & 1) A[(row >> 1) * M + x].y = v[c];
        else A[(row >> 1) * M + x].x = v[c];
      }
  }
  __syncthreads();
  fft_warp_all<T, R>(A, npair, Ws, -1, zero_band_free(M, 2 * a.Nout - 1) ? 2 : 0);
  cpx<T>* out = reinterpret_cast<cpx<T>*>(a.out);
  const int Nout = a.Nout;
  for (int t = threadIdx.x; t < nrow * Nout; t += blockDim.x) {
    const int row = a.fd_Nout.div(t);
    const int k = t - row * Nout;
    const int pp = row >> 1;
    const cpx<T> zk = A[pp * M + k];
    const cpx<T> zm = A[pp * M + (k == 0 ? 0 : M - k)];
    cpx<T> X;
    if ((row & 1) == 0) X = mk<T>(T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y));
    else X = mk<T>(T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x));
    out[row_off(row) + k] = X;
  }
}

template <typename T, int MT>
__global__ void __launch_bounds__(kPassThreads) k_xpass(XArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int M = MT > 0 ? MT : a.M;
  const int p0 = blockIdx.x * a.YB;
  const int YB = min(a.YB, a.planes - p0);
  int rhs = 0, comp0 = 0;
  const int rpp = a.fd_rpp.d;
  if (a.mode == 0) {
    rhs = blockIdx.y;
    if (a.cg != nullptr && !a.cg->active[rhs]) return;
  } else if (a.mode == 2) {
    comp0 = blockIdx.y;
  }
  constexpr int WX = xpass_warp_r<T, MT>();
  if constexpr (WX > 0) {   // mode 0 only (the launcher rejects the others)
    cpx<T>* Ws = reinterpret_cast<cpx<T>*>(smem);
    xpass_warp<T, WX>(a, Ws, Ws + M, p0, YB, rhs);
    return;
  }
  const int nrow = YB * rpp;
  const int npair = (nrow + 1) / 2;
  const int bufsz = ((a.YB * rpp + 1) / 2) * (M + 1);
  cpx<T>* Ws = reinterpret_cast<cpx<T>*>(smem);
  cpx<T>* A = Ws + M;
  cpx<T>* B = A + bufsz;
  double* red = reinterpret_cast<double*>(B + bufsz);
  const int Nin = a.Nin;
  const cpx<T>* in = reinterpret_cast<const cpx<T>*>(a.in);
  auto row_off = [&](int row) -> long long {
    const int yy = a.fd_rpp.div(row);
    const int rem = row - yy * rpp;
    const int f = a.mode == 0 ? rhs * a.C + rem : (a.mode == 1 ? rem : comp0);
    return (long long)f * a.comp_stride + (long long)(p0 + yy) * Nin;
  };
  // stage the rows
  for (int t = threadIdx.x; t < nrow * Nin; t += blockDim.x) {
    const int row = a.fd_Nin.div(t);
    const int k = t - row * Nin;
    B[t] = in[row_off(row) + k];
  }
  stage_twiddles<T>(Ws, a.W, M);
  __syncthreads();
  // Z(k) = X_a(k) + i X_b(k) over the full length-M spectrum (Hermitian extension)
  for (int t = threadIdx.x; t < npair * M; t += blockDim.x) {
    const int pp = t / M;
    const int k = t - pp * M;
    cpx<T> z[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = 2 * pp + h;
      cpx<T> v = mk<T>(T(0), T(0));
      if (row < nrow) {
        if (k < Nin) {
          v = B[row * Nin + k];
          if (k == 0) v.y = T(0);
        } else if (k > M - Nin) {
          v = conj_<T>(B[row * Nin + (M - k)]);
        }
      }
      z[h] = v;
    }
    A[pp * M + k] = mk<T>(z[0].x - z[1].y, z[0].y + z[1].x);
  }
  __syncthreads();
  cpx<T>* res = fft_any<T, MT>(A, B, npair, a.plan, Ws, +1,
                               a.mode != 2 ? ((prune3_ok(M, Nin) ? 1 : 0) | (zero_band_free(M, 2 * Nin - 1) ? 4 : 0))
                                           : 0);
  cpx<T>* oth = res == A ? B : A;
  const T* coef = reinterpret_cast<const T*>(a.coef);
  const long long cstride = (long long)a.planes * M;
  if (a.mode == 0) {
    const int C = a.C;
    const T scale = T(a.scale);
    for (int t = threadIdx.x; t < YB * M; t += blockDim.x) {
      const int yy = t / M;
      const int x = t - yy * M;
      T u[3], v[3];
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (c < C) {
          const int row = yy * C + c;
          const cpx<T> z = res[(row >> 1) * M + x];
          u[c] = (row & 1) ? z.y : z.x;
        }
      apply_coef<T>(coef, (long long)(p0 + yy) * M + x, cstride, a.ncomp, C, u, v, scale);
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (c < C) {
          const int row = yy * C + c;
          if (row & 1) res[(row >> 1) * M + x].y = v[c];
          else res[(row >> 1) * M + x].x = v[c];
        }
    }
    __syncthreads();
    cpx<T>* r2 = fft_any<T, MT>(res, oth, npair, a.plan, Ws, -1,
                                (prune3_ok(M, a.Nout) ? 2 : 0) | (zero_band_free(M, 2 * a.Nout - 1) ? 8 : 0));
    cpx<T>* out = reinterpret_cast<cpx<T>*>(a.out);
    const int Nout = a.Nout;
    for (int t = threadIdx.x; t < nrow * Nout; t += blockDim.x) {
      const int row = a.fd_Nout.div(t);
      const int k = t - row * Nout;
      const int pp = row >> 1;
      const cpx<T> zk = r2[pp * M + k];
      const cpx<T> zm = r2[pp * M + (k == 0 ? 0 : M - k)];
      cpx<T> X;
      if ((row & 1) == 0) X = mk<T>(T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y));
      else X = mk<T>(T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x));
      out[row_off(row) + k] = X;
    }
  } else if (a.mode == 1) {
    const int R = a.R, C = a.C;
    double acc[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) acc[i] = 0.0;
    for (int t = threadIdx.x; t < YB * M; t += blockDim.x) {
      const int yy = t / M;
      const int x = t - yy * M;
      T u[3][3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (r < R && c < C) {
            const int row = (yy * R + r) * C + c;
            const cpx<T> z = res[(row >> 1) * M + x];
            u[r][c] = (row & 1) ? z.y : z.x;
          }
#pragma unroll
      for (int sidx = 0; sidx < 3; ++sidx)
        if (sidx < R) {
          T v[3];
          apply_coef<T>(coef, (long long)(p0 + yy) * M + x, cstride, a.ncomp, C, u[sidx], v, T(1));
#pragma unroll
          for (int r = 0; r < 3; ++r)
            if (r < R) {
              double e = 0.0;
#pragma unroll
              for (int c = 0; c < 3; ++c)
                if (c < C) e += (double)u[r][c] * (double)v[c];
              acc[r * 3 + sidx] += e;
            }
        }
    }
    for (int r = 0; r < R; ++r)
      for (int sidx = 0; sidx < R; ++sidx) {
        const double v = block_sum(acc[r * 3 + sidx], red);
        if (threadIdx.x == 0) a.partial[(long long)blockIdx.x * R * R + r * R + sidx] = v;
      }
  } else {
    T* out = reinterpret_cast<T*>(a.out);
    for (int t = threadIdx.x; t < YB * M; t += blockDim.x) {
      const int yy = t / M;
      const int x = t - yy * M;
      const cpx<T> z = res[(yy >> 1) * M + x];
      out[((long long)comp0 * a.planes + p0 + yy) * M + x] = (yy & 1) ? z.y : z.x;
    }
  }
}

template <typename T, int MT>
__global__ void __launch_bounds__(kPassThreads) k_fft_batch(const cpx<T>* in, cpx<T>* out, int M_, int howmany,
                                                             int G, int dir, const void* W, FftPlan plan) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int M = MT > 0 ? MT : M_;
  cpx<T>* Ws = reinterpret_cast<cpx<T>*>(smem);
  cpx<T>* A = Ws + M;
  cpx<T>* B = A + (size_t)G * M;
  const int g0 = blockIdx.x * G;
  const int Ge = min(G, howmany - g0);
  stage_twiddles<T>(Ws, W, M);
  for (int t = threadIdx.x; t < Ge * M; t += blockDim.x) A[t] = in[(long long)g0 * M + t];
  __syncthreads();
  cpx<T>* res = fft_any<T, MT>(A, B, Ge, plan, Ws, dir);
  for (int t = threadIdx.x; t < Ge * M; t += blockDim.x) out[(long long)g0 * M + t] = res[t];
}

// ---------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------
template <typename T> int pencil_xc(int M, int X, int C) {
  const size_t sz = sizeof(cpx<T>);
  const size_t fixed = M * sz + 512;
  if (warp_fft_len<T>(M)) {
    // warp FFTs: one round of the CTA's lane groups (2 pencils a warp), as many positions as
    // fill it (a second, partial round left most warps idle: measured 1.4 ms slower a step
    // on the 16-ball cell's z inverse, and also with two full rounds)
    const long long slots = (kPassThreads / 32) * (32 / 15);
    const size_t per1 = (size_t)C * M * sz;
    long long xc = slots / C > 1 ? slots / C : 1;
    while (xc > 1 && fixed + (size_t)xc * per1 > kPassSmemMax) --xc;
    if (fixed + (size_t)xc * per1 > kPassSmemMax) return 0;
    if (xc > X) xc = X;
    const long long nch = (X + xc - 1) / xc;
    return (int)((X + nch - 1) / nch);
  }
  const size_t per = 2 * (size_t)C * M * sz;
  long long xc = (long long)((kPassSmemBudget > fixed ? kPassSmemBudget - fixed : 0) / per);
  if (xc < 1) xc = (fixed + per <= kPassSmemMax) ? 1 : 0;
  if (xc > 32) xc = 32;
  if (xc > X) xc = X;
  if (xc >= 1) {   // balance the chunks: the same number of chunks, as equal as possible
    const long long nch = (X + xc - 1) / xc;
    xc = (X + nch - 1) / nch;
  }
  if (xc > 1 && !warp_fft_len<T>(M)) {
    // among balanced chunk sizes, the fewest thread rounds per radix stage over all chunks
    // (each CTA does xc * C * M / r butterflies per stage on kPassThreads threads, r the
    // smallest radix), plus half a round of fixed work per CTA; ties keep the larger chunk
    int r = 2;
    while (r < M && M % r) ++r;
    const long long bfl = (long long)(M / r) * C;
    double best = 1e300;
    long long bx = xc;
    for (long long c = xc; c >= 1; --c) {
      const long long nch = (X + c - 1) / c;
      if ((X + nch - 1) / nch != c) continue;
      const double cost = (double)nch * ((double)((c * bfl + kPassThreads - 1) / kPassThreads) + 0.5);
      if (cost < best - 1e-9) {
        best = cost;
        bx = c;
      }
    }
    xc = bx;
  }
  return (int)xc;
}

template <typename T> int xpass_yb(int M, int rpp, int planes) {
  const size_t sz = sizeof(cpx<T>);
  const size_t fixed = M * sz + 512;
  if (xpass_warp_len<T>(M)) {
    // warp FFTs: at most one round of pair pencils, 2 per warp (30 of 32 lanes), and one
    // buffer of pairs (no staging copy, no ping-pong)
    long long yb = (2LL * (kPassThreads / 32) * (32 / 15)) / rpp;
    if (yb < 1) yb = 1;
    while (yb > 1 && fixed + (size_t)((yb * rpp + 1) / 2) * M * sz > kPassSmemMax) --yb;
    if (fixed + (size_t)((yb * rpp + 1) / 2) * M * sz > kPassSmemMax) return 0;
    if (yb > planes) yb = planes;
    const long long nch = (planes + yb - 1) / yb;
    return (int)((planes + nch - 1) / nch);
  }
  const long long npmax =
      kPassSmemBudget > fixed ? (long long)((kPassSmemBudget - fixed) / (2 * (size_t)(M + 1) * sz)) : 0;
  long long yb = (2 * npmax) / rpp;
  if (yb < 1) {
    const size_t need = fixed + 2 * (size_t)((rpp + 1) / 2) * (M + 1) * sz;
    yb = need <= kPassSmemMax ? 1 : 0;
  }
  if (yb > 32) yb = 32;
  if (yb > planes) yb = planes;
  if (yb >= 1) {
    const long long nch = (planes + yb - 1) / yb;
    yb = (planes + nch - 1) / nch;
  }
  return (int)yb;
}

template <typename T, int MT> cudaError_t launch_pencil_m(PencilArgs a, cudaStream_t s) {
  const size_t bufs = warp_fft_r<T, MT>() > 0 ? 1 : 2;
  const size_t smem = (size_t)a.plan.M * sizeof(cpx<T>) * (1 + bufs * (size_t)a.XC);
  static std::atomic<int> cache[kAttrDevices] = {};
  cudaError_t e = smem_attr(k_pencil<T, MT>, smem, cache);
  if (e != cudaSuccess) return e;
  dim3 grid((a.X + a.XC - 1) / a.XC, a.nslab);
  k_pencil<T, MT><<<grid, kPassThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int MT> cudaError_t launch_final_m(FinalArgs a, cudaStream_t s) {
  const size_t bufs = warp_fft_r<T, MT>() > 0 ? 1 : 2;
  const size_t smem = (size_t)a.M * sizeof(cpx<T>) * (1 + bufs * (size_t)a.C * a.XC) + 32 * sizeof(double);
  static std::atomic<int> cache[kAttrDevices] = {};
  cudaError_t e = smem_attr(k_final<T, MT>, smem, cache);
  if (e != cudaSuccess) return e;
  dim3 grid((a.X + a.XC - 1) / a.XC, a.nrhs);
  k_final<T, MT><<<grid, kPassThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int MT> cudaError_t launch_xpass_m(XArgs a, int grid_y, cudaStream_t s) {
  const int rpp = a.mode == 0 ? a.C : (a.mode == 1 ? a.R * a.C : 1);
  const int npair = (a.YB * rpp + 1) / 2;
  constexpr bool warp = xpass_warp_r<T, MT>() > 0;
  if (warp && a.mode != 0) return cudaErrorInvalidValue;
  const size_t smem = warp ? (size_t)a.M * sizeof(cpx<T>) * (1 + (size_t)npair)
                           : (size_t)a.M * sizeof(cpx<T>) + 2 * (size_t)npair * (a.M + 1) * sizeof(cpx<T>) +
                                 32 * sizeof(double);
  static std::atomic<int> cache[kAttrDevices] = {};
  cudaError_t e = smem_attr(k_xpass<T, MT>, smem, cache);
  if (e != cudaSuccess) return e;
  dim3 grid((a.planes + a.YB - 1) / a.YB, grid_y);
  k_xpass<T, MT><<<grid, kPassThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int MT>
cudaError_t launch_fft_batch_m(const void* in, void* out, int M, int howmany, int dir, const void* W,
                               const FftPlan& plan, int G, cudaStream_t s) {
  const size_t smem = (size_t)M * sizeof(cpx<T>) * (1 + 2 * (size_t)G);
  static std::atomic<int> cache[kAttrDevices] = {};
  cudaError_t e = smem_attr(k_fft_batch<T, MT>, smem, cache);
  if (e != cudaSuccess) return e;
  const int blocks = (howmany + G - 1) / G;
  k_fft_batch<T, MT><<<blocks, kPassThreads, smem, s>>>(reinterpret_cast<const cpx<T>*>(in),
                                                        reinterpret_cast<cpx<T>*>(out), M, howmany, G, dir,
                                                        W, plan);
  return cudaGetLastError();
}

// dispatch on the transform length: specialised kernels for the listed lengths
#define HOMB_CASE_PENCIL(m) case m: return launch_pencil_m<T, m>(a, s);
#define HOMB_CASE_FINAL(m) case m: return launch_final_m<T, m>(a, s);
#define HOMB_CASE_XPASS(m) case m: return launch_xpass_m<T, m>(a, grid_y, s);
#define HOMB_CASE_FFT(m) case m: return launch_fft_batch_m<T, m>(in, out, M, howmany, dir, W, plan, G, s);

template <typename T> cudaError_t launch_zpad_pipe(const PencilArgs& a, cudaStream_t s) {
  const size_t smem = zp_pad_smem<T, 15>(a.prologue == 1 ? 2 : 1);
  static std::atomic<int> cache[kAttrDevices] = {};
  cudaError_t e = smem_attr(k_zpad_pipe<T, 15>, zp_pad_smem<T, 15>(2), cache);
  if (e != cudaSuccess) return e;
  k_zpad_pipe<T, 15><<<a.pgrid, kZpThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int XC> cudaError_t launch_final_pipe_xc(const FinalArgs& a, cudaStream_t s) {
  constexpr size_t smem = zp_final_smem<T, 15, XC>();
  static std::atomic<int> cache[kAttrDevices] = {};
  cudaError_t e = smem_attr(k_final_pipe<T, 15, XC>, smem, cache);
  if (e != cudaSuccess) return e;
  k_final_pipe<T, 15, XC><<<a.pgrid, zp_final_threads(XC), smem, s>>>(a);
  return cudaGetLastError();
}
template <typename T> cudaError_t launch_final_pipe(const FinalArgs& a, cudaStream_t s) {
  return a.pxc == 16 ? launch_final_pipe_xc<T, 16>(a, s) : launch_final_pipe_xc<T, 8>(a, s);
}

template <typename T> cudaError_t launch_pencil(const PencilArgs& a0, cudaStream_t s) {
  PencilArgs a = a0;
  a.fd_XC = FastDiv((uint32_t)a.XC);
  if constexpr (sizeof(T) == 4) {
    if (a.pgrid > 0) return launch_zpad_pipe<T>(a, s);
  }
  switch (a.plan.M) {
    HOMB_FOR_EACH_M(HOMB_CASE_PENCIL)
    default: return launch_pencil_m<T, 0>(a, s);
  }
}

template <typename T> cudaError_t launch_final(const FinalArgs& a0, cudaStream_t s) {
  if (is_ff<T>::value && a0.aux != nullptr) return cudaErrorInvalidValue;   // FP64 output only
  FinalArgs a = a0;
  a.fd_XC = FastDiv((uint32_t)a.XC);
  a.fd_per = FastDiv((uint32_t)(a.M * a.XC));
  a.fd_Nh = FastDiv((uint32_t)a.Nh);
  if constexpr (sizeof(T) == 4) {
    if (a.pgrid > 0) return launch_final_pipe<T>(a, s);
  }
  switch (a.M) {
    HOMB_FOR_EACH_M(HOMB_CASE_FINAL)
    default: return launch_final_m<T, 0>(a, s);
  }
}

template <typename T> cudaError_t launch_xpass(const XArgs& a0, int grid_y, cudaStream_t s) {
  XArgs a = a0;
  const int rpp = a.mode == 0 ? a.C : (a.mode == 1 ? a.R * a.C : 1);
  a.fd_rpp = FastDiv((uint32_t)rpp);
  a.fd_Nin = FastDiv((uint32_t)a.Nin);
  a.fd_Nout = FastDiv((uint32_t)(a.Nout > 0 ? a.Nout : 1));
  switch (a.M) {
    HOMB_FOR_EACH_M(HOMB_CASE_XPASS)
    default: return launch_xpass_m<T, 0>(a, grid_y, s);
  }
}

template <typename T>
cudaError_t launch_fft_batch(const void* in, void* out, int M, int howmany, int dir, const void* W,
                             const FftPlan& plan, cudaStream_t s) {
  const int G = pencil_xc<T>(M, howmany, 1);
  if (G < 1) return cudaErrorInvalidValue;
  switch (M) {
    HOMB_FOR_EACH_M(HOMB_CASE_FFT)
    default: return launch_fft_batch_m<T, 0>(in, out, M, howmany, dir, W, plan, G, s);
  }
}

}  // namespace homb
#include "slab.cuh"
namespace homb {

#define HOMB_INST_PASSES(T)                                                           \
  template cudaError_t launch_slab<T>(const SlabArgs&, cudaStream_t);                 \
  template int slab_warps<T>(int, int);                                               \
  template cudaError_t launch_pencil<T>(const PencilArgs&, cudaStream_t);             \
  template cudaError_t launch_final<T>(const FinalArgs&, cudaStream_t);               \
  template cudaError_t launch_xpass<T>(const XArgs&, int, cudaStream_t);              \
  template int pencil_xc<T>(int, int, int);                                           \
  template int xpass_yb<T>(int, int, int);                                            \
  template cudaError_t launch_fft_batch<T>(const void*, void*, int, int, int, const void*, \
                                           const FftPlan&, cudaStream_t);

}  // namespace homb
