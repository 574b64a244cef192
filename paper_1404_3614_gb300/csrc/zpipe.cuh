// Persistent, pipelined z passes of the FP32 3D operator at transform length M = 225:
// the zero-padded inverse z transform (with the CG prologue p = r + beta p) and the last
// forward z transform with truncation, Gamma and the CG partial sums p.q. They compute what
// k_pencil and k_final compute for these passes (the same warp FFTs, projection and sums);
// the difference is the schedule. Each CTA walks chunks of pencils blockIdx.x,
// blockIdx.x + gridDim.x, ... and stages the input of its next chunk with asynchronous
// 8-byte copies (cp.async) while it transforms and stores the current one, so that every
// CTA keeps one chunk of loads in flight instead of waiting for each chunk's loads.
//
// Operator (Lemma double-grid, Eq. MBA_GA): C u = Gamma P_N F_M (A_M/|M|) F_M^{-1} Pad(u);
// these kernels are its first (Pad, F^{-1} along z) and last (F along z, P_N, Gamma) passes.
#pragma once
#include <algorithm>

#include "kernels.cuh"

namespace homb {

constexpr int kZpThreads = 384;   // 12 warps: 24 lane groups of 15 lanes, one pencil each
constexpr int kZpPencils = 24;    // pencils of one chunk (one round of the warp FFTs)
constexpr int kZpFinalXC = 8;     // last pass: positions per chunk (x 3 components)
constexpr int kZpPadXC = 24;      // inverse pass: positions per chunk (one component)

__device__ __forceinline__ void zp_cp_async8(void* smem_dst, const void* gsrc) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void zp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void zp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Threads of the last pass with XC positions per chunk (3 XC pencils, two per warp)
constexpr int zp_final_threads(int XC) { return 48 * XC; }
// Shared memory of the two kernels (bytes)
template <typename T, int R, int XC = kZpFinalXC> constexpr size_t zp_final_smem() {
  return sizeof(cpx<T>) * (size_t)(R * R) * (1 + 2 * 3 * XC) + 32 * sizeof(double);
}
template <typename T, int R> constexpr size_t zp_pad_smem(int staged_fields) {
  return sizeof(cpx<T>) * ((size_t)(R * R) * (1 + kZpPencils) + (size_t)staged_fields * ((R * R + 1) / 2) * kZpPadXC);
}

// Last forward z pass. Chunk q: right-hand side q / nxc, positions x0 .. x0 + 7 of the
// Ny * Nh (y, kx) plane, all 3 components: 24 pencils of length M. The input of chunk q + grid
// is copied into the other of two buffers during chunk q's transforms. Each thread owns one
// position (xx = tid % 8) and the rows tid / 8 + 48 k of the output, so its frequency
// decoding is done once per chunk and its loads of the CG direction are issued before the
// transforms. Partial sums: partial[rhs * partial_ld + blockIdx.x] for every rhs < nrhs.
template <typename T, int R, int XC>
__global__ void __launch_bounds__(zp_final_threads(XC), XC <= 8 ? 2 : 1) k_final_pipe(FinalArgs a) {
  constexpr int M = R * R;
  constexpr int C = 3;
  constexpr int G = C * XC;
  constexpr int NT = zp_final_threads(XC);
  constexpr int RS = NT / XC;   // rows per sweep (48)
  constexpr int IT = 3;         // output rows per thread: Nlog <= 3 * 48
  static_assert(G == 2 * (NT / 32), "one pencil per lane group");
  extern __shared__ __align__(16) unsigned char smem[];
  cpx<T>* Wt = reinterpret_cast<cpx<T>*>(smem);
  cpx<T>* buf0 = Wt + M;
  cpx<T>* buf1 = buf0 + G * M;
  double* red = reinterpret_cast<double*>(buf1 + G * M);
  const int tid = threadIdx.x;
  const int nxc = (a.X + XC - 1) / XC;
  const int nq = a.nrhs * nxc;
  stage_twiddles_kl<T, R>(Wt, a.W);
  const int xx = tid & (XC - 1);
  const int r0 = tid / XC;
  auto active = [&](int q) { return a.cg == nullptr || a.cg->active[q / nxc] != 0; };
  auto issue = [&](int q, cpx<T>* buf) {
    const int rhs = q / nxc;
    const int x = (q - rhs * nxc) * XC + xx;
    if (x >= a.X) return;
    const cpx<T>* src = reinterpret_cast<const cpx<T>*>(a.in) + (long long)rhs * C * a.in_comp + x;
#pragma unroll
    for (int c = 0; c < C; ++c)
      for (int row = r0; row < M; row += RS)
        zp_cp_async8(buf + (c * XC + xx) * M + row, src + (long long)c * a.in_comp + (long long)row * a.X);
  };
  const int half = (a.Nlog - 1) / 2;
  double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
  int q = blockIdx.x;
  if (q < nq && active(q)) issue(q, buf0);
  zp_commit();
  for (int it = 0; q < nq; q += gridDim.x, ++it) {
    cpx<T>* cur = (it & 1) ? buf1 : buf0;
    const int qn = q + gridDim.x;
    if (qn < nq && active(qn)) issue(qn, (it & 1) ? buf0 : buf1);
    zp_commit();
    zp_wait<1>();
    __syncthreads();
    if (!active(q)) continue;   // uniform over the CTA; nothing was staged for it
    const int rhs = q / nxc;
    const int x = (q - rhs * nxc) * XC + xx;
    const bool own = x < a.X;
    int kx = 0, ky = 0;
    if (own) {
      const int iy = a.fd_Nh.div(x);
      kx = x - iy * a.Nh;
      ky = sfreq(iy, a.Ny);
    }
    const long long fo = (long long)rhs * C * a.out_comp;
    const cpx<T>* pdir = (a.cg && a.aux) ? reinterpret_cast<const cpx<T>*>(a.aux) + fo : nullptr;
    cpx<T> pv[IT][C];
#pragma unroll
    for (int k = 0; k < IT; ++k) {
      const int i = r0 + RS * k;
#pragma unroll
      for (int c = 0; c < C; ++c)
        pv[k][c] = (pdir && own && i < a.Nlog) ? __ldg(pdir + (long long)c * a.out_comp + (long long)i * a.X + x)
                                               : mk<T>(T(0), T(0));
    }
    fft_warp_all<T, R>(cur, G, Wt, -1, 2);
    cpx<T>* out = reinterpret_cast<cpx<T>*>(a.out) + fo;
    float run = 0.f;
#pragma unroll
    for (int k = 0; k < IT; ++k) {
      const int i = r0 + RS * k;
      if (!own || i >= a.Nlog) continue;
      const int kl = i <= half ? i : i - a.Nlog;
      const int pos = kl < 0 ? kl + M : kl;
      const bool nyq = nyquist(kl, a.Nlog) || nyquist(ky, a.Ny);
      cpx<T> u[C];
#pragma unroll
      for (int c = 0; c < C; ++c) u[c] = nyq ? mk<T>(T(0), T(0)) : cur[(c * XC + xx) * M + pos];
      if (a.project) {
        const T xi[3] = {T(kx * a.invY[0]), T(ky * a.invY[1]), T(kl * a.invY[2])};
        T n2 = T(0);
        cpx<T> dot = mk<T>(T(0), T(0));
#pragma unroll
        for (int c = 0; c < C; ++c) {
          n2 = fma(xi[c], xi[c], n2);
          dot = mk<T>(fma(xi[c], u[c].x, dot.x), fma(xi[c], u[c].y, dot.y));
        }
        if (n2 == T(0)) {
#pragma unroll
          for (int c = 0; c < C; ++c) u[c] = mk<T>(T(0), T(0));
        } else {
          const T inv = T(1) / n2;
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const cpx<T> ge = mk<T>(xi[c] * dot.x * inv, xi[c] * dot.y * inv);
            u[c] = a.project == 1 ? ge : sub<T>(u[c], ge);
          }
        }
      }
      const long long oi = (long long)i * a.X + x;
#pragma unroll
      for (int c = 0; c < C; ++c) out[(long long)c * a.out_comp + oi] = u[c];
      if (pdir) {
        float sq = 0.f;
#pragma unroll
        for (int c = 0; c < C; ++c) sq = fmaf(pv[k][c].x, u[c].x, fmaf(pv[k][c].y, u[c].y, sq));
        run = fmaf(kx == 0 ? 1.f : 2.f, sq, run);
      }
    }
    // FP32 terms of at most 3 points, summed per right-hand side in FP64
    if (rhs == 0) acc0 += (double)run;
    else if (rhs == 1) acc1 += (double)run;
    else acc2 += (double)run;
    __syncthreads();
  }
  if (a.partial) {
    const double accs[3] = {acc0, acc1, acc2};
    for (int r = 0; r < a.nrhs; ++r) {
      const double s = block_sum(accs[r], red);
      if (tid == 0) a.partial[r * a.partial_ld + blockIdx.x] = s;
    }
  }
}

// Zero-padded inverse z pass. Chunk q: slab s = q / nxc (right-hand side s / C, component
// s % C), positions x0 .. x0 + 23 of the Ny * Nh plane: 24 pencils. The Nlog input rows of
// the chunk (and, with the CG prologue, of r) are staged by asynchronous copies issued
// while the previous chunk is transformed and stored; the prologue p = r + beta p then runs
// from shared memory (p is written back), the padded pencils are filled (their zeros only
// outside the zero band, which the padded transform does not read), and the M output rows
// are stored.
template <typename T, int R>
__global__ void __launch_bounds__(kZpThreads, 2) k_zpad_pipe(PencilArgs a) {
  constexpr int M = R * R;
  constexpr int XC = kZpPadXC;
  constexpr int G = XC;
  constexpr int PMAX = (M + 1) / 2;   // staged rows (Nlog <= (M + 1) / 2)
  static_assert(G == kZpPencils, "one pencil per lane group");
  extern __shared__ __align__(16) unsigned char smem[];
  cpx<T>* Wt = reinterpret_cast<cpx<T>*>(smem);
  cpx<T>* P = Wt + M;
  cpx<T>* Sin = P + G * M;            // staged input rows [row][xx]
  cpx<T>* Saux = Sin + PMAX * XC;     // staged r rows (prologue 1)
  const int tid = threadIdx.x;
  const int nxc = (a.X + XC - 1) / XC;
  const int nq = a.nslab * nxc;
  const int Pin = a.Pin;
  const bool with_r = a.prologue == 1;
  stage_twiddles_kl<T, R>(Wt, a.W);
  auto active = [&](int q) { return a.cg == nullptr || a.cg->active[(q / nxc) / a.slabs_per_rhs] != 0; };
  auto issue = [&](int q) {
    const int s = q / nxc;
    const int x0 = (q - s * nxc) * XC;
    const cpx<T>* pin = reinterpret_cast<const cpx<T>*>(a.in) + (long long)s * a.in_slab + x0;
    const cpx<T>* rin = reinterpret_cast<const cpx<T>*>(a.aux) + (long long)s * a.in_slab + x0;
    for (int e = tid; e < Pin * XC; e += kZpThreads) {
      const int row = e / XC, xx = e - row * XC;
      if (x0 + xx >= a.X) continue;
      const long long gi = (long long)row * a.X + xx;
      zp_cp_async8(Sin + e, pin + gi);
      if (with_r) zp_cp_async8(Saux + e, rin + gi);
    }
  };
  const int half = (a.Nlog - 1) / 2;
  int q = blockIdx.x;
  if (q < nq && active(q)) issue(q);
  zp_commit();
  for (; q < nq; q += gridDim.x) {
    zp_wait<0>();
    __syncthreads();
    const bool on = active(q);
    const int s = q / nxc;
    const int x0 = (q - s * nxc) * XC;
    if (on) {
      const int rhs = s / a.slabs_per_rhs;
      const int comp = (s / a.slabs_per_comp) % a.C;
      const T beta = with_r ? T(a.cg->beta[rhs]) : T(0);
      cpx<T>* pin = const_cast<cpx<T>*>(reinterpret_cast<const cpx<T>*>(a.in)) + (long long)s * a.in_slab + x0;
      for (int e = tid; e < Pin * XC; e += kZpThreads) {
        const int row = e / XC, xx = e - row * XC;
        if (x0 + xx >= a.X) continue;
        cpx<T> w = Sin[e];
        if (with_r) {
          const cpx<T> r = Saux[e];
          w = mk<T>(fma(beta, w.x, r.x), fma(beta, w.y, r.y));
          pin[(long long)row * a.X + xx] = w;
        } else if (a.prologue == 2) {
          if (comp == rhs && row == 0 && x0 + xx == 0) w.x += T(1);
        }
        const int pos = row <= half ? row : row - a.Nlog + M;
        P[xx * M + pos] = w;
      }
      // padding positions that the transform reads: those outside its zero band (the band's
      // rows are not read); the previous chunk's outputs are there
      const int gapn = M - a.Nlog;
      for (int e = tid; e < G * gapn; e += kZpThreads) {
        const int g = e / gapn;
        const int pos = half + 1 + (e - g * gapn);
        if (!ZeroBand<R>::in(pos / R)) P[g * M + pos] = mk<T>(T(0), T(0));
      }
    }
    __syncthreads();   // staging consumed: the next chunk's copies may land
    const int qn = q + gridDim.x;
    if (qn < nq && active(qn)) issue(qn);
    zp_commit();
    if (!on) continue;
    fft_warp_all<T, R>(P, G, Wt, +1, 1);
    cpx<T>* out = reinterpret_cast<cpx<T>*>(a.out) + (long long)s * a.out_slab + x0;
    for (int e = tid; e < M * XC; e += kZpThreads) {
      const int i = e / XC, xx = e - i * XC;
      if (x0 + xx < a.X) out[(long long)i * a.X + xx] = P[xx * M + i];
    }
    // the next chunk's prologue writes the pencils after the barrier that follows its wait
  }
}

// Persistent grids: two CTAs per SM (one with 16 positions per chunk), at most one per chunk
inline int zp_final_grid(int X, int nrhs, int sms, int XC = kZpFinalXC) {
  const int nq = nrhs * ((X + XC - 1) / XC);
  return std::max(1, std::min(nq, (XC <= 8 ? 2 : 1) * sms));
}
inline int zp_pad_grid(int X, int nslab, int sms) {
  const int nq = nslab * ((X + kZpPadXC - 1) / kZpPadXC);
  return std::max(1, std::min(nq, 2 * sms));
}

}  // namespace homb
