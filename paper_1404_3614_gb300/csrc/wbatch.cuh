// Warp-owned pencil passes of the batched solver's FP32 CG iteration (included by batch.cu).
//
// The block-level passes of batch.cu move chunks of pencils through shared memory with a CTA
// barrier around every radix stage, so that one task's iteration is a long chain of
// barriers with little work between them. Here every warp owns two pencil buffers in shared
// memory and takes whole units of work (two columns, two row pairs, or the two components of
// one column) from global memory to global memory: loads, transforms, the coefficient or the
// projection, stores, with no barrier but __syncwarp. The passes compute what col_pass,
// row_pass (mode 0) and col_final compute: the zero-padded inverse y transform, the x row
// pass (Hermitian c2r of two real rows per complex FFT, A u / |M|, r2c) and the truncating
// forward y transform with Gamma and the CG partial sums p.q (Lemma double-grid, Eq. MBA_GA).
//
// Transforms: length M = L * K by a lane group of L lanes: lane l holds x[l + L m] (m < K),
// does a register DFT of length K, multiplies by w_M^(l k2) and exchanges through the pencil
// buffer; then lane l gathers y[j][k2] (j < L) for k2 = l, l + L, ... (< K), does register
// DFTs of length L and writes X[k2 + K k1] in natural order.
#pragma once

namespace homb {

template <int M> struct WDec { static constexpr int L = 0, K = 0; };
template <> struct WDec<45> { static constexpr int L = 9, K = 5; };
template <> struct WDec<125> { static constexpr int L = 25, K = 5; };
template <> struct WDec<225> { static constexpr int L = 15, K = 15; };
template <> struct WDec<405> { static constexpr int L = 27, K = 15; };

__host__ __device__ inline bool wpass_len(int M) { return M == 45 || M == 125 || M == 225 || M == 405; }

// In-place FFT of the pencil p by the lanes l < L of a lane group (on = false: no memory
// access, but every lane of the warp takes part in the __syncwarp calls). W: w_M^j, j < M
// (forward convention); dir = +1 takes conjugate twiddles.
template <typename T, int L, int K>
__device__ __forceinline__ void wfft_one(cpx<T>* p, int l, const cpx<T>* W, int dir, bool on) {
  constexpr int M = L * K;
  constexpr int RB = (K + L - 1) / L;   // second-stage rounds per lane
  static_assert(M <= 1024, "pencil length");
  cpx<T> v[K];
#pragma unroll
  for (int m = 0; m < K; ++m) v[m] = on ? p[l + L * m] : mk<T>(T(0), T(0));
  dft_reg<T, K>(v, dir);
#pragma unroll
  for (int k2 = 1; k2 < K; ++k2) v[k2] = mulc<T>(v[k2], W[on ? l * k2 : 0], dir > 0);
  __syncwarp();
  if (on) {
#pragma unroll
    for (int k2 = 0; k2 < K; ++k2) p[l + L * k2] = v[k2];
  }
  __syncwarp();
  // lane l: k2 = l + L rb (rb < RB, k2 < K); all reads before any write
  cpx<T> u[RB][L];
#pragma unroll
  for (int rb = 0; rb < RB; ++rb) {
    const int k2 = l + L * rb;
    const bool onb = on && k2 < K;
#pragma unroll
    for (int j = 0; j < L; ++j) u[rb][j] = onb ? p[j + L * k2] : mk<T>(T(0), T(0));
  }
#pragma unroll
  for (int rb = 0; rb < RB; ++rb) dft_reg<T, L>(u[rb], dir);
  __syncwarp();
#pragma unroll
  for (int rb = 0; rb < RB; ++rb) {
    const int k2 = l + L * rb;
    if (on && k2 < K) {
#pragma unroll
      for (int k1 = 0; k1 < L; ++k1) p[k2 + K * k1] = u[rb][k1];
    }
  }
  __syncwarp();
}

// Pencil buffers of one warp: two when two lane groups fit in a warp (both transformed in one
// round), else one (a warp's units are then single pencils).
template <int L> constexpr int wbufs() { return 32 / L >= 2 ? 2 : 1; }

// The warp's pencils b0 and b1 (b1 only when two is set, warp-uniform), for NB = 2.
template <typename T, int L, int K>
__device__ __forceinline__ void wfft_two(cpx<T>* b0, cpx<T>* b1, const cpx<T>* W, int dir, bool two) {
  const int lane = threadIdx.x & 31;
  const int g = lane / L, l = lane - g * L;
  wfft_one<T, L, K>(g == 0 ? b0 : b1, l, W, dir, g == 0 || (g == 1 && two));
}

// Warp w of the team and the team's warp count: units u = w, w + nw, ...
struct WTeam {
  int w, nw;
};
__device__ __forceinline__ WTeam wteam(const Team& tm, int nslots) {
  const int warps = min(nslots, (int)(blockDim.x >> 5));
  const int warp = threadIdx.x >> 5;
  return {warp < warps ? tm.rank * warps + warp : -1, tm.size * warps};
}

// Zero-padded inverse transforms of the columns (field flist[f], x) of `in` (Nlog rows of X
// entries, FFT order) into M rows of `out`. Unit: NB consecutive columns.
template <typename T, int L, int K>
__device__ __noinline__ void wcol_pass(const cpx<T>* in, cpx<T>* out, long long in_fs, long long out_fs,
                                       const int* flist, int nfl, int X, int Nlog, const cpx<T>* W, cpx<T>* region,
                                       int nslots, Team tm) {
  constexpr int M = L * K;
  constexpr int NB = wbufs<L>();
  const WTeam wt = wteam(tm, nslots);
  if (wt.w < 0) return;
  const int lane = threadIdx.x & 31;
  cpx<T>* b0 = region + (size_t)(threadIdx.x >> 5) * NB * M;
  cpx<T>* b1 = b0 + (NB - 1) * M;
  const int half = (Nlog - 1) / 2, top = Nlog - 1 - half;
  const int npen = nfl * X;
  for (int u = wt.w; NB * u < npen; u += wt.nw) {
    const int pen0 = NB * u;
    const bool two = NB == 2 && pen0 + 1 < npen;
    const int f0 = pen0 / X, x0 = pen0 - f0 * X;
    const int pen1 = two ? pen0 + 1 : pen0;
    const int f1 = pen1 / X, x1 = pen1 - f1 * X;
    const cpx<T>* s0 = in + flist[f0] * in_fs + x0;
    const cpx<T>* s1 = in + flist[f1] * in_fs + x1;
    for (int idx = lane; idx < NB * M; idx += 32) {
      const int j = NB == 2 ? (idx & 1) : 0, t = NB == 2 ? (idx >> 1) : idx;
      const int src = t <= half ? t : (t >= M - top ? t - M + Nlog : -1);
      cpx<T> v = mk<T>(T(0), T(0));
      if (src >= 0 && (j == 0 || two)) v = (j ? s1 : s0)[(long long)src * X];
      (j ? b1 : b0)[t] = v;
    }
    __syncwarp();
    if constexpr (NB == 2) wfft_two<T, L, K>(b0, b1, W, +1, two);
    else wfft_one<T, L, K>(b0, lane, W, +1, lane < L);
    cpx<T>* d0 = out + flist[f0] * out_fs + x0;
    cpx<T>* d1 = out + flist[f1] * out_fs + x1;
    for (int idx = lane; idx < NB * M; idx += 32) {
      const int j = NB == 2 ? (idx & 1) : 0, t = NB == 2 ? (idx >> 1) : idx;
      if (j == 0 || two) (j ? d1 : d0)[(long long)t * X] = (j ? b1 : b0)[t];
    }
    __syncwarp();
  }
}

// x row pass (mode 0 of row_pass) on the rows of `rows`: pair (r, y) packs the two
// components of field rlist[r] at row y into one complex row of length M; unit: NB pairs.
template <typename T, int L, int K>
__device__ __noinline__ void wrow_pass(cpx<T>* rows, long long field_stride, int M1, int Nh, const T* coef,
                                       int ncomp, T scale, const int* rlist, int nrl, const cpx<T>* W,
                                       cpx<T>* region, int nslots, Team tm) {
  constexpr int M = L * K;
  constexpr int NB = wbufs<L>();
  const WTeam wt = wteam(tm, nslots);
  if (wt.w < 0) return;
  const int lane = threadIdx.x & 31;
  cpx<T>* buf[2];
  buf[0] = region + (size_t)(threadIdx.x >> 5) * NB * M;
  buf[1] = buf[0] + (NB - 1) * M;
  const long long cs = (long long)M1 * M;
  const int npairs = nrl * M1;
  for (int u = wt.w; NB * u < npairs; u += wt.nw) {
    const bool two = NB == 2 && NB * u + 1 < npairs;
    long long base[2][2];
    int yy[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int pr = NB * u + (j == 1 && two ? 1 : 0);
      const int a = pr / M1;
      const int y = pr - a * M1;
      const int r = rlist[a];
      yy[j] = y;
      base[j][0] = (long long)(r * 2) * field_stride + (long long)y * Nh;
      base[j][1] = (long long)(r * 2 + 1) * field_stride + (long long)y * Nh;
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if (j == 1 && !two) break;
      for (int k = lane; k < M; k += 32) {
        cpx<T> z[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          cpx<T> v = mk<T>(T(0), T(0));
          if (k < Nh) {
            v = rows[base[j][h] + k];
            if (k == 0) v.y = T(0);
          } else if (k > M - Nh) {
            v = conj_<T>(rows[base[j][h] + (M - k)]);
          }
          z[h] = v;
        }
        buf[j][k] = mk<T>(z[0].x - z[1].y, z[0].y + z[1].x);
      }
    }
    __syncwarp();
    if constexpr (NB == 2) wfft_two<T, L, K>(buf[0], buf[1], W, +1, two);
    else wfft_one<T, L, K>(buf[0], lane, W, +1, lane < L);
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if (j == 1 && !two) break;
      for (int x = lane; x < M; x += 32) {
        const cpx<T> z = buf[j][x];
        T v0, v1;
        coef_apply<T>(coef, (long long)yy[j] * M + x, cs, ncomp, z.x, z.y, &v0, &v1, scale);
        buf[j][x] = mk<T>(v0, v1);
      }
    }
    __syncwarp();
    if constexpr (NB == 2) wfft_two<T, L, K>(buf[0], buf[1], W, -1, two);
    else wfft_one<T, L, K>(buf[0], lane, W, -1, lane < L);
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if (j == 1 && !two) break;
      for (int k = lane; k < Nh; k += 32) {
        const cpx<T> zk = buf[j][k];
        const cpx<T> zm = buf[j][k == 0 ? 0 : M - k];
        rows[base[j][0] + k] = mk<T>(T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y));
        rows[base[j][1] + k] = mk<T>(T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x));
      }
    }
    __syncwarp();
  }
}

// Truncating forward transforms of both components of field rlist[r] at column kx, Gamma^E
// (side 0) or Gamma^J (side 1), q written, partial p.q per right-hand side in pq_acc (FP32
// terms, FP64 sums). Unit: one column. With one buffer per warp the first component's kept
// outputs wait in registers (N1 <= 32 * kWRows) while the second is transformed.
constexpr int kWRows = 8;
template <typename T, int L, int K>
__device__ __noinline__ void wcol_final(const cpx<T>* T2, cpx<T>* q, const cpx<T>* p, long long t2_fs,
                                        long long fld_fs, const int* rlist, int nrl, int Nh, int N1, double iy0,
                                        double iy1, int side, const cpx<T>* W, cpx<T>* region, int nslots,
                                        double* pq_acc, Team tm) {
  constexpr int M = L * K;
  constexpr int NB = wbufs<L>();
  const WTeam wt = wteam(tm, nslots);
  if (wt.w < 0) return;
  const int lane = threadIdx.x & 31;
  cpx<T>* b0 = region + (size_t)(threadIdx.x >> 5) * NB * M;
  cpx<T>* b1 = b0 + (NB - 1) * M;
  const int half = (N1 - 1) / 2;
  const int ncol = nrl * Nh;
  for (int col = wt.w; col < ncol; col += wt.nw) {
    const int a = col / Nh;
    const int kx = col - a * Nh;
    const int r = rlist[a];
    const cpx<T>* s0 = T2 + (long long)(r * 2) * t2_fs + kx;
    const cpx<T>* s1 = T2 + (long long)(r * 2 + 1) * t2_fs + kx;
    cpx<T> keep0[NB == 2 ? 1 : kWRows];
    if constexpr (NB == 2) {
      for (int idx = lane; idx < 2 * M; idx += 32) {
        const int c = idx & 1, t = idx >> 1;
        (c ? b1 : b0)[t] = (c ? s1 : s0)[(long long)t * Nh];
      }
      __syncwarp();
      wfft_two<T, L, K>(b0, b1, W, -1, true);
    } else {
      for (int t = lane; t < M; t += 32) b0[t] = s0[(long long)t * Nh];
      __syncwarp();
      wfft_one<T, L, K>(b0, lane, W, -1, lane < L);
#pragma unroll
      for (int k = 0; k < kWRows; ++k) {
        const int i = lane + 32 * k;
        const int ky = i <= half ? i : i - N1;
        keep0[k] = i < N1 ? b0[ky < 0 ? ky + M : ky] : mk<T>(T(0), T(0));
      }
      __syncwarp();
      for (int t = lane; t < M; t += 32) b0[t] = s1[(long long)t * Nh];
      __syncwarp();
      wfft_one<T, L, K>(b0, lane, W, -1, lane < L);
    }
    float run = 0.f;
#pragma unroll
    for (int k = 0; k < kWRows; ++k) {
      const int i = lane + 32 * k;
      if (i >= N1) break;
      const int ky = i <= half ? i : i - N1;
      const int pos = ky < 0 ? ky + M : ky;
      cpx<T> u0, u1;
      if constexpr (NB == 2) {
        u0 = b0[pos];
        u1 = b1[pos];
      } else {
        u0 = keep0[k];
        u1 = b0[pos];
      }
      const T xi0 = T(kx * iy0), xi1 = T(ky * iy1);
      const T n2 = xi0 * xi0 + xi1 * xi1;
      if (n2 == T(0)) {
        u0 = mk<T>(T(0), T(0));
        u1 = u0;
      } else {
        const T inv = T(1) / n2;
        const cpx<T> dot = mk<T>(xi0 * u0.x + xi1 * u1.x, xi0 * u0.y + xi1 * u1.y);
        const cpx<T> g0 = mk<T>(xi0 * dot.x * inv, xi0 * dot.y * inv);
        const cpx<T> g1 = mk<T>(xi1 * dot.x * inv, xi1 * dot.y * inv);
        if (side == 0) {
          u0 = g0;
          u1 = g1;
        } else {
          u0 = sub<T>(u0, g0);
          u1 = sub<T>(u1, g1);
        }
      }
      const long long e = (long long)i * Nh + kx;
      q[(r * 2 + 0) * fld_fs + e] = u0;
      q[(r * 2 + 1) * fld_fs + e] = u1;
      const cpx<T> p0 = p[(r * 2 + 0) * fld_fs + e], p1 = p[(r * 2 + 1) * fld_fs + e];
      const float sq = fmaf(p0.x, u0.x, fmaf(p0.y, u0.y, fmaf(p1.x, u1.x, p1.y * u1.y)));
      run = fmaf(kx == 0 ? 1.f : 2.f, sq, run);
    }
    if (r == 0) pq_acc[0] += (double)run;
    else pq_acc[1] += (double)run;
    __syncwarp();
  }
}

// Warps with a pencil slot in the 2 capT-element shared region of a CTA
template <int M> __device__ __forceinline__ int wslots(int capT) {
  return (2 * capT) / (wbufs<WDec<M>::L>() * M);
}

// Dispatch on the compile-time lengths; false when M has no warp decomposition here.
template <typename T>
__device__ bool wcol_pass_any(int M, const cpx<T>* in, cpx<T>* out, long long in_fs, long long out_fs,
                              const int* flist, int nfl, int X, int Nlog, const cpx<T>* W, cpx<T>* region, int capT,
                              Team tm) {
  if constexpr (sizeof(T) != 4) {
    return false;
  } else {
  switch (M) {
#define HOMB_WCOL(m)                                                                                          \
  case m:                                                                                                     \
    wcol_pass<T, WDec<m>::L, WDec<m>::K>(in, out, in_fs, out_fs, flist, nfl, X, Nlog, W, region, wslots<m>(capT), tm); \
    return true;
    HOMB_WCOL(45) HOMB_WCOL(125) HOMB_WCOL(225) HOMB_WCOL(405)
#undef HOMB_WCOL
    default: return false;
  }
  }
}

template <typename T>
__device__ bool wrow_pass_any(int M, cpx<T>* rows, long long field_stride, int M1, int Nh, const T* coef, int ncomp,
                              T scale, const int* rlist, int nrl, const cpx<T>* W, cpx<T>* region, int capT, Team tm) {
  if constexpr (sizeof(T) != 4) {
    return false;
  } else {
  switch (M) {
#define HOMB_WROW(m)                                                                                        \
  case m:                                                                                                   \
    wrow_pass<T, WDec<m>::L, WDec<m>::K>(rows, field_stride, M1, Nh, coef, ncomp, scale, rlist, nrl, W, region, \
                                         wslots<m>(capT), tm);                                                     \
    return true;
    HOMB_WROW(45) HOMB_WROW(125) HOMB_WROW(225) HOMB_WROW(405)
#undef HOMB_WROW
    default: return false;
  }
  }
}

template <typename T>
__device__ bool wcol_final_any(int M, const cpx<T>* T2, cpx<T>* q, const cpx<T>* p, long long t2_fs, long long fld_fs,
                               const int* rlist, int nrl, int Nh, int N1, double iy0, double iy1, int side,
                               const cpx<T>* W, cpx<T>* region, int capT, double* pq_acc, Team tm) {
  if constexpr (sizeof(T) != 4) {
    return false;
  } else {
  switch (M) {
#define HOMB_WFIN(m)                                                                                        \
  case m:                                                                                                   \
    wcol_final<T, WDec<m>::L, WDec<m>::K>(T2, q, p, t2_fs, fld_fs, rlist, nrl, Nh, N1, iy0, iy1, side, W, region, \
                                          wslots<m>(capT), pq_acc, tm);                                            \
    return true;
    HOMB_WFIN(45) HOMB_WFIN(125) HOMB_WFIN(225) HOMB_WFIN(405)
#undef HOMB_WFIN
    default: return false;
  }
  }
}

}  // namespace homb
