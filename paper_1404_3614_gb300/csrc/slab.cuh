// Fused y-x-y slab pass of the FP32 3D operator for an isotropic coefficient (one real
// coefficient value per double-grid point), transform length M = R * R on the x and y
// axes. One CTA owns one (right-hand side, component, z) slab of the field after the z
// inverse transform: it loads the Ny x Nh half-spectrum slab, runs the zero-padded
// inverse y transforms, the x row pass (Hermitian c2r of two real rows per complex FFT,
// pointwise coefficient A_M / |M|, r2c), and the truncating forward y transforms, all in
// shared memory, and writes the Ny x Nh slab back. This is the middle of the operator
// C u = Gamma P_N F_M (A_M/|M|) F_M^{-1} Pad(u) (Lemma double-grid, Eq. MBA_GA) with the
// intermediate double-grid slab never leaving the SM.
//
// Transforms are warp-level in-register Cooley-Tukey FFTs of length R * R: R lanes own
// one pencil; lane l loads x[l + R n2] (n2 < R), does a register DFT of length R, applies
// the twiddles w_M^(l k2), exchanges through shared memory, and does the second register
// DFT; lane l then holds X[l + R k1] (k1 < R). The output layout of the inverse x
// transform is the input layout of the forward one, so the coefficient product happens
// in registers between them.
#pragma once
#include "kernels.cuh"

namespace homb {

constexpr int kSlabMaxThreads = 768;

// In-place FFT of one contiguous pencil of length R*R by the R lanes of a lane group
// (lane index l < R). Every lane of the warp calls it (on = false: no memory access).
// Wt holds w_M^(l k) at [k][l].
template <typename T, int R>
__device__ __forceinline__ void pencil_fft_inplace(cpx<T>* p, int l, const cpx<T>* Wt, int dir, bool on) {
  cpx<T> v[R];
#pragma unroll
  for (int n = 0; n < R; ++n) v[n] = on ? p[l + R * n] : mk<T>(T(0), T(0));
  dft_reg<T, R>(v, dir);
#pragma unroll
  for (int k = 1; k < R; ++k) v[k] = mulc<T>(v[k], Wt[k * R + l], dir > 0);
  __syncwarp();
  if (on) {
#pragma unroll
    for (int k = 0; k < R; ++k) p[l + R * k] = v[k];
  }
  __syncwarp();
#pragma unroll
  for (int n = 0; n < R; ++n) v[n] = on ? p[n + R * l] : mk<T>(T(0), T(0));
  dft_reg<T, R>(v, dir);
  __syncwarp();
  if (on) {
#pragma unroll
    for (int k = 0; k < R; ++k) p[l + R * k] = v[k];
  }
  __syncwarp();
}

// Second half of a register FFT whose first-stage results v (lane l, index k2) are
// exchanged through the scratch pencil S of this lane group: on return v[k1] =
// X[l + R k1]. Lanes with own = false (no lane group) touch no memory.
template <typename T, int R>
__device__ __forceinline__ void fft_finish(cpx<T>* v, cpx<T>* S, int l, const cpx<T>* Wt, int dir, bool own) {
#pragma unroll
  for (int k = 1; k < R; ++k) v[k] = mulc<T>(v[k], Wt[k * R + l], dir > 0);
  __syncwarp();
  if (own) {
#pragma unroll
    for (int k = 0; k < R; ++k) S[l + R * k] = v[k];
  }
  __syncwarp();
#pragma unroll
  for (int n = 0; n < R; ++n) v[n] = own ? S[n + R * l] : mk<T>(T(0), T(0));
  dft_reg<T, R>(v, dir);
}

template <typename T, int R>
__global__ void __launch_bounds__(kSlabMaxThreads) k_slab(SlabArgs a) {
  constexpr int M = R * R;
  constexpr int PW = 32 / R;   // pencils per warp
  extern __shared__ __align__(16) unsigned char smem[];
  cpx<T>* Wt = reinterpret_cast<cpx<T>*>(smem);
  cpx<T>* P = Wt + M;                              // [Nh][M]: column kx, y contiguous
  cpx<T>* S = P + (size_t)a.Nh * M;                // [warps * PW][M] scratch pencils
  // slab order: z major, so the slabs that share a coefficient plane run together
  const int z = blockIdx.x / a.nrc;
  const int rc = blockIdx.x - z * a.nrc;
  const int rhs = rc / a.C;
  if (a.cg != nullptr && !a.cg->active[rhs]) return;
  const long long s = (long long)rc * a.Mz + z;
  const int Ny = a.Ny, Nh = a.Nh, half = (Ny - 1) / 2;
  const cpx<T>* in = reinterpret_cast<const cpx<T>*>(a.in) + s * Ny * Nh;
  cpx<T>* out = reinterpret_cast<cpx<T>*>(a.out) + s * Ny * Nh;
  // twiddles w_M^(l k) stored at [k][l] so that the R lanes of a group read consecutive words
  const cpx<T>* W = reinterpret_cast<const cpx<T>*>(a.W);
  for (int t = threadIdx.x; t < M; t += blockDim.x) {
    const int k = t / R;
    Wt[t] = W[(t - k * R) * k];
  }
  const int npad = M - Ny;
  for (int t = threadIdx.x; t < Nh * npad; t += blockDim.x) {
    const int kx = t / npad;
    P[kx * M + half + 1 + (t - kx * npad)] = mk<T>(T(0), T(0));
  }
  for (int t = threadIdx.x; t < Ny * Nh; t += blockDim.x) {
    const int y = t / Nh;
    const int kx = t - y * Nh;
    const int pos = y <= half ? y : y - Ny + M;
    P[kx * M + pos] = in[t];
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane / R, l = lane - sub * R;
  const bool act = sub < PW;
  const int slots = (blockDim.x >> 5) * PW;
  const int slot = warp * PW + sub;

  // inverse y transforms of the Nh columns (zero padded)
  for (int c0 = 0; c0 < Nh; c0 += slots) {
    const int kx = c0 + slot;
    const bool on = act && kx < Nh;
    pencil_fft_inplace<T, R>(P + (size_t)(on ? kx : 0) * M, l, Wt, +1, on);
  }
  __syncthreads();

  // x row pass: rows ya = 2 pr and yb = 2 pr + 1 packed as Z = X_a + i X_b
  cpx<T>* Sw = S + (size_t)(act ? slot : 0) * M;
  const T* coefz = reinterpret_cast<const T*>(a.coef) + (size_t)z * M * M;
  const T scale = T(a.scale);
  constexpr int npairs = (M + 1) / 2;
  for (int p0 = 0; p0 < npairs; p0 += slots) {
    const int pr = p0 + slot;
    const bool on = act && pr < npairs;
    const int ya = 2 * pr, yb = 2 * pr + 1;
    const bool hb = on && yb < M;
    // coefficient rows first: their global loads overlap the gather and the inverse FFT
    T ca[R], cb[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      ca[k] = on ? __ldg(coefz + (size_t)ya * M + l + R * k) : T(0);
      cb[k] = hb ? __ldg(coefz + (size_t)yb * M + l + R * k) : T(0);
    }
    cpx<T> v[R];
#pragma unroll
    for (int n = 0; n < R; ++n) {
      const int k = l + R * n;
      cpx<T> A = mk<T>(T(0), T(0)), B = mk<T>(T(0), T(0));
      if (on) {
        if (k < Nh) {
          A = P[k * M + ya];
          if (hb) B = P[k * M + yb];
          if (k == 0) { A.y = T(0); B.y = T(0); }
        } else if (k > M - Nh) {
          A = conj_<T>(P[(M - k) * M + ya]);
          if (hb) B = conj_<T>(P[(M - k) * M + yb]);
        }
      }
      v[n] = mk<T>(A.x - B.y, A.y + B.x);
    }
    dft_reg<T, R>(v, +1);
    fft_finish<T, R>(v, Sw, l, Wt, +1, act);
    // v[k1] = z(x = l + R k1): real part row ya, imaginary part row yb
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = mk<T>(v[k].x * (ca[k] * scale), v[k].y * (cb[k] * scale));
    // forward transform: lane l holds x[l + R n2] with n2 = k1
    dft_reg<T, R>(v, -1);
    fft_finish<T, R>(v, Sw, l, Wt, -1, act);
    __syncwarp();
    if (act) {
#pragma unroll
      for (int k = 0; k < R; ++k) Sw[l + R * k] = v[k];
    }
    __syncwarp();
    if (on) {
      for (int kx = l; kx < Nh; kx += R) {
        const cpx<T> zk = Sw[kx];
        const cpx<T> zm = Sw[kx == 0 ? 0 : M - kx];
        P[kx * M + ya] = mk<T>(T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y));
        if (hb) P[kx * M + yb] = mk<T>(T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x));
      }
    }
    __syncwarp();
  }
  __syncthreads();

  // forward y transforms (truncated on store)
  for (int c0 = 0; c0 < Nh; c0 += slots) {
    const int kx = c0 + slot;
    const bool on = act && kx < Nh;
    pencil_fft_inplace<T, R>(P + (size_t)(on ? kx : 0) * M, l, Wt, -1, on);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < Ny * Nh; t += blockDim.x) {
    const int y = t / Nh;
    const int kx = t - y * Nh;
    const int pos = y <= half ? y : y - Ny + M;
    out[t] = P[kx * M + pos];
  }
}

// shared memory of one slab CTA with `warps` warps (R*R = M)
inline size_t slab_smem_bytes(int M, int R, int Nh, int warps, size_t elem) {
  return elem * ((size_t)M + (size_t)Nh * M + (size_t)warps * (32 / R) * M);
}

template <typename T, int R> cudaError_t launch_slab_r(const SlabArgs& a, int warps, cudaStream_t s) {
  const size_t smem = slab_smem_bytes(R * R, R, a.Nh, warps, sizeof(cpx<T>));
  static std::atomic<size_t> cache[16] = {};
  cudaError_t e = smem_attr(k_slab<T, R>, smem, cache);
  if (e != cudaSuccess) return e;
  k_slab<T, R><<<a.nrc * a.Mz, warps * 32, smem, s>>>(a);
  return cudaGetLastError();
}

// Warps per slab CTA, or 0 when the slab pass does not apply (length not R*R with R in
// {3, 5, 9, 15}, or the slab does not fit in shared memory).
template <typename T> int slab_warps(int M, int Nh) {
  int R = 0;
  for (int r : {3, 5, 9, 15})
    if (r * r == M) R = r;
  // FP64 stays on the separate passes: it is bound by the FP64 pipe, and lane groups of R
  // leave 32 mod R lanes of every warp issuing FP64 work on zeros
  if (R == 0 || sizeof(T) == 8) return 0;
  const size_t elem = sizeof(cpx<T>);
  // eight warps when at least two CTAs fit on an SM; else one CTA per SM with the fewest
  // warps that reach the fewest rounds of lane-group tasks (two column rounds, weight 1
  // each, plus row-pair rounds, weight 2.5), measured best at 225^3 (20 warps: 0.44 ms,
  // 16: 0.47, 24: 0.47)
  if (2 * slab_smem_bytes(M, R, Nh, 8, elem) <= 220 * 1024) return 8;
  const int PW = 32 / R, npairs = (M + 1) / 2;
  int best = 0;
  double best_cost = 1e30;
  for (int w = 8; w <= 24; w += 4) {
    if (slab_smem_bytes(M, R, Nh, w, elem) > 220 * 1024) break;
    const int slots = w * PW;
    const double cost = 2.0 * ((Nh + slots - 1) / slots) + 2.5 * ((npairs + slots - 1) / slots);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = w;
    }
  }
  return best;
}

template <typename T> cudaError_t launch_slab(const SlabArgs& a, cudaStream_t s) {
  if constexpr (sizeof(T) != 4) {
    return cudaErrorNotSupported;
  } else {
    int warps = slab_warps<T>(a.M, a.Nh);
    if (warps && a.warps > 0) {   // a caller's choice, where it fits
      const int r = a.M == 225 ? 15 : (a.M == 81 ? 9 : (a.M == 25 ? 5 : 3));
      if (a.warps * 32 <= kSlabMaxThreads && slab_smem_bytes(a.M, r, a.Nh, a.warps, sizeof(cpx<T>)) <= 220 * 1024)
        warps = a.warps;
    }
    switch (warps ? a.M : 0) {
      case 9: return launch_slab_r<T, 3>(a, warps, s);
      case 25: return launch_slab_r<T, 5>(a, warps, s);
      case 81: return launch_slab_r<T, 9>(a, warps, s);
      case 225: return launch_slab_r<T, 15>(a, warps, s);
      default: return cudaErrorNotSupported;
    }
  }
}

}  // namespace homb
