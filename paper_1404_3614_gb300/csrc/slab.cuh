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
#include <algorithm>

#include "kernels.cuh"

namespace homb {

constexpr int kSlabMaxThreads = 640;   // 20 warps: up to 102 registers a thread

// Byte offset of the scratch / staging region of a slab CTA: after the barrier (16 bytes),
// the twiddles [M] and the slab [Nh][M], rounded up to 16 bytes (the bulk copy lands there).
__host__ __device__ inline size_t slab_scratch_offset(int M, int Nh, size_t elem) {
  return (16 + elem * ((size_t)M + (size_t)Nh * M) + 15) & ~(size_t)15;
}

// shared memory of one slab CTA with `warps` warps (R*R = M): the scratch region holds the
// x pass's pencils or the staged input slab (Ny x Nh plus one element of alignment slack)
inline size_t slab_smem_bytes(int M, int R, int Nh, int warps, size_t elem) {
  const int Ny = (M + 1) / 2;
  const size_t scratch = std::max((size_t)warps * (32 / R) * M, (size_t)Ny * Nh + 2);
  return slab_scratch_offset(M, Nh, elem) + elem * scratch;
}


// First-stage DFT of a zero-padded inverse transform (inputs of the zero band not read) and
// last-stage DFT of a truncating forward one (outputs of the band not computed)
template <typename T, int R>
__device__ __forceinline__ void dft_reg_zin(cpx<T>* v, int dir) {
  if constexpr (R == 15) dft15_zin<T>(v, dir);
  else {
#pragma unroll
    for (int n = 0; n < R; ++n)
      if (ZeroBand<R>::in(n)) v[n] = mk<T>(T(0), T(0));
    dft_reg<T, R>(v, dir);
  }
}
template <typename T, int R>
__device__ __forceinline__ void dft_reg_zout(cpx<T>* v, int dir) {
  if constexpr (R == 15) dft15_zout<T>(v, dir);
  else dft_reg<T, R>(v, dir);
}

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
    for (int k = 0; k < R; ++k) p[l + R * k] = st_norm<T>(v[k]);
  }
  __syncwarp();
#pragma unroll
  for (int n = 0; n < R; ++n) v[n] = on ? p[n + R * l] : mk<T>(T(0), T(0));
  dft_reg<T, R>(v, dir);
  __syncwarp();
  if (on) {
#pragma unroll
    for (int k = 0; k < R; ++k) p[l + R * k] = st_norm<T>(v[k]);
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
    for (int k = 0; k < R; ++k) S[l + R * k] = st_norm<T>(v[k]);
  }
  __syncwarp();
#pragma unroll
  for (int n = 0; n < R; ++n) v[n] = own ? S[n + R * l] : mk<T>(T(0), T(0));
  dft_reg<T, R>(v, dir);
}

constexpr long long kSlabSpinLimit = 1LL << 22;   // polls of the staged-copy barrier

__device__ __forceinline__ uint32_t slab_smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Bounded wait for one phase of the staging barrier; false if it gave up.
__device__ __forceinline__ bool slab_wait(uint32_t mbar, uint32_t phase) {
  for (long long it = 0; it < kSlabSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Where the Ny x Nh input slab starting at global address `src` goes in the staging buffer
// and how it is copied: a bulk copy of the 16-byte aligned middle (`body` bytes from element
// `head`), plus at most one plain element in front (head = 1) and one behind (tail = 1).
struct SlabStage {
  int head, tail;
  unsigned body;
};
template <typename T>
__device__ __forceinline__ SlabStage slab_stage_plan(const cpx<T>* src, long long elems) {
  SlabStage st;
  st.head = (reinterpret_cast<uintptr_t>(src) & 15) ? 1 : 0;
  const long long bytes = (elems - st.head) * (long long)sizeof(cpx<T>);
  st.body = (unsigned)(bytes & ~15LL);
  st.tail = (int)((bytes - st.body) / (long long)sizeof(cpx<T>));
  return st;
}

// Persistent fused slab pass. Each CTA walks the slabs blockIdx.x, blockIdx.x + gridDim.x, ...
// (z-major, so the slabs in flight share few coefficient planes). The input of a slab is
// staged in shared memory by one bulk asynchronous copy (an mbarrier tracks its bytes),
// issued for the next slab as soon as the x pass of the current one has released the
// staging buffer, so the copy overlaps the forward y transforms and the stores. The inverse
// y transforms read the staged rows directly (zero padding implicit).
// pencil_fft_inplace for a truncating forward transform (dir = -1): the outputs of the zero
// band are neither computed nor stored
template <typename T, int R>
__device__ __forceinline__ void pencil_fft_fwd_trunc(cpx<T>* p, int l, const cpx<T>* Wt, bool on) {
  cpx<T> v[R];
#pragma unroll
  for (int n = 0; n < R; ++n) v[n] = on ? p[l + R * n] : mk<T>(T(0), T(0));
  dft_reg<T, R>(v, -1);
#pragma unroll
  for (int k = 1; k < R; ++k) v[k] = mulc<T>(v[k], Wt[k * R + l], false);
  __syncwarp();
  if (on) {
#pragma unroll
    for (int k = 0; k < R; ++k) p[l + R * k] = st_norm<T>(v[k]);
  }
  __syncwarp();
#pragma unroll
  for (int n = 0; n < R; ++n) v[n] = on ? p[n + R * l] : mk<T>(T(0), T(0));
  dft_reg_zout<T, R>(v, -1);
  __syncwarp();
  if (on) {
#pragma unroll
    for (int k = 0; k < R; ++k)
      if (!ZeroBand<R>::in(k)) p[l + R * k] = st_norm<T>(v[k]);
  }
  __syncwarp();
}

// pencil_fft_inplace for a zero-padded inverse transform (dir = +1): the zero band's inputs
// are not read
template <typename T, int R>
__device__ __forceinline__ void pencil_fft_pad_inv(cpx<T>* p, int l, const cpx<T>* Wt, bool on) {
  cpx<T> v[R];
#pragma unroll
  for (int n = 0; n < R; ++n)
    if (!ZeroBand<R>::in(n)) v[n] = on ? p[l + R * n] : mk<T>(T(0), T(0));
  dft_reg_zin<T, R>(v, +1);
#pragma unroll
  for (int k = 1; k < R; ++k) v[k] = mulc<T>(v[k], Wt[k * R + l], true);
  __syncwarp();
  if (on) {
#pragma unroll
    for (int k = 0; k < R; ++k) p[l + R * k] = st_norm<T>(v[k]);
  }
  __syncwarp();
#pragma unroll
  for (int n = 0; n < R; ++n) v[n] = on ? p[n + R * l] : mk<T>(T(0), T(0));
  dft_reg<T, R>(v, +1);
  __syncwarp();
  if (on) {
#pragma unroll
    for (int k = 0; k < R; ++k) p[l + R * k] = st_norm<T>(v[k]);
  }
  __syncwarp();
}

// fft_finish whose outputs of the zero band are not needed (a truncating forward transform)
template <typename T, int R>
__device__ __forceinline__ void fft_finish_zout(cpx<T>* v, cpx<T>* S, int l, const cpx<T>* Wt, bool own) {
#pragma unroll
  for (int k = 1; k < R; ++k) v[k] = mulc<T>(v[k], Wt[k * R + l], false);
  __syncwarp();
  if (own) {
#pragma unroll
    for (int k = 0; k < R; ++k) S[l + R * k] = st_norm<T>(v[k]);
  }
  __syncwarp();
#pragma unroll
  for (int n = 0; n < R; ++n) v[n] = own ? S[n + R * l] : mk<T>(T(0), T(0));
  dft_reg_zout<T, R>(v, -1);
}

template <typename T, int R, bool ZB>
__global__ void __launch_bounds__(kSlabMaxThreads) k_slab(SlabArgs a) {
  constexpr int M = R * R;
  constexpr int PW = 32 / R;   // pencils per warp
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);
  cpx<T>* Wt = reinterpret_cast<cpx<T>*>(smem + 16);
  cpx<T>* P = Wt + M;                              // [Nh][M]: column kx, y contiguous
  // x-pass scratch pencils [warps * PW][M], and between x passes the staged next input
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smem + slab_scratch_offset(M, a.Nh, sizeof(cpx<T>)));
  const int Ny = a.Ny, Nh = a.Nh, half = (Ny - 1) / 2;
  const long long slab_elems = (long long)Ny * Nh;
  const long long nslabs = (long long)a.nrc * a.Mz;
  const cpx<T>* in = reinterpret_cast<const cpx<T>*>(a.in);
  cpx<T>* out = reinterpret_cast<cpx<T>*>(a.out);
  // twiddles w_M^(l k) stored at [k][l] so that the R lanes of a group read consecutive words
  const cpx<T>* W = reinterpret_cast<const cpx<T>*>(a.W);
  for (int t = threadIdx.x; t < M; t += blockDim.x) {
    const int k = t / R;
    Wt[t] = W[(t - k * R) * k];
  }
  // slab q of the walk is (z, rc) = (q / nrc, q mod nrc) (z-major); in memory it is slab
  // rc * Mz + z of the [nrc][Mz][Ny][Nh] field
  auto mem = [&](long long q) {
    const long long z = q / a.nrc;
    return (q - z * a.nrc) * a.Mz + z;
  };
  auto active = [&](long long s) {
    if (a.cg == nullptr) return true;
    const int rc = (int)(s % a.nrc);
    return a.cg->active[rc / a.C] != 0;
  };
  auto next_active = [&](long long s) {
    do {
      s += gridDim.x;
    } while (s < nslabs && !active(s));
    return s;
  };
  long long s = blockIdx.x;
  if (s < nslabs && !active(s)) s = next_active(s);
  const uint32_t mb = slab_smem_u32(mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // thread 0: start the staged copy of slab t; the plain end elements go to registers
  cpx<T> edge0 = mk<T>(T(0), T(0)), edge1 = mk<T>(T(0), T(0));
  auto issue = [&](long long t) {
    const cpx<T>* src = in + mem(t) * slab_elems;
    const SlabStage st = slab_stage_plan<T>(src, slab_elems);
    cpx<T>* stage = S + st.head;   // S is 16-byte aligned: element `head` lands aligned
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(st.body) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     slab_smem_u32(stage + st.head)),
                 "l"(src + st.head), "r"(st.body), "r"(mb)
                 : "memory");
    if (st.head) edge0 = src[0];
    if (st.tail) edge1 = src[slab_elems - 1];
  };
  if (threadIdx.x == 0 && s < nslabs) issue(s);
  uint32_t phase = 0;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane / R, l = lane - sub * R;
  const bool act = sub < PW;
  const int slots = (blockDim.x >> 5) * PW;
  const int slot = warp * PW + sub;
  constexpr int npairs = (M + 1) / 2;
  const T scale = T(a.scale);

  while (s < nslabs) {
    const int z = (int)(s / a.nrc);
    const SlabStage st = slab_stage_plan<T>(in + mem(s) * slab_elems, slab_elems);
    const cpx<T>* stage = S + st.head;
    // ---- wait for the staged input (bounded), complete its plain end elements
    const bool ok = __syncthreads_and(slab_wait(mb, phase) ? 1 : 0) != 0;
    if (!ok) {
      // the copy never completed: report it, give it one more bounded wait, stop this CTA
      if (threadIdx.x == 0 && a.fault) atomicExch(a.fault, 1);
      slab_wait(mb, phase);
      return;
    }
    phase ^= 1u;
    if (threadIdx.x == 0) {
      if (st.head) const_cast<cpx<T>*>(stage)[0] = edge0;
      if (st.tail) const_cast<cpx<T>*>(stage)[slab_elems - 1] = edge1;
    }
    __syncthreads();

    // ---- inverse y transforms of the Nh columns: input rows from the staged slab
    // (row-major [Ny][Nh]), zero padded to M, results into column kx of P
    for (int c0 = 0; c0 < Nh; c0 += slots) {
      if (c0 + warp * PW >= Nh) break;   // no column for this warp in this or a later round
      const int kx = c0 + slot;
      const bool on = act && kx < Nh;
      cpx<T>* p = P + (size_t)(on ? kx : 0) * M;
      cpx<T> v[R];
#pragma unroll
      for (int n = 0; n < R; ++n) {
        if (ZB && ZeroBand<R>::in(n)) continue;   // padding rows only
        const int pos = l + R * n;
        const int y = pos <= half ? pos : (pos >= M - half ? pos - M + Ny : -1);
        v[n] = (on && y >= 0) ? stage[(size_t)y * Nh + kx] : mk<T>(T(0), T(0));
      }
      if constexpr (ZB) dft_reg_zin<T, R>(v, +1);
      else dft_reg<T, R>(v, +1);
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = mulc<T>(v[k], Wt[k * R + l], true);   // inverse: conjugate twiddles
      __syncwarp();
      if (on) {
#pragma unroll
        for (int k = 0; k < R; ++k) p[l + R * k] = v[k];
      }
      __syncwarp();
#pragma unroll
      for (int n = 0; n < R; ++n) v[n] = on ? p[n + R * l] : mk<T>(T(0), T(0));
      dft_reg<T, R>(v, +1);
      __syncwarp();
      if (on) {
#pragma unroll
        for (int k = 0; k < R; ++k) p[l + R * k] = v[k];
      }
      __syncwarp();
    }
    __syncthreads();

    // ---- x row pass: rows ya = 2 pr and yb = 2 pr + 1 packed as Z = X_a + i X_b
    cpx<T>* Sw = S + (size_t)(act ? slot : 0) * M;
    const T* coefz = reinterpret_cast<const T*>(a.coef) + (size_t)z * M * M;
    for (int p0 = 0; p0 < npairs; p0 += slots) {
      if (p0 + warp * PW >= npairs) break;   // no row pair for this warp
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
        if (ZB && ZeroBand<R>::in(n)) continue;   // frequencies of the padding only
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
      if constexpr (ZB) dft_reg_zin<T, R>(v, +1);
      else dft_reg<T, R>(v, +1);
      fft_finish<T, R>(v, Sw, l, Wt, +1, act);
      // v[k1] = z(x = l + R k1): real part row ya, imaginary part row yb
#pragma unroll
      for (int k = 0; k < R; ++k) v[k] = mk<T>(v[k].x * (ca[k] * scale), v[k].y * (cb[k] * scale));
      // forward transform: lane l holds x[l + R n2] with n2 = k1; the kept frequencies only
      dft_reg<T, R>(v, -1);
      if constexpr (ZB) fft_finish_zout<T, R>(v, Sw, l, Wt, act);
      else fft_finish<T, R>(v, Sw, l, Wt, -1, act);
      __syncwarp();
      if (act) {
#pragma unroll
        for (int k = 0; k < R; ++k)
          if (!(ZB && ZeroBand<R>::in(k))) Sw[l + R * k] = v[k];
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
    // ---- the staging buffer is free: start the copy of the next slab's input (the async
    // proxy writes where the generic proxy just read and wrote: every thread orders its own
    // accesses before it, then the barrier, then one thread issues the copy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const long long sn = next_active(s);
    if (threadIdx.x == 0 && sn < nslabs) issue(sn);

    // ---- forward y transforms (truncated; with ZB the zero band's rows are neither computed nor
    // stored)
    for (int c0 = 0; c0 < Nh; c0 += slots) {
      if (c0 + warp * PW >= Nh) break;
      const int kx = c0 + slot;
      const bool on = act && kx < Nh;
      if constexpr (ZB) pencil_fft_fwd_trunc<T, R>(P + (size_t)(on ? kx : 0) * M, l, Wt, on);
      else pencil_fft_inplace<T, R>(P + (size_t)(on ? kx : 0) * M, l, Wt, -1, on);
    }
    __syncthreads();
    cpx<T>* o = out + mem(s) * slab_elems;
    for (int t = threadIdx.x; t < Ny * Nh; t += blockDim.x) {
      const int y = t / Nh;
      const int kx = t - y * Nh;
      const int pos = y <= half ? y : y - Ny + M;
      o[t] = P[kx * M + pos];
    }
    __syncthreads();   // P is rewritten by the next slab's inverse y transforms
    s = sn;
  }
}

template <typename T, int R, bool ZB> cudaError_t launch_slab_rz(const SlabArgs& a, int warps, cudaStream_t s) {
  const size_t smem = slab_smem_bytes(R * R, R, a.Nh, warps, sizeof(cpx<T>));
  static std::atomic<int> cache[kAttrDevices] = {};
  cudaError_t e = smem_attr(k_slab<T, R, ZB>, smem, cache);
  if (e != cudaSuccess) return e;
  // persistent: as many CTAs as are resident at once, at most one per slab
  int dev = 0, sms = 0, per = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_slab<T, R, ZB>, warps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorInvalidConfiguration;
  const long long nslabs = (long long)a.nrc * a.Mz;
  const int grid = (int)std::min<long long>(nslabs, (long long)sms * per);
  k_slab<T, R, ZB><<<grid, warps * 32, smem, s>>>(a);
  return cudaGetLastError();
}

// The zero band applies when the y rows (Ny stored around 0) and the Hermitian x extension
// (2 Nh - 1 frequencies around 0) leave it empty: a zero-padded double grid M >= 2N - 1; not
// when the transforms are as long as the data (GaNi on the N grid, M = N)
inline bool slab_band_free(int M, int Ny, int Nh) {
  auto f = [M](int n) {
    const int half = (n - 1) / 2, top = n - 1 - half;
    return half < (M + 3) / 4 && M - top > (3 * M - 3) / 4;
  };
  return f(Ny) && f(2 * Nh - 1);
}

template <typename T, int R> cudaError_t launch_slab_r(const SlabArgs& a, int warps, cudaStream_t s) {
  return slab_band_free(a.M, a.Ny, a.Nh) ? launch_slab_rz<T, R, true>(a, warps, s)
                                         : launch_slab_rz<T, R, false>(a, warps, s);
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
  for (int w = 8; w * 32 <= kSlabMaxThreads; w += 4) {
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
