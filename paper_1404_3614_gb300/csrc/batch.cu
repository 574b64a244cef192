// Persistent batched solver for many small 2D cells of uneven N (one launch).
//
// Each CTA pops (problem, side) tasks from an atomic counter and runs the whole
// pipeline for one task on its own: the double-grid coefficient from the closed-form
// inclusion coefficients (Lemma bounds_for_matrix-inclusion, Eq. MBA_GA), the
// right-hand sides b = -Gamma A_hat(k) e_r (Eqs. linear_system_primal / _dual), CG for
// both right-hand sides with block-level deterministic reductions (Sec. 6.1), the FP64
// re-projection and the exact double-grid energies (Lemma double-grid, Def.
// upper_lower_bounds). No grid-wide synchronisation and no waits between CTAs: each
// task is independent. Data live in a per-CTA global scratch slot (L2-resident for the
// small grids) and pass through shared memory in chunks of FFT pencils.
#include <atomic>
#include <type_traits>
#include <cooperative_groups.h>
#include <math.h>

#include "attr.cuh"
#include "kernels.cuh"
#include "spectrum.cuh"

namespace homb {

namespace cg = cooperative_groups;

// The CTAs that work on one task together: the whole thread-block cluster (rank, size)
// for a cooperative task, or this CTA alone (0, 1). Task-wide loops stride over the
// team's threads, chunk loops over its CTAs; team_sync orders their global and shared
// memory accesses (a cluster barrier with release / acquire semantics, or
// __syncthreads for a team of one).
struct Team {
  int rank, size;
  __device__ long long tid() const { return (long long)rank * blockDim.x + threadIdx.x; }
  __device__ long long nth() const { return (long long)size * blockDim.x; }
};

__device__ __forceinline__ void team_sync(const Team& tm) {
  if (tm.size > 1) {
    __threadfence();
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
}

// Deterministic sum of one double per thread over the team, valid in thread 0 of every
// CTA of the team: block sums in a fixed tree, then the per-CTA sums in rank order from
// rank 0's exchange buffer xch[2][8] (alternating halves, so that one barrier per sum
// suffices).
__device__ double team_sum(const Team& tm, double v, double* red, double* xch, int& parity) {
  const double s = block_sum(v, red);
  if (tm.size == 1) return s;
  cg::cluster_group cl = cg::this_cluster();
  double* x0 = cl.map_shared_rank(xch, 0);
  if (threadIdx.x == 0) x0[parity * 8 + tm.rank] = s;
  cl.sync();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int r = 0; r < tm.size; ++r) t += x0[parity * 8 + r];
  parity ^= 1;
  return t;
}


// G pencils of compile-time length M with one radix schedule (BIG: composite register
// radices), or the runtime plan for any other length. Each schedule is its own function
// so that its registers are allocated on their own.
template <typename T, bool BIG>
__device__ __noinline__ cpx<T>* fft_sched(cpx<T>* a, cpx<T>* b, int G, int M, const FftPlan& plan,
                                            const cpx<T>* W, int dir) {
  switch (M) {
    case 45: return cfft_from<T, 45, 0, BIG>(a, b, G, W, dir);
    case 81: return cfft_from<T, 81, 0, BIG>(a, b, G, W, dir);
    case 125: return cfft_from<T, 125, 0, BIG>(a, b, G, W, dir);
    case 225: return cfft_from<T, 225, 0, BIG>(a, b, G, W, dir);
    case 405: return cfft_from<T, 405, 0, BIG>(a, b, G, W, dir);
    default: return fft_pencils<T>(a, b, G, M, plan, W, dir);
  }
}

// G pencils of length M with the radix schedule of the plan (picked per batch by the
// autotuner; 0 takes the precision's default).
template <typename T>
__device__ __forceinline__ cpx<T>* fft_dyn(cpx<T>* a, cpx<T>* b, int G, int M, const FftPlan& plan,
                                           const cpx<T>* W, int dir) {
  if constexpr (is_ff<T>::value) {   // float-float: the register radices only
    return fft_sched<T, true>(a, b, G, M, plan, W, dir);
  } else {
    const bool big = plan.sched == 0 ? sizeof(T) == 4 : plan.sched == 2;
    return big ? fft_sched<T, true>(a, b, G, M, plan, W, dir) : fft_sched<T, false>(a, b, G, M, plan, W, dir);
  }
}

// Column pass over a list of fields: in field f (base in + f*in_fs) a column x holds Pin
// values with stride X; it is transformed with length M and Pout values are written to
// out (stride X). dir = +1: input frequencies in FFT order of length Nlog, zero padded;
// dir = -1: Nlog kept output frequencies (Pout == Nlog) or the full M (Pout == M).
// prologue add_e: add 1 at k = 0 of field f when fe[f] is set.
template <typename U>
__device__ __noinline__ void col_pass(const cpx<U>* in, cpx<U>* out, long long in_fs, long long out_fs,
                         const int* flist, int nfl, int X, int Pin, int Pout, int Nlog, int M,
                         int dir, const FftPlan& plan, const cpx<U>* W, cpx<U>* A, cpx<U>* B, int cap,
                         const int* add_e, Team tm) {
  const int G = max(1, min(cap / M, 32));
  const int ncol = nfl * X;
  const bool pad = dir > 0 && Pin != M;
  const bool trunc = dir < 0 && Pout != M;
  const int half = (Nlog - 1) / 2;
  const FastDiv fdX((uint32_t)X);
  for (int c0 = tm.rank * G; c0 < ncol; c0 += tm.size * G) {
    const int Gc = min(G, ncol - c0);
    const FastDiv fdG((uint32_t)Gc);
    if (pad) {
      for (int t = threadIdx.x; t < Gc * M; t += blockDim.x) A[t] = mk<U>(U(0), U(0));
      __syncthreads();
    }
    for (int t = threadIdx.x; t < Gc * Pin; t += blockDim.x) {
      const int p = fdG.div(t);
      const int g = t - p * Gc;
      const int col = c0 + g;
      const int fi = fdX.div(col);
      const int x = col - fi * X;
      const int f = flist[fi];
      cpx<U> v = in[f * in_fs + (long long)p * X + x];
      if (add_e && add_e[f] && p == 0 && x == 0) v.x += U(1);
      const int pos = pad ? (p <= half ? p : p - Nlog + M) : p;
      A[g * M + pos] = v;
    }
    __syncthreads();
    cpx<U>* res = fft_dyn<U>(A, B, Gc, M, plan, W, dir);
    for (int t = threadIdx.x; t < Gc * Pout; t += blockDim.x) {
      const int i = fdG.div(t);
      const int g = t - i * Gc;
      const int col = c0 + g;
      const int fi = fdX.div(col);
      const int x = col - fi * X;
      const int f = flist[fi];
      const int pos = trunc ? (i <= half ? i : i - Nlog + M) : i;
      out[f * out_fs + (long long)i * X + x] = res[g * M + pos];
    }
    __syncthreads();
  }
}

template <typename U>
__device__ __forceinline__ void coef_apply(const U* coef, long long gi, long long cs, int ncomp, U u0, U u1,
                                           U* v0, U* v1, U scale) {
  if (ncomp == 1) {
    const U a = coef[gi] * scale;
    *v0 = a * u0;
    *v1 = a * u1;
  } else {
    const U a11 = coef[gi] * scale, a22 = coef[gi + cs] * scale, a12 = coef[gi + 2 * cs] * scale;
    *v0 = fma(a11, u0, a12 * u1);
    *v1 = fma(a12, u0, a22 * u1);
  }
}

}  // namespace homb
#include "wbatch.cuh"
namespace homb {

// Row pass along x over real rows stored as Hermitian halves of Nin values.
// mode 0: rows (r, y) pair the two components of one field: c2r, A u * scale, r2c (in place);
// mode 1: energy, rows (y, r, c) in groups of 4: accumulate u_r . A u_s into acc[4];
// mode 2: c2r only of rows (q, y) into the real coefficient.
template <typename U>
__device__ __noinline__ void row_pass(int mode, cpx<U>* rows, long long field_stride, int M1, int Nin, int Nout, int M,
                         const U* coef, int ncomp, U scale, const int* rlist, int nrl, U* coef_out,
                         const FftPlan& plan, const cpx<U>* W, cpx<U>* A, cpx<U>* B, int cap, double* acc,
                         Team tm) {
  // number of pairs in the pass and pairs per chunk
  int npairs, per_chunk;
  if (mode == 0) {
    npairs = nrl * M1;                       // (r, y)
    per_chunk = max(1, min(cap / (M + 1), 32));
  } else if (mode == 1) {
    npairs = 2 * M1;                         // (y, r): rows (c0, c1)
    per_chunk = max(2, min(cap / (M + 1), 32)) & ~1;
  } else {
    npairs = (ncomp * M1 + 1) / 2;           // consecutive rows (q, y)
    per_chunk = max(1, min(cap / (M + 1), 32));
  }
  const FftPlan& pl = plan;
  const FastDiv fdNin((uint32_t)Nin);
  const FastDiv fdNout((uint32_t)(Nout > 0 ? Nout : 1));
  const int nrows_total = ncomp * M1;
  for (int q0 = tm.rank * per_chunk; q0 < npairs; q0 += tm.size * per_chunk) {
    const int P = min(per_chunk, npairs - q0);
    const int nrow = 2 * P;
    // storage row of chunk row h (0 <= h < 2P): returns pointer offset or -1
    auto row_ptr = [&](int h) -> long long {
      const int pr = q0 + (h >> 1);
      if (mode == 0) {
        const int a = pr / M1;
        const int y = pr - a * M1;
        const int r = rlist[a];
        return (long long)(r * 2 + (h & 1)) * field_stride + (long long)y * Nin;
      } else if (mode == 1) {
        const int y = pr >> 1;
        const int r = pr & 1;
        return (long long)(r * 2 + (h & 1)) * field_stride + (long long)y * Nin;
      } else {
        const int rr = 2 * q0 + h;
        if (rr >= nrows_total) return -1;
        const int qq = rr / M1;
        const int y = rr - qq * M1;
        return (long long)qq * field_stride + (long long)y * Nin;
      }
    };
    // stage rows into B
    for (int t = threadIdx.x; t < nrow * Nin; t += blockDim.x) {
      const int h = fdNin.div(t);
      const int k = t - h * Nin;
      const long long off = row_ptr(h);
      B[t] = off >= 0 ? rows[off + k] : mk<U>(U(0), U(0));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < P * M; t += blockDim.x) {
      const int pp = t / M;
      const int k = t - pp * M;
      cpx<U> z[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = 2 * pp + h;
        cpx<U> v = mk<U>(U(0), U(0));
        if (k < Nin) {
          v = B[row * Nin + k];
          if (k == 0) v.y = U(0);
        } else if (k > M - Nin) {
          v = conj_<U>(B[row * Nin + (M - k)]);
        }
        z[h] = v;
      }
      A[pp * M + k] = mk<U>(z[0].x - z[1].y, z[0].y + z[1].x);
    }
    __syncthreads();
    cpx<U>* res = fft_dyn<U>(A, B, P, M, pl, W, +1);
    cpx<U>* oth = res == A ? B : A;
    const long long cs = (long long)M1 * M;
    if (mode == 0) {
      for (int t = threadIdx.x; t < P * M; t += blockDim.x) {
        const int pp = t / M;
        const int x = t - pp * M;
        const int pr = q0 + pp;
        const int a = pr / M1;
        const int y = pr - a * M1;
        cpx<U> z = res[pp * M + x];
        U v0, v1;
        coef_apply<U>(coef, (long long)y * M + x, cs, ncomp, z.x, z.y, &v0, &v1, scale);
        res[pp * M + x] = mk<U>(v0, v1);
      }
      __syncthreads();
      cpx<U>* r2 = fft_dyn<U>(res, oth, P, M, pl, W, -1);
      for (int t = threadIdx.x; t < nrow * Nout; t += blockDim.x) {
        const int h = fdNout.div(t);
        const int k = t - h * Nout;
        const int pp = h >> 1;
        const cpx<U> zk = r2[pp * M + k];
        const cpx<U> zm = r2[pp * M + (k == 0 ? 0 : M - k)];
        cpx<U> X;
        if ((h & 1) == 0) X = mk<U>(U(0.5) * (zk.x + zm.x), U(0.5) * (zk.y - zm.y));
        else X = mk<U>(U(0.5) * (zk.y + zm.y), U(-0.5) * (zk.x - zm.x));
        rows[row_ptr(h) + k] = X;
      }
    } else if (mode == 1) {
      for (int t = threadIdx.x; t < (P / 2) * M; t += blockDim.x) {
        const int yy = t / M;
        const int x = t - yy * M;
        const int y = (q0 >> 1) + yy;
        const cpx<U> z0 = res[(2 * yy) * M + x];       // r = 0: (c0, c1)
        const cpx<U> z1 = res[(2 * yy + 1) * M + x];   // r = 1
        U a0, a1, b0, b1;
        coef_apply<U>(coef, (long long)y * M + x, cs, ncomp, z0.x, z0.y, &a0, &a1, U(1));
        coef_apply<U>(coef, (long long)y * M + x, cs, ncomp, z1.x, z1.y, &b0, &b1, U(1));
        acc[0] += (double)z0.x * (double)a0 + (double)z0.y * (double)a1;   // W[0][0]
        acc[1] += (double)z0.x * (double)b0 + (double)z0.y * (double)b1;   // W[0][1]
        acc[2] += (double)z1.x * (double)a0 + (double)z1.y * (double)a1;   // W[1][0]
        acc[3] += (double)z1.x * (double)b0 + (double)z1.y * (double)b1;   // W[1][1]
      }
    } else {
      for (int t = threadIdx.x; t < P * M; t += blockDim.x) {
        const int pp = t / M;
        const int x = t - pp * M;
        const cpx<U> z = res[pp * M + x];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int rr = 2 * (q0 + pp) + h;
          if (rr < nrows_total) coef_out[(long long)rr * M + x] = h ? z.y : z.x;
        }
      }
    }
    __syncthreads();
  }
}

// Final column pass for the active right-hand sides: forward y transform of both
// components of field r, truncation to N1, Gamma^E/J, q written, partial p.q per rhs.
template <typename T>
__device__ __noinline__ void col_final(const cpx<T>* T2, cpx<T>* q, const cpx<T>* p, long long t2_fs, long long fld_fs,
                          const int* rlist, int nrl, int Nh, int N1, int M1, double iy0, double iy1,
                          int side, const FftPlan& plan, const cpx<T>* W, cpx<T>* A, cpx<T>* B, int cap,
                          double* pq_acc, Team tm) {
  const int G = max(1, min(cap / (2 * M1), 16));     // columns per chunk (2 pencils each)
  const int ncol = nrl * Nh;
  const FastDiv fdNh((uint32_t)Nh);
  const int half = (N1 - 1) / 2;
  for (int c0 = tm.rank * G; c0 < ncol; c0 += tm.size * G) {
    const int Gc = min(G, ncol - c0);
    const FastDiv fd2G((uint32_t)(2 * Gc));
    for (int t = threadIdx.x; t < 2 * Gc * M1; t += blockDim.x) {
      const int p_ = fd2G.div(t);
      const int g2 = t - p_ * 2 * Gc;            // (column g, component c) with c fastest
      const int g = g2 >> 1, c = g2 & 1;
      const int col = c0 + g;
      const int a = fdNh.div(col);
      const int kx = col - a * Nh;
      const int r = rlist[a];
      A[g2 * M1 + p_] = T2[(r * 2 + c) * t2_fs + (long long)p_ * Nh + kx];
    }
    __syncthreads();
    cpx<T>* res = fft_dyn<T>(A, B, 2 * Gc, M1, plan, W, -1);
    for (int t = threadIdx.x; t < Gc * N1; t += blockDim.x) {
      const int i = t / Gc;
      const int g = t - i * Gc;
      const int col = c0 + g;
      const int a = fdNh.div(col);
      const int kx = col - a * Nh;
      const int r = rlist[a];
      const int ky = i <= half ? i : i - N1;
      const int pos = ky < 0 ? ky + M1 : ky;
      cpx<T> u0 = res[(2 * g) * M1 + pos], u1 = res[(2 * g + 1) * M1 + pos];
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
      if constexpr (sizeof(T) == 4) {
        // each term in FP32, summed in FP64 (FP64 instructions issue at a small fraction of
        // the FP32 rate)
        const float sq = fmaf(p0.x, u0.x, fmaf(p0.y, u0.y, fmaf(p1.x, u1.x, p1.y * u1.y)));
        pq_acc[r] += (double)(kx == 0 ? sq : 2.f * sq);
      } else {
        const double w = kx == 0 ? 1.0 : 2.0;
        pq_acc[r] += w * ((double)p0.x * u0.x + (double)p0.y * u0.y + (double)p1.x * u1.x + (double)p1.y * u1.y);
      }
    }
    __syncthreads();
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT, NT <= 256 ? 2 : 1) k_batch(BArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_task;
  __shared__ BTask s_t;
  __shared__ double s_red[32];
  __shared__ double s_rr[2], s_alpha[2], s_beta[2], s_rrmin[2];
  __shared__ int s_active[2], s_iters[2], s_status[2], s_minit[2];
  __shared__ int s_rlist[2], s_nrl;
  __shared__ int s_flist[4], s_nfl;
  __shared__ int s_adde[4];
  __shared__ double s_xch[16];   // cluster sums: [parity][rank] (read from rank 0's copy)
  // shared memory: FP64 twiddles, working-precision twiddles, two chunk buffers (batch_smem_bytes)
  double2* W0d = reinterpret_cast<double2*>(smem);
  double2* W1d = W0d + a.M0max;
  cpx<T>* W0t = reinterpret_cast<cpx<T>*>(W1d + a.M1max);
  cpx<T>* W1t = W0t + a.M0max;
  const size_t tw_bytes = ((size_t)(a.M0max + a.M1max) * (16 + sizeof(cpx<T>)) + 15) & ~(size_t)15;
  double2* Ad = reinterpret_cast<double2*>(smem + tw_bytes);
  double2* Bd = Ad + a.cap;
  const bool f32 = sizeof(T) == 4;
  // Arithmetic of the coefficient's inverse transform and of the energies' transforms: FP64,
  // or for FP32 iterations float-float (pairs of FP32 on the FP32 pipes, about 48 bits, in
  // the same 16-byte complex slots: the FP64 tables, scratch and chunk buffers are reused)
  using E = typename std::conditional<sizeof(T) == 4, ffloat, double>::type;
  constexpr bool eff = is_ff<E>::value;
  cpx<E>* W0e = reinterpret_cast<cpx<E>*>(W0d);
  cpx<E>* W1e = reinterpret_cast<cpx<E>*>(W1d);
  cpx<E>* Ae = reinterpret_cast<cpx<E>*>(Ad);
  cpx<E>* Be = reinterpret_cast<cpx<E>*>(Bd);
  // Tasks [0, ncoop) are taken by whole clusters (the CTAs of a cluster work on one task
  // together, in the scratch slot of its rank-0 CTA); then every CTA takes tasks
  // [ncoop, ntasks) on its own. The switch happens at the same pop in every CTA of a
  // cluster, and no cluster barrier follows it.
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank(), csize = (int)cl.num_blocks();
  bool coop = csize > 1 && a.ncoop > 0;
  int parity = 0;

  for (;;) {
    Team tm{0, 1};
    int task;
    if (coop) {
      tm = Team{crank, csize};
      if (crank == 0 && threadIdx.x == 0) {
        const int tk = atomicAdd(a.counter, 1);
        for (int r = 0; r < csize; ++r) *cl.map_shared_rank(&s_task, r) = tk;
      }
      cl.sync();
      task = s_task;
      if (task >= a.ncoop) {
        coop = false;
        cl.sync();   // every CTA has read s_task before a later pop rewrites it
        continue;
      }
    } else {
      if (threadIdx.x == 0) s_task = a.ncoop + atomicAdd(a.counter2, 1);
      __syncthreads();
      task = s_task;
      if (task >= a.ntasks) break;
    }
    unsigned char* slot = a.slots + (long long)(blockIdx.x - tm.rank) * a.slot_bytes;
    {
      // the task descriptor lives in shared memory (keeps the FFT plans out of registers)
      const int* src = reinterpret_cast<const int*>(a.tasks + task);
      int* dst = reinterpret_cast<int*>(&s_t);
      for (int i = threadIdx.x; i < (int)(sizeof(BTask) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const BTask& t = s_t;
    const int M0 = t.M0, M1 = t.M1, N1 = t.N1, Nh = t.Nh, Nxs = t.Nxs;
    const int Mmax = M0 > M1 ? M0 : M1;
    // ---- slot carve-up (batch_slot_bytes)
    auto al = [](long long b) { return (b + 255) & ~255LL; };
    const long long fld = (long long)N1 * Nh;
    long long off = 0;
    double* coef64 = reinterpret_cast<double*>(slot + off);
    off += al((long long)t.ncomp * M1 * M0 * 8);
    T* coefT = f32 ? reinterpret_cast<T*>(slot + off) : reinterpret_cast<T*>(coef64);
    off += al((long long)t.ncomp * M1 * M0 * (long long)sizeof(T));
    double2* phase = reinterpret_cast<double2*>(slot + off);
    off += al((long long)(t.nincl > 0 ? t.nincl : 1) * 3 * Mmax * 16);
    double* sinc = reinterpret_cast<double*>(slot + off);
    off += al((long long)(t.nincl > 0 ? t.nincl : 1) * 3 * Mmax * 8);
    long long work_el = (long long)t.ncomp * M1 * Nxs;
    if (4LL * M1 * Nh > work_el) work_el = 4LL * M1 * Nh;
    double2* work = reinterpret_cast<double2*>(slot + off);
    off += al(work_el * 16);
    cpx<T>* vx = reinterpret_cast<cpx<T>*>(slot + off);
    off += al(4 * fld * (long long)sizeof(cpx<T>));
    cpx<T>* vr = reinterpret_cast<cpx<T>*>(slot + off);
    off += al(4 * fld * (long long)sizeof(cpx<T>));
    cpx<T>* vp = reinterpret_cast<cpx<T>*>(slot + off);
    off += al(4 * fld * (long long)sizeof(cpx<T>));
    cpx<T>* vq = reinterpret_cast<cpx<T>*>(slot + off);
    off += al(4 * fld * (long long)sizeof(cpx<T>));
    double2* x64 = reinterpret_cast<double2*>(slot + off);
    cpx<T>* T2 = reinterpret_cast<cpx<T>*>(work);
    const long long t2_fs = (long long)M1 * Nh;
    const int capT = f32 ? 2 * a.cap : a.cap;
    // FP32 iterations: warp-owned pencil passes (wbatch.cuh) where the lengths allow
    const bool wp = f32 && a.wpass != 0;
    cpx<T>* At = reinterpret_cast<cpx<T>*>(Ad);
    cpx<T>* Bt = reinterpret_cast<cpx<T>*>(Bd);

    // ---- twiddles
    for (int i = threadIdx.x; i < M0; i += blockDim.x) {
      if constexpr (eff) W0e[i] = ff2_from(a.tw64[t.tw0 + i]);
      else W0d[i] = a.tw64[t.tw0 + i];
      if (f32) reinterpret_cast<float2*>(W0t)[i] = a.tw32[t.tw0 + i];
    }
    for (int i = threadIdx.x; i < M1; i += blockDim.x) {
      if constexpr (eff) W1e[i] = ff2_from(a.tw64[t.tw1 + i]);
      else W1d[i] = a.tw64[t.tw1 + i];
      if (f32) reinterpret_cast<float2*>(W1t)[i] = a.tw32[t.tw1 + i];
    }
    const cpx<T>* W0 = f32 ? W0t : reinterpret_cast<const cpx<T>*>(W0d);
    const cpx<T>* W1 = f32 ? W1t : reinterpret_cast<const cpx<T>*>(W1d);

    // ---- coefficient (FP64): per-axis tables, spectrum on the half of Z_M, 2D inverse FFT
    SpecArgs sa;
    sa.d = 2;
    sa.ncomp = t.ncomp;
    sa.nincl = t.nincl;
    sa.M[0] = M0; sa.M[1] = M1; sa.M[2] = 1;
    sa.len[0] = Nxs; sa.len[1] = M1; sa.len[2] = 1;
    sa.Nmod[0] = M0; sa.Nmod[1] = M1; sa.Nmod[2] = 1;
    sa.invY[0] = t.invY[0]; sa.invY[1] = t.invY[1]; sa.invY[2] = 1.0;
    sa.invVol = t.invVol;
    for (int q = 0; q < 3; ++q) sa.A0p[q] = t.C0p[q];
    sa.A0p[3] = sa.A0p[4] = sa.A0p[5] = 0.0;
    sa.incl = a.incl + t.incl_off;
    sa.phase = phase;
    sa.sinc = sinc;
    sa.Mmax = Mmax;
    for (long long i = tm.tid(); i < (long long)t.nincl * 3 * Mmax; i += tm.nth()) {
      const int n = (int)(i % Mmax);
      const int al_ = (int)((i / Mmax) % 3);
      const int j = (int)(i / (3LL * Mmax));
      const int Ma = al_ == 0 ? M0 : M1;
      if (al_ >= 2 || n >= Ma) {
        phase[i] = make_double2(1.0, 0.0);
        sinc[i] = 1.0;
        continue;
      }
      const DevIncl& I = sa.incl[j];
      const int ns = sfreq(n, Ma);
      double tt = (double)ns * (I.c[al_] * t.invY[al_]);
      tt -= rint(tt);
      double sn, cs;
      sincospi(-2.0 * tt, &sn, &cs);
      phase[i] = make_double2(cs, sn);
      const double h = I.h[al_];
      const double xx = h * ns * t.invY[al_];
      sinc[i] = xx == 0.0 ? h : h * sinpi(xx) / (M_PI * xx);
    }
    team_sync(tm);
    {
      const long long plane = (long long)M1 * Nxs;
      for (long long e = tm.tid(); e < plane; e += tm.nth()) {
        const int ix = (int)(e % Nxs);
        const int iy = (int)(e / Nxs);
        const int ns[3] = {ix, sfreq(iy, M1), 0};
        const int ni[3] = {ix, iy, 0};
        double2 v[6];
        ahat_eval(sa, ni, ns, v);
        for (int q = 0; q < t.ncomp; ++q) {
          if constexpr (eff) reinterpret_cast<cpx<E>*>(work)[q * plane + e] = ff2_from(v[q]);
          else work[q * plane + e] = v[q];
        }
      }
    }
    team_sync(tm);
    {
      int flist[3] = {0, 1, 2};
      cpx<E>* workE = reinterpret_cast<cpx<E>*>(work);
      col_pass<E>(workE, workE, (long long)M1 * Nxs, (long long)M1 * Nxs, flist, t.ncomp, Nxs, M1, M1, M1, M1, +1,
                  t.plan1, W1e, Ae, Be, a.cap, nullptr, tm);
      team_sync(tm);
      double dummy[4];
      row_pass<E>(2, workE, (long long)M1 * Nxs, M1, Nxs, 0, M0, nullptr, t.ncomp, E(1.0), nullptr, 0,
                  reinterpret_cast<E*>(coef64), t.plan0, W0e, Ae, Be, a.cap, dummy, tm);
      team_sync(tm);
    }
    if (f32) {
      for (long long i = tm.tid(); i < (long long)t.ncomp * M1 * M0; i += tm.nth()) {
        if constexpr (eff) coefT[i] = T(ff_norm(reinterpret_cast<const E*>(coef64)[i]).hi);
        else coefT[i] = T(coef64[i]);
      }
      team_sync(tm);
    }

    // ---- right-hand sides, x = p = 0
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long e = tm.tid(); e < fld; e += tm.nth()) {
      const int kx = (int)(e % Nh);
      const int iy = (int)(e / Nh);
      const int ns[3] = {kx, sfreq(iy, N1), 0};
      const int ni[3] = {kx, ns[1] < 0 ? ns[1] + M1 : ns[1], 0};
      double2 Ah[6];
      ahat_eval(sa, ni, ns, Ah);
      const double xi0 = kx * t.invY[0], xi1 = ns[1] * t.invY[1];
      const double n2 = xi0 * xi0 + xi1 * xi1;
      const double w = kx == 0 ? 1.0 : 2.0;
      for (int r = 0; r < 2; ++r) {
        double2 v0, v1;
        if (t.ncomp == 1) {
          v0 = r == 0 ? Ah[0] : make_double2(0.0, 0.0);
          v1 = r == 1 ? Ah[0] : make_double2(0.0, 0.0);
        } else {
          v0 = Ah[sym_index(2, 0, r)];
          v1 = Ah[sym_index(2, 1, r)];
        }
        double2 g0 = make_double2(0.0, 0.0), g1 = g0;
        if (n2 > 0.0) {
          const double dx = (xi0 * v0.x + xi1 * v1.x) / n2, dy = (xi0 * v0.y + xi1 * v1.y) / n2;
          g0 = make_double2(xi0 * dx, xi0 * dy);
          g1 = make_double2(xi1 * dx, xi1 * dy);
          if (t.side == 1) {
            g0 = make_double2(v0.x - g0.x, v0.y - g0.y);
            g1 = make_double2(v1.x - g1.x, v1.y - g1.y);
          }
        }
        const cpx<T> b0 = mk<T>(T(-g0.x), T(-g0.y)), b1 = mk<T>(T(-g1.x), T(-g1.y));
        vr[(r * 2 + 0) * fld + e] = b0;
        vr[(r * 2 + 1) * fld + e] = b1;
        const cpx<T> z = mk<T>(T(0), T(0));
        vx[(r * 2 + 0) * fld + e] = z;
        vx[(r * 2 + 1) * fld + e] = z;
        vp[(r * 2 + 0) * fld + e] = z;
        vp[(r * 2 + 1) * fld + e] = z;
        acc[r] += w * ((double)b0.x * b0.x + (double)b0.y * b0.y + (double)b1.x * b1.x + (double)b1.y * b1.y);
      }
    }
    const double scale = 1.0 / ((double)M0 * M1);
    const long long io_off = ((long long)t.prob * 2 + t.side) * 4 * fld;   // start of this task's block
    if (a.x0) {
      // warm start: x = Gamma x0, r = b - C x (one operator application), p = 0
      team_sync(tm);
      const cpx<T>* x0 = reinterpret_cast<const cpx<T>*>(a.x0) + io_off;
      for (long long e = tm.tid(); e < 2 * fld; e += tm.nth()) {
        const int r = (int)(e / fld);
        const long long k = e - r * fld;
        const int kx = (int)(k % Nh);
        const int iy = (int)(k / Nh);
        const T xi0 = T(kx * t.invY[0]), xi1 = T(sfreq(iy, N1) * t.invY[1]);
        const T n2 = xi0 * xi0 + xi1 * xi1;
        const cpx<T> u0 = x0[(r * 2 + 0) * fld + k], u1 = x0[(r * 2 + 1) * fld + k];
        cpx<T> g0 = mk<T>(T(0), T(0)), g1 = g0;
        if (n2 > T(0)) {
          const T dx = (xi0 * u0.x + xi1 * u1.x) / n2, dy = (xi0 * u0.y + xi1 * u1.y) / n2;
          g0 = mk<T>(xi0 * dx, xi0 * dy);
          g1 = mk<T>(xi1 * dx, xi1 * dy);
          if (t.side == 1) {
            g0 = sub<T>(u0, g0);
            g1 = sub<T>(u1, g1);
          }
        }
        vx[(r * 2 + 0) * fld + k] = g0;
        vx[(r * 2 + 1) * fld + k] = g1;
        vp[(r * 2 + 0) * fld + k] = g0;
        vp[(r * 2 + 1) * fld + k] = g1;
      }
      if (threadIdx.x == 0) {
        s_rlist[0] = 0; s_rlist[1] = 1; s_nrl = 2;
        s_flist[0] = 0; s_flist[1] = 1; s_flist[2] = 2; s_flist[3] = 3; s_nfl = 4;
      }
      team_sync(tm);
      if (!(wp && wcol_pass_any<T>(M1, vp, T2, fld, t2_fs, s_flist, s_nfl, Nh, N1, W1, At, capT, tm)))
        col_pass<T>(vp, T2, fld, t2_fs, s_flist, s_nfl, Nh, N1, M1, N1, M1, +1, t.plan1, W1, At, Bt, capT, nullptr,
                    tm);
      team_sync(tm);
      double dummy0[4];
      if (!(wp && wrow_pass_any<T>(M0, T2, t2_fs, M1, Nh, coefT, t.ncomp, T(scale), s_rlist, s_nrl, W0, At, capT,
                                   tm)))
        row_pass<T>(0, T2, t2_fs, M1, Nh, Nh, M0, coefT, t.ncomp, T(scale), s_rlist, s_nrl, nullptr, t.plan0, W0,
                    At, Bt, capT, dummy0, tm);
      team_sync(tm);
      double pqd[2] = {0.0, 0.0};
      if (!(wp && wcol_final_any<T>(M1, T2, vq, vp, t2_fs, fld, s_rlist, s_nrl, Nh, N1, t.invY[0], t.invY[1], t.side,
                                    W1, At, capT, pqd, tm)))
        col_final<T>(T2, vq, vp, t2_fs, fld, s_rlist, s_nrl, Nh, N1, M1, t.invY[0], t.invY[1], t.side, t.plan1, W1,
                     At, Bt, capT, pqd, tm);
      // Rayleigh-Ritz on span{x0}: x = s x0 with s = (x0.b)/(x0.C x0) minimises the energy
      // functional along the start direction, so a start never does worse than x = 0
      double xb[2] = {0.0, 0.0};
      for (long long i = tm.tid(); i < 4 * fld; i += tm.nth()) {
        const int r = (int)(i / (2 * fld));
        const cpx<T> pv = vp[i], bv = vr[i];
        const double w = (i % Nh) == 0 ? 1.0 : 2.0;
        xb[r] += w * ((double)pv.x * bv.x + (double)pv.y * bv.y);
      }
      for (int r = 0; r < 2; ++r) {
        const double num = team_sum(tm, xb[r], s_red, s_xch, parity);
        const double den = team_sum(tm, pqd[r], s_red, s_xch, parity);   // x0 . C x0 (col_final's partial sums)
        if (threadIdx.x == 0) {
          const double s_ = den > 0.0 ? num / den : 0.0;
          s_alpha[r] = isfinite(s_) ? s_ : 0.0;
        }
      }
      __syncthreads();
      acc[0] = acc[1] = 0.0;
      for (long long i = tm.tid(); i < 4 * fld; i += tm.nth()) {
        const int r = (int)(i / (2 * fld));
        const T sr = T(s_alpha[r]);
        const cpx<T> xv = vx[i], qv = vq[i];
        vx[i] = mk<T>(sr * xv.x, sr * xv.y);
        const cpx<T> rv = mk<T>(fma(-sr, qv.x, vr[i].x), fma(-sr, qv.y, vr[i].y));
        vr[i] = rv;
        vp[i] = mk<T>(T(0), T(0));
        const double w = (i % Nh) == 0 ? 1.0 : 2.0;
        acc[r] += w * ((double)rv.x * rv.x + (double)rv.y * rv.y);
      }
    }
    for (int r = 0; r < 2; ++r) {
      const double s = team_sum(tm, acc[r], s_red, s_xch, parity);
      if (threadIdx.x == 0) {
        s_rr[r] = s;
        s_rrmin[r] = s;
        s_minit[r] = 0;
        s_beta[r] = 0.0;
        s_iters[r] = 0;
        s_active[r] = s > a.tol2 ? 1 : 0;
        s_status[r] = isfinite(s) ? 0 : -2;
        if (!isfinite(s)) s_active[r] = 0;
      }
    }
    __syncthreads();

    // ---- CG on both right-hand sides
    for (int it = 0; it < a.max_iter && (s_active[0] || s_active[1]); ++it) {
      if (threadIdx.x == 0) {
        int n = 0, m = 0;
        for (int r = 0; r < 2; ++r)
          if (s_active[r]) {
            s_rlist[n++] = r;
            s_flist[m++] = 2 * r;
            s_flist[m++] = 2 * r + 1;
          }
        s_nrl = n;
        s_nfl = m;
      }
      __syncthreads();
      // p = r + beta p (per right-hand side: 32-bit indices, no division per element)
      const int n2f = (int)(2 * fld);
      const int tid0 = (int)tm.tid(), nth = (int)tm.nth();
      for (int r = 0; r < 2; ++r) {
        if (!s_active[r]) continue;
        const T b = T(s_beta[r]);
        cpx<T>* pr_ = vp + (long long)r * n2f;
        const cpx<T>* rr_ = vr + (long long)r * n2f;
        for (int i = tid0; i < n2f; i += nth) {
          const cpx<T> pv = pr_[i], rv = rr_[i];
          pr_[i] = mk<T>(fma(b, pv.x, rv.x), fma(b, pv.y, rv.y));
        }
      }
      team_sync(tm);
      if (!(wp && wcol_pass_any<T>(M1, vp, T2, fld, t2_fs, s_flist, s_nfl, Nh, N1, W1, At, capT, tm)))
        col_pass<T>(vp, T2, fld, t2_fs, s_flist, s_nfl, Nh, N1, M1, N1, M1, +1, t.plan1, W1, At, Bt, capT,
                    nullptr, tm);
      team_sync(tm);
      double dummy[4];
      if (!(wp && wrow_pass_any<T>(M0, T2, t2_fs, M1, Nh, coefT, t.ncomp, T(scale), s_rlist, s_nrl, W0, At, capT,
                                   tm)))
        row_pass<T>(0, T2, t2_fs, M1, Nh, Nh, M0, coefT, t.ncomp, T(scale), s_rlist, s_nrl, nullptr, t.plan0, W0,
                    At, Bt, capT, dummy, tm);
      team_sync(tm);
      double pq[2] = {0.0, 0.0};
      if (!(wp && wcol_final_any<T>(M1, T2, vq, vp, t2_fs, fld, s_rlist, s_nrl, Nh, N1, t.invY[0], t.invY[1], t.side,
                                    W1, At, capT, pq, tm)))
        col_final<T>(T2, vq, vp, t2_fs, fld, s_rlist, s_nrl, Nh, N1, M1, t.invY[0], t.invY[1], t.side, t.plan1, W1,
                     At, Bt, capT, pq, tm);
      for (int r = 0; r < 2; ++r) {
        const double s = team_sum(tm, pq[r], s_red, s_xch, parity);
        if (threadIdx.x == 0 && s_active[r]) {
          if (!(s > 0.0) || !isfinite(s)) {
            s_active[r] = 0;
            s_status[r] = f32 ? 2 : -2;
            s_alpha[r] = 0.0;
          } else {
            s_alpha[r] = s_rr[r] / s;
          }
        }
      }
      __syncthreads();
      double rr[2] = {0.0, 0.0};
      const FastDiv fdNh((uint32_t)Nh);
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        if (!s_active[r]) continue;
        const T al_ = T(s_alpha[r]);
        const long long o = (long long)r * n2f;
        double acc_r = 0.0;
        float run = 0.f;   // FP32: runs of up to 8 terms, summed in FP64
        int cnt = 0;
        for (int i = tid0; i < n2f; i += nth) {
          const cpx<T> pv = vp[o + i], qv = vq[o + i];
          cpx<T> xv = vx[o + i], rv = vr[o + i];
          xv = mk<T>(fma(al_, pv.x, xv.x), fma(al_, pv.y, xv.y));
          rv = mk<T>(fma(-al_, qv.x, rv.x), fma(-al_, qv.y, rv.y));
          vx[o + i] = xv;
          vr[o + i] = rv;
          const bool k0 = i - (int)fdNh.div(i) * Nh == 0;
          if constexpr (sizeof(T) == 4) {
            const float sq = fmaf(rv.x, rv.x, rv.y * rv.y);
            run = fmaf(k0 ? 1.f : 2.f, sq, run);
            if (++cnt == 8) {
              acc_r += (double)run;
              run = 0.f;
              cnt = 0;
            }
          } else {
            acc_r += (k0 ? 1.0 : 2.0) * ((double)rv.x * rv.x + (double)rv.y * rv.y);
          }
        }
        rr[r] = acc_r + (double)run;
      }
      for (int r = 0; r < 2; ++r) {
        const double s = team_sum(tm, rr[r], s_red, s_xch, parity);
        if (threadIdx.x == 0 && s_active[r]) {
          s_iters[r] += 1;
          if (!isfinite(s)) {
            s_active[r] = 0;
            s_status[r] = f32 ? 2 : -2;
          } else if (s <= a.tol2) {
            s_active[r] = 0;
            s_status[r] = 0;
            s_rr[r] = s;
          } else if (f32 && (s > 1e4 * s_rrmin[r] || s_iters[r] - s_minit[r] > 40)) {
            s_active[r] = 0;
            s_status[r] = 2;
            s_rr[r] = s;
          } else {
            s_beta[r] = s / s_rr[r];
            s_rr[r] = s;
            if (s < s_rrmin[r]) {
              s_rrmin[r] = s;
              s_minit[r] = s_iters[r];
            }
          }
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0)
      for (int r = 0; r < 2; ++r)
        if (s_active[r]) s_status[r] = 1;   // max_iter reached
    __syncthreads();

    if (a.fields) {
      cpx<T>* fo = reinterpret_cast<cpx<T>*>(a.fields) + io_off;
      for (long long i = tm.tid(); i < 4 * fld; i += tm.nth()) fo[i] = vx[i];
    }
    // ---- FP64 re-projection of the fields and the exact double-grid energies
    for (long long e = tm.tid(); e < 2 * fld; e += tm.nth()) {
      const int r = (int)(e / fld);
      const long long k = e - r * fld;
      const int kx = (int)(k % Nh);
      const int iy = (int)(k / Nh);
      const double xi0 = kx * t.invY[0], xi1 = sfreq(iy, N1) * t.invY[1];
      const double n2 = xi0 * xi0 + xi1 * xi1;
      const cpx<T> a0 = vx[(r * 2 + 0) * fld + k], a1 = vx[(r * 2 + 1) * fld + k];
      double2 u0 = make_double2((double)a0.x, (double)a0.y), u1 = make_double2((double)a1.x, (double)a1.y);
      double2 g0 = make_double2(0.0, 0.0), g1 = g0;
      if (n2 > 0.0) {
        const double dx = (xi0 * u0.x + xi1 * u1.x) / n2, dy = (xi0 * u0.y + xi1 * u1.y) / n2;
        g0 = make_double2(xi0 * dx, xi0 * dy);
        g1 = make_double2(xi1 * dx, xi1 * dy);
        if (t.side == 1) {
          g0 = make_double2(u0.x - g0.x, u0.y - g0.y);
          g1 = make_double2(u1.x - g1.x, u1.y - g1.y);
        }
      }
      if constexpr (eff) {
        reinterpret_cast<cpx<E>*>(x64)[(r * 2 + 0) * fld + k] = ff2_from(g0);
        reinterpret_cast<cpx<E>*>(x64)[(r * 2 + 1) * fld + k] = ff2_from(g1);
      } else {
        x64[(r * 2 + 0) * fld + k] = g0;
        x64[(r * 2 + 1) * fld + k] = g1;
      }
    }
    if (threadIdx.x == 0) {
      s_flist[0] = 0; s_flist[1] = 1; s_flist[2] = 2; s_flist[3] = 3;
      s_adde[0] = 1; s_adde[1] = 0; s_adde[2] = 0; s_adde[3] = 1;   // e_r in component r of field r
    }
    team_sync(tm);
    col_pass<E>(reinterpret_cast<cpx<E>*>(x64), reinterpret_cast<cpx<E>*>(work), fld, t2_fs, s_flist, 4, Nh, N1, M1,
                N1, M1, +1, t.plan1, W1e, Ae, Be, a.cap, s_adde, tm);
    team_sync(tm);
    double eacc[4] = {0.0, 0.0, 0.0, 0.0};
    row_pass<E>(1, reinterpret_cast<cpx<E>*>(work), t2_fs, M1, Nh, 0, M0, reinterpret_cast<const E*>(coef64), t.ncomp,
                E(1.0), nullptr, 0, nullptr, t.plan0, W0e, Ae, Be, a.cap, eacc, tm);
    for (int i = 0; i < 4; ++i) {
      const double s = team_sum(tm, eacc[i], s_red, s_xch, parity);
      if (threadIdx.x == 0 && tm.rank == 0) a.energy[(long long)task * 4 + i] = s * scale;
    }
    if (threadIdx.x == 0 && tm.rank == 0)
      for (int r = 0; r < 2; ++r) {
        a.iters[task * 2 + r] = s_iters[r];
        a.status[task * 2 + r] = s_status[r];
        a.resid[task * 2 + r] = sqrt(fmax(s_rr[r], 0.0));
      }
    team_sync(tm);
  }
}

template <typename T, int NT>
cudaError_t launch_batch_nt(const BArgs& a, int nblocks, size_t smem, int cluster, cudaStream_t s) {
  static std::atomic<int> cache[kAttrDevices] = {};
  const cudaError_t e = smem_attr(k_batch<T, NT>, smem, cache);
  if (e != cudaSuccess) return e;
  if (cluster <= 1) {
    k_batch<T, NT><<<nblocks, NT, smem, s>>>(a);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nblocks);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_batch<T, NT>, a);
}

template <typename T>
cudaError_t launch_batch(const BArgs& a, int nblocks, size_t smem, int threads, int cluster, cudaStream_t s) {
  if (cluster != 1 && cluster != 2 && cluster != 4 && cluster != 8) return cudaErrorInvalidValue;
  if (nblocks % cluster) return cudaErrorInvalidValue;
  switch (threads) {
    case 256: return launch_batch_nt<T, 256>(a, nblocks, smem, cluster, s);
    case 512: return launch_batch_nt<T, 512>(a, nblocks, smem, cluster, s);
    case 1024: return launch_batch_nt<T, 1024>(a, nblocks, smem, cluster, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int NT> int batch_max_blocks_nt(size_t smem, int cluster) {
  static std::atomic<int> cache[kAttrDevices] = {};
  if (smem_attr(k_batch<T, NT>, smem, cache) != cudaSuccess) return 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
  if (cluster <= 1) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<T, NT>, NT, smem) != cudaSuccess || n < 1) n = 1;
    return n * sms;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster * sms);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, k_batch<T, NT>, &cfg) != cudaSuccess || nc < 1) {
    cudaGetLastError();
    return 0;   // this cluster shape cannot be placed
  }
  return nc * cluster;
}

template <typename T> int batch_max_blocks(size_t smem, int threads, int cluster) {
  switch (threads) {
    case 512: return batch_max_blocks_nt<T, 512>(smem, cluster);
    case 1024: return batch_max_blocks_nt<T, 1024>(smem, cluster);
    default: return batch_max_blocks_nt<T, 256>(smem, cluster);
  }
}
template int batch_max_blocks<double>(size_t, int, int);
template int batch_max_blocks<float>(size_t, int, int);

template cudaError_t launch_batch<double>(const BArgs&, int, size_t, int, int, cudaStream_t);
template cudaError_t launch_batch<float>(const BArgs&, int, size_t, int, int, cudaStream_t);

}  // namespace homb
