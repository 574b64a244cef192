// CUDA kernels of the double-grid Galerkin operator, the coefficient build, the CG
// vector updates and the deterministic reductions (sm_103a).
//
// Operator (Lemma double-grid, Eq. MBA_GA, structure of Eq. linear_system_primal):
//   C u = Gamma P_N F_M (A_M/|M|) F_M^{-1} Pad(u),  M = 2N-1,
// applied to half-spectrum fields as a chain of pencil passes: inverse transforms
// along z and y with zero padding, a row pass along x (Hermitian-half c2r, pointwise
// coefficient, r2c), forward transforms along y and z with truncation, and Gamma in
// the epilogue of the last pass together with the CG partial sum p.Cp.
#include <math.h>

#include <algorithm>

#include "kernels.cuh"
#include "spectrum.cuh"

namespace homb {

constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ void load_twiddles(cpx<T>* Ws, const void* W, int M) {
  const cpx<T>* w = reinterpret_cast<const cpx<T>*>(W);
  for (int t = threadIdx.x; t < M; t += blockDim.x) Ws[t] = w[t];
}

// ---------------------------------------------------------------------------------
// closed-form Fourier coefficients of the matrix-inclusion coefficient
// ---------------------------------------------------------------------------------
__global__ void k_axis_tables(int nincl, int d, int M0, int M1, int M2, int Mmax, double iy0,
                              double iy1, double iy2, const DevIncl* incl, double2* phase,
                              double* sinc) {
  const int Ms[3] = {M0, M1, M2};
  const double invY[3] = {iy0, iy1, iy2};
  const long long total = (long long)nincl * 3 * Mmax;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(t % Mmax);
    const int al = (int)((t / Mmax) % 3);
    const int j = (int)(t / (3LL * Mmax));
    if (al >= d || n >= Ms[al]) {
      phase[t] = make_double2(1.0, 0.0);
      sinc[t] = 1.0;
      continue;
    }
    const int ns = sfreq(n, Ms[al]);
    double tt = (double)ns * (incl[j].c[al] * invY[al]);
    tt -= rint(tt);
    double s, c;
    sincospi(-2.0 * tt, &s, &c);
    phase[t] = make_double2(c, s);
    const double h = incl[j].h[al];
    const double x = h * ns * invY[al];
    sinc[t] = x == 0.0 ? h : h * sinpi(x) / (M_PI * x);
  }
}

__global__ void k_spectrum(SpecArgs a, double2* out) {
  const long long plane = (long long)a.len[0] * a.len[1];
  const long long total = plane * a.len[2];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(e % a.len[0]);
    const int iy = (int)((e / a.len[0]) % a.len[1]);
    const int iz = (int)(e / plane);
    const int ns[3] = {ix, sfreq(iy, a.Nmod[1]), a.d == 3 ? sfreq(iz, a.Nmod[2]) : 0};
    const int ni[3] = {ix, ns[1] < 0 ? ns[1] + a.M[1] : ns[1], ns[2] < 0 ? ns[2] + a.M[2] : ns[2]};
    double2 v[6];
    ahat_eval(a, ni, ns, v);
    for (int q = 0; q < a.ncomp; ++q) out[q * total + e] = v[q];
  }
}

// b_r(k) = -Gamma(k) A_hat(k) e_r for every right-hand side r < nrhs from one evaluation of
// A_hat(k) per frequency (the closed form is the costly part: FP64 transcendental functions and
// a phase product per inclusion), with the |b_r|^2 partials of each r. With `hat` the values
// A_hat(k) are read instead ([ncomp][N2][N1][Nh], e.g. from launch_spectrum_ff on the N grid).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_rhs(SpecArgs a, int side, int nrhs, int Nh, int N1, int N2,
                                                   cpx<T>* b, double* partial, int ld, const double2* hat) {
  __shared__ double red[32];
  const int C = a.d;
  const int field = Nh * N1 * N2;   // < 2^31 (checked by the launcher)
  const FastDiv fdNh((uint32_t)Nh), fdN1((uint32_t)N1);
  double acc[3] = {0.0, 0.0, 0.0};
  for (long long el = blockIdx.x * (long long)blockDim.x + threadIdx.x; el < field;
       el += (long long)gridDim.x * blockDim.x) {
    const int e = (int)el;
    const int q1 = fdNh.div(e);
    const int kx = e - q1 * Nh;
    const int iz = fdN1.div(q1);
    const int iy = q1 - iz * N1;
    const int ns[3] = {kx, sfreq(iy, N1), a.d == 3 ? sfreq(iz, N2) : 0};
    const int ni[3] = {kx, ns[1] < 0 ? ns[1] + a.M[1] : ns[1], ns[2] < 0 ? ns[2] + a.M[2] : ns[2]};
    double2 Ah[6];
    if (hat) {
      for (int q = 0; q < a.ncomp; ++q) Ah[q] = hat[(long long)q * field + e];
    } else {
      ahat_eval(a, ni, ns, Ah);
    }
    double xi[3], n2 = 0.0;
    for (int c = 0; c < C; ++c) {
      xi[c] = ns[c] * a.invY[c];
      n2 += xi[c] * xi[c];
    }
    const double w = kx == 0 ? 1.0 : 2.0;
    const bool nyq = nyquist(ns[1], N1) || (a.d == 3 && nyquist(ns[2], N2));
    const double inv = n2 > 0.0 ? 1.0 / n2 : 0.0;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (r >= nrhs) break;
      double2 v[3];
      double2 dot = make_double2(0.0, 0.0);
      for (int c = 0; c < C; ++c) {
        if (a.ncomp == 1) v[c] = c == r ? Ah[0] : make_double2(0.0, 0.0);
        else v[c] = Ah[sym_index(a.d, c, r)];
        dot.x += xi[c] * v[c].x;
        dot.y += xi[c] * v[c].y;
      }
      dot = make_double2(dot.x * inv, dot.y * inv);
      for (int c = 0; c < C; ++c) {
        double2 g = make_double2(0.0, 0.0);
        if (n2 > 0.0 && !nyq) {
          const double2 ge = make_double2(xi[c] * dot.x, xi[c] * dot.y);
          g = side == 0 ? ge : make_double2(v[c].x - ge.x, v[c].y - ge.y);
        }
        const cpx<T> bv = mk<T>(T(-g.x), T(-g.y));
        b[((long long)r * C + c) * field + e] = bv;
        acc[r] += w * ((double)bv.x * bv.x + (double)bv.y * bv.y);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    if (r >= nrhs) break;
    const double s = block_sum(acc[r], red);
    if (threadIdx.x == 0) partial[r * ld + blockIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------------
// CG vector update and scalar kernels (one CTA), deterministic reductions
// ---------------------------------------------------------------------------------
__device__ double reduce_row(const double* v, int n, double* red);

// CG step of one right-hand side: alpha = r.r / p.Cp from the last operator pass's partial
// sums pq_part[rhs][pq_nblk] (every CTA forms the same sum in the same order, so all agree;
// CTA 0 records alpha and p.Cp, or the breakdown p.Cp <= 0 / non-finite, which stops the
// right-hand side in every CTA), then x += alpha p, r -= alpha Cp and the |r|^2 partials.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_cg_update(cpx<T>* x, cpx<T>* r, const cpx<T>* p,
                                                         const cpx<T>* q, int C, long long field,
                                                         FastDiv fdNh, CgScalars* cg, double* partial,
                                                         int ld, const double* pq_part, int pq_ld,
                                                         int pq_nblk) {
  __shared__ double red[32];
  __shared__ double s_alpha;
  __shared__ int s_on;
  const int rhs = blockIdx.y;
  if (!cg->active[rhs]) return;
  const double pq = reduce_row(pq_part + (long long)rhs * pq_ld, pq_nblk, red);
  if (threadIdx.x == 0) {
    const bool ok = pq > 0.0 && isfinite(pq);
    s_on = ok ? 1 : 0;
    s_alpha = ok ? cg->rr[rhs] / pq : 0.0;
    if (blockIdx.x == 0) {
      cg->pq[rhs] = pq;
      if (ok) {
        cg->alpha[rhs] = s_alpha;
      } else {
        cg->active[rhs] = 0;
        cg->status[rhs] = cg->guard ? 2 : -2;
      }
    }
  }
  __syncthreads();
  if (!s_on) return;
  const T al = T(s_alpha);
  const long long n = (long long)C * field;
  const long long base = (long long)rhs * n;
  double acc = 0.0;
  // FP32 vectors: each |r|^2 term and runs of up to 8 terms in FP32, the sum of the runs over
  // the thread and the block in FP64 (on this GPU an FP64 instruction issues at 1/64 of the
  // FP32 rate: converting and multiplying every term in FP64 made this pass FP64-bound)
  float run = 0.f;
  int cnt = 0;
  // four entries per thread and iteration: their 16 loads are in flight together
  constexpr int U = 4;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; e0 < n; e0 += U * stride) {
    cpx<T> pv[U], qv[U], xv[U], rv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long e = e0 + u * stride;
      if (e < n) {
        pv[u] = p[base + e];
        qv[u] = q[base + e];
        xv[u] = x[base + e];
        rv[u] = r[base + e];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long e = e0 + u * stride;
      if (e >= n) break;
      xv[u] = mk<T>(fma(al, pv[u].x, xv[u].x), fma(al, pv[u].y, xv[u].y));
      rv[u] = mk<T>(fma(-al, qv[u].x, rv[u].x), fma(-al, qv[u].y, rv[u].y));
      x[base + e] = xv[u];
      r[base + e] = rv[u];
      const int ei = (int)e;   // < 2^31 elements per right-hand side (checked by the launcher)
      const bool k0 = ei - fdNh.div(ei) * (int)fdNh.d == 0;
      if constexpr (sizeof(T) == 4) {
        run = fmaf(k0 ? 1.f : 2.f, fmaf(rv[u].x, rv[u].x, rv[u].y * rv[u].y), run);
        if (++cnt == 8) {
          acc += (double)run;
          run = 0.f;
          cnt = 0;
        }
      } else {
        acc += (k0 ? 1.0 : 2.0) * ((double)rv[u].x * rv[u].x + (double)rv[u].y * rv[u].y);
      }
    }
  }
  acc += (double)run;
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partial[rhs * ld + blockIdx.x] = s;
}

__device__ double reduce_row(const double* v, int n, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
  s = block_sum(s, red);
  return s;  // thread 0
}

// Absolute target of an inner solve that starts from |r0|^2 = s (see launch_cg_init)
__device__ __forceinline__ double inner_target(double tol2_abs, double tol2_hi, double drift, double s) {
  if (!(drift > 0.0) || !isfinite(s)) return tol2_abs;
  const double t = sqrt(tol2_hi) - drift * sqrt(s);
  return t > 0.0 ? fmax(tol2_abs, t * t) : tol2_abs;
}

__global__ void k_cg_init(CgScalars* cg, const double* partial, int ld, int nblk, int nrhs,
                          double tol2_abs, double rel2, int guard, double tol2_hi, double drift) {
  __shared__ double red[32];
  for (int r = 0; r < 3; ++r) {
    double s = 0.0;
    if (r < nrhs) s = reduce_row(partial + (long long)r * ld, nblk, red);
    __syncthreads();
    if (threadIdx.x == 0) {
      const double t2 = fmax(inner_target(tol2_abs, tol2_hi, drift, s), rel2 * s);
      cg->tol2[r] = t2;
      cg->beta[r] = 0.0;
      cg->alpha[r] = 0.0;
      cg->iters[r] = 0;
      cg->rr[r] = s;
      cg->rr_min[r] = s;
      cg->min_iter[r] = 0;
      cg->guard = guard;
      cg->fault = 0;
      if (r >= nrhs) {
        cg->active[r] = 0;
        cg->status[r] = 0;
      } else if (!isfinite(s)) {
        cg->active[r] = 0;
        cg->status[r] = -2;
      } else {
        cg->active[r] = s > t2 ? 1 : 0;
        cg->status[r] = s > t2 ? 1 : 0;
      }
    }
  }
}

// Three block sums at once, each in block_sum's order (thread strides, then the warp
// shuffle tree, then the warps in order by thread 0): the loads and the shuffles of the
// right-hand sides overlap instead of running one reduction after another.
__device__ __forceinline__ void block_sum3(double (&v)[3], double (*red)[32]) {
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < 3; ++c) red[c][wid] = v[c];
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += red[c][w];
      v[c] = t;
    }
  }
}

// The beta step: r.r of every right-hand side from the partials, then per right-hand side
// (one thread each) the stopping tests and beta = r.r / r.r_old. Each thread loads its
// side's scalars together before it stores any of them, so that the small kernel waits for
// one round of memory latency instead of a chain of dependent loads.
__global__ void k_cg_beta(CgScalars* cg, const double* partial, int ld, int nblk, int nrhs) {
  __shared__ double red[3][32];
  __shared__ double s_rr[3];
  double v[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int r = 0; r < 3; ++r)
    if (r < nrhs)
      for (int i = threadIdx.x; i < nblk; i += blockDim.x) v[r] += partial[(long long)r * ld + i];
  block_sum3(v, red);
  if (threadIdx.x == 0)
    for (int r = 0; r < 3; ++r) s_rr[r] = v[r];
  __syncthreads();
  const int r = threadIdx.x;
  if (r >= nrhs) return;
  const int active = cg->active[r], guard = cg->guard, it = cg->iters[r] + 1, min_iter = cg->min_iter[r];
  const double tol2 = cg->tol2[r], rr_min = cg->rr_min[r], rr_old = cg->rr[r];
  if (!active) return;
  const double rr = s_rr[r];
  cg->iters[r] = it;
  if (!isfinite(rr)) {
    cg->active[r] = 0;
    cg->status[r] = guard ? 2 : -2;
  } else if (rr <= tol2) {
    cg->active[r] = 0;
    cg->status[r] = 0;
    cg->rr[r] = rr;
  } else if (guard && (rr > 1e4 * rr_min || it - min_iter > 40)) {
    // FP32 inner solve diverging or stagnating at its accuracy floor: stop, keep x
    cg->active[r] = 0;
    cg->status[r] = 2;
    cg->rr[r] = rr;
  } else {
    cg->beta[r] = rr / rr_old;
    cg->rr[r] = rr;
    if (rr < rr_min) {
      cg->rr_min[r] = rr;
      cg->min_iter[r] = it;
    }
  }
}

__global__ void k_outer_check(CgScalars* cg, const double* partial, int ld, int nblk, int nrhs,
                              double shrink2) {
  __shared__ double red[32];
  for (int r = 0; r < nrhs; ++r) {
    if (!cg->active[r]) continue;
    const double rr = reduce_row(partial + (long long)r * ld, nblk, red);
    __syncthreads();
    if (threadIdx.x == 0) {
      cg->iters[r] += 1;
      if (!isfinite(rr)) {
        cg->active[r] = 0;
        cg->status[r] = -2;
      } else if (rr <= cg->tol2[r]) {
        cg->active[r] = 0;
        cg->status[r] = 0;
        cg->rr[r] = rr;
      } else if (rr > shrink2 * cg->rr[r]) {
        cg->active[r] = 0;   // refinement stalled: the field is kept, bounds stay guaranteed
        cg->status[r] = 1;
        cg->rr[r] = rr;
      } else {
        cg->rr[r] = rr;
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads) k_demote(const double2* r64, float2* r32, int C,
                                                      long long field, FastDiv fdNh, const CgScalars* outer,
                                                      double* partial, int ld) {
  __shared__ double red[32];
  const int rhs = blockIdx.y;
  const bool on = outer->active[rhs] != 0;
  const long long n = (long long)C * field;
  const long long base = (long long)rhs * n;
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    float2 v = make_float2(0.f, 0.f);
    if (on) {
      const double2 w = r64[base + e];
      v = make_float2((float)w.x, (float)w.y);
    }
    r32[base + e] = v;
    const int ei = (int)e;
    const double wt = ei - fdNh.div(ei) * (int)fdNh.d == 0 ? 1.0 : 2.0;
    acc += wt * ((double)v.x * v.x + (double)v.y * v.y);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partial[rhs * ld + blockIdx.x] = s;
}

__global__ void k_promote_add(const float2* x32, double2* x64, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 a = x32[i];
    double2 b = x64[i];
    b.x += (double)a.x;
    b.y += (double)a.y;
    x64[i] = b;
  }
}

// GaNi coefficient (Def. GaNi, Eq. grid_points): the side's coefficient sampled at the grid
// points x_k = k_a Y_a / N_a of the M = N grid (FFT storage order), packed symmetric
// [q][j3][j2][j1]. A point on an inclusion boundary belongs to the matrix (strict
// inequalities, Eq. S1), or to the inclusion when the problem is closed (Eq. S2), with
// periodic images; the dual side samples the pointwise inverse.
__global__ void k_sample_coef(SpecArgs a, double* coef) {
  const long long grid = (long long)a.M[0] * a.M[1] * a.M[2];
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < grid;
       j += (long long)gridDim.x * blockDim.x) {
    const int j1 = (int)(j % a.M[0]);
    const int j2 = (int)((j / a.M[0]) % a.M[1]);
    const int j3 = (int)(j / ((long long)a.M[0] * a.M[1]));
    const int js[3] = {j1, j2, j3};
    double x[3];
    for (int c = 0; c < 3; ++c) x[c] = (double)sfreq(js[c], a.M[c]) / ((double)a.M[c] * a.invY[c]);
    double v[6];
    for (int q = 0; q < 6; ++q) v[q] = a.A0p[q];
    if (a.bitmap) {   // the pixel holding the grid point
      long long idx = 0;
      for (int c = a.d - 1; c >= 0; --c) {
        int i = (int)floor((x[c] * a.invY[c] + 0.5) * a.P[c]);
        i = i < 0 ? 0 : (i >= a.P[c] ? a.P[c] - 1 : i);
        idx = idx * a.P[c] + i;
      }
      const double b = a.bitmap[idx];
      coef[j] = a.invert ? 1.0 / b : b;
      continue;
    }
    for (int i = 0; i < a.nincl; ++i) {
      const DevIncl& I = a.incl[i];
      bool in = true;
      double r2 = 0.0;
      for (int c = 0; c < a.d; ++c) {
        const double Yc = 1.0 / a.invY[c];
        double dx = x[c] - I.c[c];
        dx -= Yc * rint(dx * a.invY[c]);
        if (I.shape == 0) in = in && (a.closed ? fabs(dx) <= 0.5 * I.h[c] : fabs(dx) < 0.5 * I.h[c]);
        r2 += dx * dx;
      }
      if (I.shape != 0) in = a.closed ? sqrt(r2) <= I.h[0] : sqrt(r2) < I.h[0];
      if (in)
        for (int q = 0; q < a.ncomp; ++q) v[q] = a.A0p[q] + I.dA[q];
    }
    for (int q = 0; q < a.ncomp; ++q) coef[q * grid + j] = v[q];
  }
}

__global__ void k_bitmap_load(const double* bmp, double2* D, long long n, int invert) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    D[i] = make_double2(invert ? 1.0 / bmp[i] : bmp[i], 0.0);
}

// The image's local average of Sec. 7.3: weight 1/2 for the pixel and 1/4 for each of its
// two periodic neighbours along every axis, multiplied over the axes (in 2D: 4/16 the
// pixel, 2/16 the edge neighbours, 1/16 the corners; 3D images take the same per-axis
// weights). One output pixel per thread, summed in FP64.
__global__ void k_bitmap_smooth(const double* __restrict__ raw, double* __restrict__ out, int d, int P0, int P1,
                                int P2) {
  const long long n = (long long)P0 * P1 * P2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int i0 = (int)(e % P0);
    const int i1 = (int)((e / P0) % P1);
    const int i2 = (int)(e / ((long long)P0 * P1));
    const int r2 = d == 3 ? 1 : 0;
    double acc = 0.0;
    for (int o2 = -r2; o2 <= r2; ++o2) {
      const int j2 = (i2 + o2 + P2) % P2;
      const double w2 = d == 3 ? (o2 == 0 ? 0.5 : 0.25) : 1.0;
      for (int o1 = -1; o1 <= 1; ++o1) {
        const int j1 = (i1 + o1 + P1) % P1;
        const double w1 = o1 == 0 ? 0.5 : 0.25;
        const double* row = raw + ((long long)j2 * P1 + j1) * P0;
        const double s = 0.25 * row[(i0 + P0 - 1) % P0] + 0.5 * row[i0] + 0.25 * row[(i0 + 1) % P0];
        acc += (w2 * w1) * s;
      }
    }
    out[e] = acc;
  }
}

__global__ void k_rotate3(const double2* in, double2* out, int P0, int P1, int P2) {
  const long long n = (long long)P0 * P1 * P2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(i % P0);
    const int b = (int)((i / P0) % P1);
    const int c = (int)(i / ((long long)P0 * P1));
    out[((long long)a * P2 + c) * P1 + b] = in[i];
  }
}

// A_hat(n) = prod_a [(1/P_a) sinc(n_a/P_a) exp(i pi n_a (1 - 1/P_a))] D(n mod P): the pixel
// boxes of side Y_a/P_a centred at -Y_a/2 + (i_a + 1/2) Y_a/P_a (Remark "inclusion")
__global__ void k_bitmap_spectrum(SpecArgs a, const double2* D, double2* S) {
  const long long n = (long long)a.len[0] * a.len[1] * a.len[2];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int i0 = (int)(e % a.len[0]);
    const int i1 = (int)((e / a.len[0]) % a.len[1]);
    const int i2 = (int)(e / ((long long)a.len[0] * a.len[1]));
    const int ns[3] = {i0, sfreq(i1, a.Nmod[1]), sfreq(i2, a.Nmod[2])};
    double re = 1.0, im = 0.0;
    long long idx = 0;
    for (int c = a.d - 1; c >= 0; --c) {
      const int P = a.P[c];
      int m = ns[c] % P;
      if (m < 0) m += P;
      idx = idx * P + m;
    }
    for (int c = 0; c < a.d; ++c) {
      const int P = a.P[c];
      const int nn = ns[c];
      // sinc(n/P) and the phase pi n (P - 1)/P, arguments reduced to [0, 2) exactly
      int r = nn % (2 * P);
      if (r < 0) r += 2 * P;
      const double sn = nn == 0 ? 1.0 : sinpi((double)r / P) / (M_PI * (double)nn / P);
      long long q = ((long long)nn * (P - 1)) % (2LL * P);
      if (q < 0) q += 2LL * P;
      double ps, pc;
      sincospi((double)q / P, &ps, &pc);
      const double f = sn / P;
      const double nre = (re * pc - im * ps) * f, nim = (re * ps + im * pc) * f;
      re = nre;
      im = nim;
    }
    const double2 dv = D[idx];
    S[e] = make_double2(re * dv.x - im * dv.y, re * dv.y + im * dv.x);
  }
}

// Half spectrum on Z_M (layout of k_spectrum) of the N-periodic extension of a DFT D of
// N-grid samples ([N2][N1][N0], x fastest): S(n) = scale * D(n mod N).
__global__ void k_periodic_spectrum(SpecArgs a, const double2* D, double2* S, int N0, int N1, int N2, double scale) {
  const long long n = (long long)a.len[0] * a.len[1] * a.len[2];
  const int Nn[3] = {N0, N1, N2};
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int i0 = (int)(e % a.len[0]);
    const int i1 = (int)((e / a.len[0]) % a.len[1]);
    const int i2 = (int)(e / ((long long)a.len[0] * a.len[1]));
    const int ns[3] = {i0, sfreq(i1, a.Nmod[1]), sfreq(i2, a.Nmod[2])};
    long long idx = 0;
    for (int c = a.d - 1; c >= 0; --c) {
      int m = ns[c] % Nn[c];
      if (m < 0) m += Nn[c];
      idx = idx * Nn[c] + m;
    }
    const double2 dv = D[idx];
    S[e] = make_double2(scale * dv.x, scale * dv.y);
  }
}

// Rayleigh-Ritz on span{x}: per right-hand side the partial sums of x.b and x.q (q = C x),
// Hermitian weights, rows [rhs][2][nblk]
template <typename T>
__global__ void __launch_bounds__(kThreads) k_rr_dots(const cpx<T>* x, const cpx<T>* b, const cpx<T>* q, int C,
                                                      long long field, FastDiv fdNh, double* part, int ld) {
  __shared__ double red[32];
  const int rhs = blockIdx.y;
  const long long n = (long long)C * field;
  const long long base = (long long)rhs * n;
  double xb = 0.0, xq = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int ei = (int)e;
    const double w = ei - fdNh.div(ei) * (int)fdNh.d == 0 ? 1.0 : 2.0;
    const cpx<T> xv = x[base + e], bv = b[base + e], qv = q[base + e];
    xb += w * ((double)xv.x * bv.x + (double)xv.y * bv.y);
    xq += w * ((double)xv.x * qv.x + (double)xv.y * qv.y);
  }
  const double s1 = block_sum(xb, red);
  if (threadIdx.x == 0) part[(rhs * 2) * ld + blockIdx.x] = s1;
  const double s2 = block_sum(xq, red);
  if (threadIdx.x == 0) part[(rhs * 2 + 1) * ld + blockIdx.x] = s2;
}

// s = (x.b)/(x.Cx) (0 when x.Cx <= 0): x = s x, r = b - s q, |r|^2 partials
template <typename T>
__global__ void __launch_bounds__(kThreads) k_rr_apply(cpx<T>* x, cpx<T>* r, const cpx<T>* b, const cpx<T>* q, int C,
                                                       long long field, FastDiv fdNh, const double* rrpart, int nblk,
                                                       double* partial, int ld) {
  __shared__ double red[32];
  __shared__ double s_s;
  const int rhs = blockIdx.y;
  double a = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
    a += rrpart[(rhs * 2) * ld + i];
    c += rrpart[(rhs * 2 + 1) * ld + i];
  }
  const double num = block_sum(a, red);
  const double den = block_sum(c, red);
  if (threadIdx.x == 0) {
    const double sc = den > 0.0 ? num / den : 0.0;
    s_s = isfinite(sc) ? sc : 0.0;
  }
  __syncthreads();
  const T sr = T(s_s);
  const long long n = (long long)C * field;
  const long long base = (long long)rhs * n;
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const cpx<T> xv = x[base + e], bv = b[base + e], qv = q[base + e];
    x[base + e] = mk<T>(sr * xv.x, sr * xv.y);
    const cpx<T> rv = mk<T>(fma(-sr, qv.x, bv.x), fma(-sr, qv.y, bv.y));
    r[base + e] = rv;
    const int ei = (int)e;
    const double w = ei - fdNh.div(ei) * (int)fdNh.d == 0 ? 1.0 : 2.0;
    acc += w * ((double)rv.x * rv.x + (double)rv.y * rv.y);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partial[rhs * ld + blockIdx.x] = s;
}

// r = -r over nrhs fields of C components, with the Hermitian-weighted |r|^2 partials
template <typename T>
__global__ void __launch_bounds__(kThreads) k_negate_norm(cpx<T>* r, int C, long long field, FastDiv fdNh,
                                                          double* partial, int ld) {
  __shared__ double red[32];
  const int rhs = blockIdx.y;
  const long long n = (long long)C * field;
  const long long base = (long long)rhs * n;
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    cpx<T> v = r[base + e];
    v = mk<T>(-v.x, -v.y);
    r[base + e] = v;
    const int ei = (int)e;
    const double w = ei - fdNh.div(ei) * (int)fdNh.d == 0 ? 1.0 : 2.0;
    acc += w * ((double)v.x * v.x + (double)v.y * v.y);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partial[rhs * ld + blockIdx.x] = s;
}

// In place over nrhs FP64 fields of d components: u_b = sum_a c[b][a] (e_a + x_a), the
// constant e_a sitting at k = 0 of component a (the superposition of Eq.
// FD_superposition_odd_A).
__global__ void k_combine_fields(double2* x, int nrhs, int d, long long field, Coef3 c) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < d * field;
       t += (long long)gridDim.x * blockDim.x) {
    const int comp = (int)(t / field);
    const long long e = t - comp * field;
    double2 v[3], o[3];
    for (int a = 0; a < nrhs; ++a) v[a] = x[((long long)a * d + comp) * field + e];
    for (int b = 0; b < nrhs; ++b) {
      o[b] = make_double2(e == 0 ? c.v[3 * b + comp] : 0.0, 0.0);
      for (int a = 0; a < nrhs; ++a) {
        o[b].x = fma(c.v[3 * b + a], v[a].x, o[b].x);
        o[b].y = fma(c.v[3 * b + a], v[a].y, o[b].y);
      }
    }
    for (int b = 0; b < nrhs; ++b) x[((long long)b * d + comp) * field + e] = o[b];
  }
}

template <typename T>
__global__ void k_project_promote(const cpx<T>* x, double2* x64, int nrhs, int d, int Ny, int Nz,
                                  int Nh, double iy0, double iy1, double iy2, int side, FastDiv fdNh, FastDiv fdNy) {
  // one right-hand side per grid row (blockIdx.y); 32-bit index decoding (field < 2^31, checked
  // by the launcher) and one FP64 reciprocal a frequency: FP64 division and 64-bit integer
  // division are many instructions on this GPU
  const int field = Nh * Ny * Nz;
  const double invY[3] = {iy0, iy1, iy2};
  const int r = blockIdx.y;
  for (long long el = blockIdx.x * (long long)blockDim.x + threadIdx.x; el < field;
       el += (long long)gridDim.x * blockDim.x) {
    const int e = (int)el;
    const int q1 = fdNh.div(e);
    const int kx = e - q1 * Nh;
    const int iz = fdNy.div(q1);
    const int iy = q1 - iz * Ny;
    const int ks[3] = {kx, sfreq(iy, Ny), d == 3 ? sfreq(iz, Nz) : 0};
    double2 u[3];
    double xi[3], n2 = 0.0;
    double2 dot = make_double2(0.0, 0.0);
    for (int c = 0; c < d; ++c) {
      const cpx<T> v = x[((long long)r * d + c) * field + e];
      u[c] = make_double2((double)v.x, (double)v.y);
      xi[c] = ks[c] * invY[c];
      n2 += xi[c] * xi[c];
      dot.x += xi[c] * u[c].x;
      dot.y += xi[c] * u[c].y;
    }
    const bool nyq = nyquist(ks[1], Ny) || (d == 3 && nyquist(ks[2], Nz));
    const double inv = n2 > 0.0 ? 1.0 / n2 : 0.0;
    const double2 dn = make_double2(dot.x * inv, dot.y * inv);
    for (int c = 0; c < d; ++c) {
      double2 g = make_double2(0.0, 0.0);
      if (n2 > 0.0 && !nyq) {
        const double2 ge = make_double2(xi[c] * dn.x, xi[c] * dn.y);
        g = side == 0 ? ge : make_double2(u[c].x - ge.x, u[c].y - ge.y);
      }
      x64[((long long)r * d + c) * field + e] = g;
    }
  }
}

__global__ void k_energy_reduce(const double* partial, int nblk, int nrr, double* out) {
  __shared__ double red[32];
  for (int i = 0; i < nrr; ++i) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[(long long)b * nrr + i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[i] = s;
    __syncthreads();
  }
}

// The bound energies from the last FP64 residual of the mixed solve (Def. upper_lower_bounds
// expanded in Fourier space): for x_b in the range of Gamma with residual r_b = b_b - C x_b
// and b_a = -Gamma A_hat E_a,
//   a(E_b + x_b, E_a + x_a) = E_a . <A> E_b - <b_a, x_b> - <x_a, r_b>,
// <A> = A_hat(0) the cell mean of the coefficient and <u, v> the Parseval inner product of the
// stored half spectra (weight 1 at kx = 0, else 2). Per block: the R^2 sums <b_a, x_b> and the
// R^2 sums <x_a, r_b>, over all components and frequencies, [blk][2 R^2].
__global__ void __launch_bounds__(kThreads) k_energy_identity_part(const double2* b, const double2* x, const double2* r,
                                                                   int R, int C, long long field, FastDiv fdNh,
                                                                   double* part) {
  __shared__ double red[32];
  double acc[18];
#pragma unroll
  for (int i = 0; i < 18; ++i) acc[i] = 0.0;
  const long long n = (long long)C * field;   // entries of one right-hand side
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e % field);
    const double w = k - fdNh.div(k) * (int)fdNh.d == 0 ? 1.0 : 2.0;
    double2 bv[3], xv[3], rv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (a < R) {
        bv[a] = b[(long long)a * n + e];
        xv[a] = x[(long long)a * n + e];
        rv[a] = r[(long long)a * n + e];
      }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (a < R && c < R) {
          acc[a * 3 + c] += w * (bv[a].x * xv[c].x + bv[a].y * xv[c].y);
          acc[9 + a * 3 + c] += w * (xv[a].x * rv[c].x + xv[a].y * rv[c].y);
        }
  }
  for (int a = 0; a < R; ++a)
    for (int c = 0; c < R; ++c)
      for (int h = 0; h < 2; ++h) {
        const double s = block_sum(acc[h * 9 + a * 3 + c], red);
        if (threadIdx.x == 0) part[(long long)blockIdx.x * 2 * R * R + h * R * R + a * R + c] = s;
      }
}

// per block: the sum of each of the ncomp coefficient components over the double grid
__global__ void __launch_bounds__(kThreads) k_coef_sum_part(const double* coef, int ncomp, long long grid,
                                                            double* part) {
  __shared__ double red[32];
  for (int q = 0; q < ncomp; ++q) {
    double acc = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < grid;
         e += (long long)gridDim.x * blockDim.x)
      acc += coef[(long long)q * grid + e];
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) part[(long long)blockIdx.x * ncomp + q] = s;
  }
}

// out[a R + c] = |M| (E_a . <A> E_c - <b_a, x_c> - <x_a, r_c>): the energy-pass convention
// (grid sums, later scaled by 1/|M|)
__global__ void k_energy_identity_finish(const double* part, int nblk, const double* cpart, int cblk, int R, int d,
                                         int ncomp, double gridsize, double* out) {
  __shared__ double red[32];
  __shared__ double mean[6];
  for (int q = 0; q < ncomp; ++q) {
    double s = 0.0;
    for (int b = threadIdx.x; b < cblk; b += blockDim.x) s += cpart[(long long)b * ncomp + q];
    s = block_sum(s, red);
    if (threadIdx.x == 0) mean[q] = s;   // the grid sum of component q
    __syncthreads();
  }
  for (int i = 0; i < 2 * R * R; ++i) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[(long long)b * 2 * R * R + i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
      const int h = i / (R * R), ac = i - h * R * R, a = ac / R, c = ac - a * R;
      if (h == 0) {
        int q = 0;
        if (ncomp > 1) {
          if (a == c) q = a;
          else if (d == 2) q = 2;
          else q = (a + c == 3) ? 3 : ((a + c == 2) ? 4 : 5);
        }
        const double A = (ncomp == 1 && a != c) ? 0.0 : mean[q];
        out[ac] = A - gridsize * s;
      } else {
        out[ac] -= gridsize * s;
      }
    }
    __syncthreads();
  }
}

// x = c + b (x - a) elementwise (the dual coefficient of a one-material cell from the primal one)
__global__ void k_affine(double* x, long long n, double a, double b, double c) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = fma(b, x[i] - a, c);
}

__global__ void k_convert_d2f(const double* in, float* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// FP64 -> FP32 (out, may be null) and the nearest float-float (hi = the FP32 value,
// lo = fl32(x - hi)) in one pass
__global__ void k_convert_d2f_ff(const double* in, float* out, ffloat* off, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const ffloat v = ff_from(in[i]);
    if (out) out[i] = v.hi;
    off[i] = v;
  }
}

// ---------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------
cudaError_t launch_axis_tables(int nincl, int d, const int* M, int Mmax, const double* invY,
                               const DevIncl* incl, double2* phase, double* sinc, cudaStream_t s) {
  if (nincl == 0) return cudaSuccess;
  const long long total = (long long)nincl * 3 * Mmax;
  const int blocks = (int)((total + kThreads - 1) / kThreads);
  k_axis_tables<<<blocks, kThreads, 0, s>>>(nincl, d, M[0], M[1], M[2], Mmax, invY[0], invY[1],
                                            invY[2], incl, phase, sinc);
  return cudaGetLastError();
}

// A_hat on the half of Z_M, one (y, z) row of x frequencies at a time per CTA: the y and z
// factors of every inclusion's phase (and of a box's sinc) are formed once per row in shared
// memory, so that an x frequency needs one complex product per inclusion instead of d - 1.
// Same terms as ahat_eval, the phase product taken as p_x (p_y p_z).
constexpr int kSpecRowIncl = 128;
constexpr int kSpecRowThreads = 128;
__global__ void __launch_bounds__(kSpecRowThreads) k_spectrum_rows(SpecArgs a, double2* out) {
  __shared__ double2 qyz[kSpecRowIncl];
  __shared__ double syz[kSpecRowIncl];
  const long long total = (long long)a.len[0] * a.len[1] * a.len[2];
  const int nrows = a.len[1] * a.len[2];
  for (int row = blockIdx.x; row < nrows; row += gridDim.x) {
    const int iy = row % a.len[1], iz = row / a.len[1];
    const int nsy = sfreq(iy, a.Nmod[1]), nsz = a.d == 3 ? sfreq(iz, a.Nmod[2]) : 0;
    const int niy = nsy < 0 ? nsy + a.M[1] : nsy, niz = nsz < 0 ? nsz + a.M[2] : nsz;
    __syncthreads();   // the previous row's factors are no longer read
    for (int j = threadIdx.x; j < a.nincl; j += blockDim.x) {
      double2 q = a.phase[((long long)j * 3 + 1) * a.Mmax + niy];
      double sy = a.sinc[((long long)j * 3 + 1) * a.Mmax + niy];
      if (a.d == 3) {
        const double2 t = a.phase[((long long)j * 3 + 2) * a.Mmax + niz];
        q = make_double2(q.x * t.x - q.y * t.y, q.x * t.y + q.y * t.x);
        sy *= a.sinc[((long long)j * 3 + 2) * a.Mmax + niz];
      }
      qyz[j] = q;
      syz[j] = sy * a.invVol;
    }
    __syncthreads();
    const double yz2 = (nsy * a.invY[1]) * (nsy * a.invY[1]) + (nsz * a.invY[2]) * (nsz * a.invY[2]);
    for (int ix = threadIdx.x; ix < a.len[0]; ix += blockDim.x) {
      double2 v[6];
      for (int q = 0; q < a.ncomp; ++q) v[q] = make_double2(0.0, 0.0);
      if (ix == 0 && nsy == 0 && nsz == 0)
        for (int q = 0; q < a.ncomp; ++q) v[q].x = a.A0p[q];
      double rad = 0.0;
      int grp = -1;
      const int n2 = ix * ix + nsy * nsy + nsz * nsz;
      for (int j = 0; j < a.nincl; ++j) {
        const DevIncl& I = a.incl[j];
        double f;
        if (I.shape == 0) {
          f = syz[j] * a.sinc[((long long)j * 3) * a.Mmax + ix];
        } else {
          if (!I.same_as_prev) {
            ++grp;
            if (a.radtab) {
              rad = a.radtab[(long long)grp * a.radlen + n2];
            } else {
              const double xi = ix * a.invY[0];
              rad = radial_factor(a.d, I.h[0], sqrt(xi * xi + yz2));
            }
          }
          f = rad * a.invVol;
        }
        const double2 px = a.phase[((long long)j * 3) * a.Mmax + ix];
        const double2 q = qyz[j];
        const double2 ph = make_double2(px.x * q.x - px.y * q.y, px.x * q.y + px.y * q.x);
        for (int c = 0; c < a.ncomp; ++c) {
          const double sc = f * I.dA[c];
          v[c].x = fma(sc, ph.x, v[c].x);
          v[c].y = fma(sc, ph.y, v[c].y);
        }
      }
      const long long e = (long long)row * a.len[0] + ix;
      for (int c = 0; c < a.ncomp; ++c) out[c * total + e] = v[c];
    }
  }
}

// The closed-form coefficient spectrum of k_spectrum_rows in float-float arithmetic (pairs of
// FP32 on the FP32 pipes, about 48 bits; the mixed-precision path, whose operator and
// residuals run in FP32 and float-float): the same terms in the same order, from float-float
// copies of the phase, sinc and radial tables (k_tables_ff); the spectrum is written in FP64.
__global__ void k_tables_ff(const double2* phase, const double* sinc, long long nps, const double* radtab,
                            long long nrad, ffloat2* phase_ff, ffloat* sinc_ff, ffloat* rad_ff) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nps + nrad;
       i += (long long)gridDim.x * blockDim.x) {
    if (i < nps) {
      phase_ff[i] = ff2_from(phase[i]);
      sinc_ff[i] = ff_from(sinc[i]);
    } else {
      rad_ff[i - nps] = ff_from(radtab[i - nps]);
    }
  }
}

__device__ __forceinline__ ffloat2 ff_cmul(ffloat2 a, ffloat2 b) {
  ffloat2 r;
  r.x = fma(a.x, b.x, -(a.y * b.y));
  r.y = fma(a.x, b.y, a.y * b.x);
  return r;
}

__global__ void __launch_bounds__(kSpecRowThreads) k_spectrum_rows_ff(SpecArgs a, const ffloat2* phase,
                                                                     const ffloat* sinc, const ffloat* radtab,
                                                                     double2* out) {
  __shared__ ffloat2 qyz[kSpecRowIncl];
  __shared__ ffloat syz[kSpecRowIncl];
  __shared__ ffloat sdA[kSpecRowIncl][6];
  const long long total = (long long)a.len[0] * a.len[1] * a.len[2];
  const int nrows = a.len[1] * a.len[2];
  const ffloat invVol(a.invVol);
  for (int j = threadIdx.x; j < a.nincl; j += blockDim.x)
    for (int c = 0; c < a.ncomp; ++c) sdA[j][c] = ffloat(a.incl[j].dA[c]);
  for (int row = blockIdx.x; row < nrows; row += gridDim.x) {
    const int iy = row % a.len[1], iz = row / a.len[1];
    const int nsy = sfreq(iy, a.Nmod[1]), nsz = a.d == 3 ? sfreq(iz, a.Nmod[2]) : 0;
    const int niy = nsy < 0 ? nsy + a.M[1] : nsy, niz = nsz < 0 ? nsz + a.M[2] : nsz;
    __syncthreads();   // the previous row's factors are no longer read (and sdA is written)
    for (int j = threadIdx.x; j < a.nincl; j += blockDim.x) {
      ffloat2 q = phase[((long long)j * 3 + 1) * a.Mmax + niy];
      ffloat sy = sinc[((long long)j * 3 + 1) * a.Mmax + niy];
      if (a.d == 3) {
        q = ff_cmul(q, phase[((long long)j * 3 + 2) * a.Mmax + niz]);
        sy = sy * sinc[((long long)j * 3 + 2) * a.Mmax + niz];
      }
      qyz[j] = q;
      syz[j] = sy * invVol;
    }
    __syncthreads();
    for (int ix = threadIdx.x; ix < a.len[0]; ix += blockDim.x) {
      ffloat2 v[6];
      for (int q = 0; q < a.ncomp; ++q) v[q] = ffloat2{ffloat(0.f, 0.f), ffloat(0.f, 0.f)};
      if (ix == 0 && nsy == 0 && nsz == 0)
        for (int q = 0; q < a.ncomp; ++q) v[q].x = ffloat(a.A0p[q]);
      ffloat rad(0.f, 0.f);
      int grp = -1;
      const int n2 = ix * ix + nsy * nsy + nsz * nsz;
      for (int j = 0; j < a.nincl; ++j) {
        const DevIncl& I = a.incl[j];
        ffloat f;
        if (I.shape == 0) {
          f = syz[j] * sinc[((long long)j * 3) * a.Mmax + ix];
        } else {
          if (!I.same_as_prev) {
            ++grp;
            rad = radtab[(long long)grp * a.radlen + n2];
          }
          f = rad * invVol;
        }
        const ffloat2 ph = ff_cmul(phase[((long long)j * 3) * a.Mmax + ix], qyz[j]);
        for (int c = 0; c < a.ncomp; ++c) {
          const ffloat sc = f * sdA[j][c];
          v[c].x = fma(sc, ph.x, v[c].x);
          v[c].y = fma(sc, ph.y, v[c].y);
        }
      }
      const long long e = (long long)row * a.len[0] + ix;
      for (int c = 0; c < a.ncomp; ++c) out[c * total + e] = ff2_to(v[c]);
    }
  }
}

// One entry per (ball group, integer |k|^2): the group's radial factor at |xi| = sqrt(n) / Y
__global__ void k_radial_table(SpecArgs a, double* tab, int groups) {
  const long long total = (long long)groups * a.radlen;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(e / a.radlen);
    const int n = (int)(e - (long long)g * a.radlen);
    int grp = -1, j = 0;
    for (; j < a.nincl; ++j)
      if (a.incl[j].shape != 0 && !a.incl[j].same_as_prev && ++grp == g) break;
    tab[e] = j < a.nincl ? radial_factor(a.d, a.incl[j].h[0], sqrt((double)n) * a.invY[0]) : 0.0;
  }
}

cudaError_t launch_radial_table(const SpecArgs& a, double* radtab, int groups, cudaStream_t s) {
  if (groups < 1 || a.radlen < 1) return cudaSuccess;
  const long long total = (long long)groups * a.radlen;
  const int blocks = (int)std::min<long long>((total + kThreads - 1) / kThreads, 152 * 16);
  k_radial_table<<<blocks, kThreads, 0, s>>>(a, radtab, groups);
  return cudaGetLastError();
}

cudaError_t launch_spectrum_ff(const SpecArgs& a, long long nrad, ffloat2* phase_ff, ffloat* sinc_ff, ffloat* rad_ff,
                              double2* out, cudaStream_t s) {
  if (a.nincl > kSpecRowIncl || a.ncomp > 6) return cudaErrorInvalidValue;
  const long long nps = (long long)a.nincl * 3 * a.Mmax;
  if (nps + nrad > 0) {
    long long blocks = (nps + nrad + kThreads - 1) / kThreads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_tables_ff<<<(int)blocks, kThreads, 0, s>>>(a.phase, a.sinc, nps, a.radtab, nrad, phase_ff, sinc_ff, rad_ff);
  }
  const int nrows = a.len[1] * a.len[2];
  const int blocks = nrows < 152 * 16 ? nrows : 152 * 16;
  k_spectrum_rows_ff<<<blocks, kSpecRowThreads, 0, s>>>(a, phase_ff, sinc_ff, rad_ff, out);
  return cudaGetLastError();
}

cudaError_t launch_spectrum(const SpecArgs& a, double2* out, cudaStream_t s) {
  if (a.nincl <= kSpecRowIncl) {
    const int nrows = a.len[1] * a.len[2];
    const int blocks = nrows < 152 * 16 ? nrows : 152 * 16;
    k_spectrum_rows<<<blocks, kSpecRowThreads, 0, s>>>(a, out);
    return cudaGetLastError();
  }
  const long long total = (long long)a.len[0] * a.len[1] * a.len[2];
  long long blocks = (total + kThreads - 1) / kThreads;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_spectrum<<<(int)blocks, kThreads, 0, s>>>(a, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rhs(const SpecArgs& a, int side, int nrhs, int Nh, const int* N, void* b,
                       double* partial, int nblk, cudaStream_t s, const double2* hat) {
  if (nrhs < 1 || nrhs > 3) return cudaErrorInvalidValue;
  if ((long long)Nh * N[1] * N[2] >= (1LL << 31)) return cudaErrorInvalidValue;
  k_rhs<T><<<nblk, kThreads, 0, s>>>(a, side, nrhs, Nh, N[1], N[2], reinterpret_cast<cpx<T>*>(b), partial,
                                     nblk, hat);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_update(void* x, void* r, const void* p, const void* q, int nrhs, int C,
                             long long field, int Nh, CgScalars* cg, double* partial, int nblk,
                             const double* pq_part, int pq_ld, int pq_nblk, cudaStream_t s) {
  if ((long long)C * field >= (1LL << 31)) return cudaErrorInvalidValue;
  dim3 grid(nblk, nrhs);
  k_cg_update<T><<<grid, kThreads, 0, s>>>(
      reinterpret_cast<cpx<T>*>(x), reinterpret_cast<cpx<T>*>(r), reinterpret_cast<const cpx<T>*>(p),
      reinterpret_cast<const cpx<T>*>(q), C, field, FastDiv((uint32_t)Nh), cg, partial, nblk, pq_part, pq_ld,
      pq_nblk);
  return cudaGetLastError();
}

cudaError_t launch_cg_init(CgScalars* cg, const double* partial, int ld, int nblk, int nrhs,
                           double tol2_abs, double rel2, int guard, cudaStream_t s, double tol2_hi, double drift) {
  k_cg_init<<<1, kThreads, 0, s>>>(cg, partial, ld, nblk, nrhs, tol2_abs, rel2, guard, tol2_hi, drift);
  return cudaGetLastError();
}
cudaError_t launch_outer_check(CgScalars* cg, const double* partial, int ld, int nblk, int nrhs,
                               double shrink2, cudaStream_t s) {
  k_outer_check<<<1, kThreads, 0, s>>>(cg, partial, ld, nblk, nrhs, shrink2);
  return cudaGetLastError();
}
cudaError_t launch_demote(const double2* r64, float2* r32, int nrhs, int C, long long field, int Nh,
                          const CgScalars* outer, double* partial, int nblk, cudaStream_t s) {
  if ((long long)C * field >= (1LL << 31)) return cudaErrorInvalidValue;
  dim3 grid(nblk, nrhs);
  k_demote<<<grid, kThreads, 0, s>>>(r64, r32, C, field, FastDiv((uint32_t)Nh), outer, partial, nblk);
  return cudaGetLastError();
}
cudaError_t launch_promote_add(const float2* x32, double2* x64, long long n, cudaStream_t s) {
  long long blocks = (n + kThreads - 1) / kThreads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_promote_add<<<(int)blocks, kThreads, 0, s>>>(x32, x64, n);
  return cudaGetLastError();
}
cudaError_t launch_cg_beta(CgScalars* cg, const double* partial, int ld, int nblk, int nrhs,
                           cudaStream_t s) {
  k_cg_beta<<<1, kThreads, 0, s>>>(cg, partial, ld, nblk, nrhs);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_project_promote(const void* x, double2* x64, int nrhs, int d, int Ny, int Nz,
                                   int Nh, const double* invY, int side, cudaStream_t s) {
  const long long field = (long long)Nh * Ny * Nz;
  if (field >= (1LL << 31) || nrhs < 1) return cudaErrorInvalidValue;
  long long blocks = (field + kThreads - 1) / kThreads;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_project_promote<T><<<dim3((unsigned)blocks, (unsigned)nrhs), kThreads, 0, s>>>(
      reinterpret_cast<const cpx<T>*>(x), x64, nrhs, d, Ny, Nz, Nh, invY[0], invY[1], invY[2], side,
      FastDiv((uint32_t)Nh), FastDiv((uint32_t)Ny));
  return cudaGetLastError();
}

// Half-spectrum fields of one grid on another: out(k) = in(k) where the source grid holds
// frequency k (Nyquist rows of even grids excluded), 0 elsewhere. Fourier coefficients of a
// trigonometric polynomial do not depend on the grid (Eq. DFT with 1/|N|), so this is the
// exact prolongation of a coarse field (E_N and J_N are nested for odd grids) and the
// truncation P_N of a fine one. One thread per output element.
template <typename T>
__global__ void k_resample(const cpx<T>* in, cpx<T>* out, long long count, int d, int fx, int fy, int fz, int tx,
                           int ty, int tz) {
  const int tnh = (tx + 1) / 2, fnh = (fx + 1) / 2;
  const long long tfield = (long long)tnh * ty * tz, ffield = (long long)fnh * fy * fz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count * tfield;
       t += (long long)gridDim.x * blockDim.x) {
    const long long f = t / tfield;
    const long long e = t - f * tfield;
    const int kx = (int)(e % tnh);
    const int iy = (int)((e / tnh) % ty);
    const int iz = (int)(e / ((long long)tnh * ty));
    const int ky = sfreq(iy, ty), kz = d == 3 ? sfreq(iz, tz) : 0;
    // the source holds k when |k| fits its reduced set (Nyquist rows excluded)
    auto holds = [](int k, int n) { return k >= -((n - 1) / 2) && k <= (n - 1) / 2; };
    const bool ok = kx < fnh && holds(ky, fy) && (d != 3 || holds(kz, fz)) && !nyquist(ky, ty) &&
                    !(d == 3 && nyquist(kz, tz));
    cpx<T> v = mk<T>(T(0), T(0));
    if (ok) {
      const int sy = ky < 0 ? ky + fy : ky, sz = kz < 0 ? kz + fz : kz;
      v = in[f * ffield + ((long long)sz * fy + sy) * fnh + kx];
    }
    out[t] = v;
  }
}

template <typename T>
cudaError_t launch_resample(const void* in, void* out, long long count, int d, const int* from, const int* to,
                            cudaStream_t s) {
  const long long total = count * ((to[0] + 1) / 2) * (long long)to[1] * (d == 3 ? to[2] : 1);
  long long blocks = (total + kThreads - 1) / kThreads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  k_resample<T><<<(int)blocks, kThreads, 0, s>>>(reinterpret_cast<const cpx<T>*>(in), reinterpret_cast<cpx<T>*>(out),
                                                 count, d, from[0], from[1], d == 3 ? from[2] : 1, to[0], to[1],
                                                 d == 3 ? to[2] : 1);
  return cudaGetLastError();
}
template cudaError_t launch_resample<double>(const void*, void*, long long, int, const int*, const int*, cudaStream_t);
template cudaError_t launch_resample<float>(const void*, void*, long long, int, const int*, const int*, cudaStream_t);

cudaError_t launch_combine_fields(double2* x, int nrhs, int d, long long field, const double* c,
                                  cudaStream_t s) {
  if (nrhs < 1 || nrhs > 3 || d < 1 || d > 3) return cudaErrorInvalidValue;
  Coef3 cc;
  for (int i = 0; i < 9; ++i) cc.v[i] = c[i];
  long long blocks = (d * field + kThreads - 1) / kThreads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_combine_fields<<<(int)blocks, kThreads, 0, s>>>(x, nrhs, d, field, cc);
  return cudaGetLastError();
}

cudaError_t launch_sample_coef(const SpecArgs& a, double* coef, cudaStream_t s) {
  const long long grid = (long long)a.M[0] * a.M[1] * a.M[2];
  long long blocks = (grid + kThreads - 1) / kThreads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_sample_coef<<<(int)blocks, kThreads, 0, s>>>(a, coef);
  return cudaGetLastError();
}

static int grid_blocks(long long n) {
  long long blocks = (n + kThreads - 1) / kThreads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  return (int)(blocks < 1 ? 1 : blocks);
}
cudaError_t launch_bitmap_load(const double* bmp, double2* D, long long n, int invert, cudaStream_t s) {
  k_bitmap_load<<<grid_blocks(n), kThreads, 0, s>>>(bmp, D, n, invert);
  return cudaGetLastError();
}
cudaError_t launch_bitmap_smooth(const double* raw, double* out, int d, const int P[3], cudaStream_t s) {
  const long long n = (long long)P[0] * P[1] * P[2];
  k_bitmap_smooth<<<grid_blocks(n), kThreads, 0, s>>>(raw, out, d, P[0], P[1], P[2]);
  return cudaGetLastError();
}
cudaError_t launch_rotate3(const double2* in, double2* out, int P0, int P1, int P2, cudaStream_t s) {
  k_rotate3<<<grid_blocks((long long)P0 * P1 * P2), kThreads, 0, s>>>(in, out, P0, P1, P2);
  return cudaGetLastError();
}
cudaError_t launch_periodic_spectrum(const SpecArgs& a, const double2* D, double2* S, const int* N, double scale,
                                     cudaStream_t s) {
  const long long n = (long long)a.len[0] * a.len[1] * a.len[2];
  k_periodic_spectrum<<<grid_blocks(n), kThreads, 0, s>>>(a, D, S, N[0], N[1], N[2], scale);
  return cudaGetLastError();
}

cudaError_t launch_bitmap_spectrum(const SpecArgs& a, const double2* D, double2* S, cudaStream_t s) {
  k_bitmap_spectrum<<<grid_blocks((long long)a.len[0] * a.len[1] * a.len[2]), kThreads, 0, s>>>(a, D, S);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_negate_norm(void* r, int nrhs, int C, long long field, int Nh, double* partial, int nblk,
                               cudaStream_t s) {
  if ((long long)C * field >= (1LL << 31)) return cudaErrorInvalidValue;
  dim3 grid(nblk, nrhs);
  k_negate_norm<T><<<grid, kThreads, 0, s>>>(reinterpret_cast<cpx<T>*>(r), C, field, FastDiv((uint32_t)Nh), partial,
                                             nblk);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_rayleigh_ritz(void* x, void* r, const void* b, const void* q, int nrhs, int C, long long field,
                                 int Nh, double* rrpart, double* partial, int nblk, cudaStream_t s) {
  if ((long long)C * field >= (1LL << 31)) return cudaErrorInvalidValue;
  dim3 grid(nblk, nrhs);
  const FastDiv fd((uint32_t)Nh);
  k_rr_dots<T><<<grid, kThreads, 0, s>>>(reinterpret_cast<const cpx<T>*>(x), reinterpret_cast<const cpx<T>*>(b),
                                         reinterpret_cast<const cpx<T>*>(q), C, field, fd, rrpart, nblk);
  k_rr_apply<T><<<grid, kThreads, 0, s>>>(reinterpret_cast<cpx<T>*>(x), reinterpret_cast<cpx<T>*>(r),
                                          reinterpret_cast<const cpx<T>*>(b), reinterpret_cast<const cpx<T>*>(q), C,
                                          field, fd, rrpart, nblk, partial, nblk);
  return cudaGetLastError();
}
template cudaError_t launch_rayleigh_ritz<double>(void*, void*, const void*, const void*, int, int, long long, int,
                                                  double*, double*, int, cudaStream_t);
template cudaError_t launch_negate_norm<double>(void*, int, int, long long, int, double*, int, cudaStream_t);
template cudaError_t launch_negate_norm<float>(void*, int, int, long long, int, double*, int, cudaStream_t);

// Block Rayleigh-Ritz start over the R starting fields x_i of one side (their span V):
// G = V^T C V, H = V^T B with q_i = C x_i; each right-hand side gets the Galerkin solution in V,
// x_j <- sum_i c_ij x_i with G c_j = H e_j, and r_j = b_j - sum_i c_ij q_i (never a larger
// energy error than the per-right-hand-side Rayleigh-Ritz scaling or than x = 0). When G is
// not safely positive definite (dependent starts) the diagonal scaling c_jj = H_jj / G_jj is
// used instead.
__global__ void k_brr_solve(const double* part, int nblk, int R, double* coefs) {
  __shared__ double red[32];
  __shared__ double GH[18];
  for (int i = 0; i < 2 * R * R; ++i) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[(long long)b * 2 * R * R + i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) GH[i] = s;
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  // part holds <b_a, x_c> (H^T) then <x_a, q_c> (G)
  double G[9], H[9], L[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, c[9];
  for (int a = 0; a < R; ++a)
    for (int b = 0; b < R; ++b) {
      H[a * R + b] = GH[b * R + a];                                        // <x_a, b_b>
      G[a * R + b] = 0.5 * (GH[R * R + a * R + b] + GH[R * R + b * R + a]);   // symmetric part
    }
  bool ok = true;
  double tr = 0.0;
  for (int a = 0; a < R; ++a) tr += fabs(G[a * R + a]);
  for (int j = 0; j < R && ok; ++j) {   // Cholesky G = L L^T
    double dgl = G[j * R + j];
    for (int k = 0; k < j; ++k) dgl -= L[j * R + k] * L[j * R + k];
    if (!(dgl > 1e-12 * tr) || !isfinite(dgl)) {
      ok = false;
      break;
    }
    L[j * R + j] = sqrt(dgl);
    for (int i = j + 1; i < R; ++i) {
      double v = G[i * R + j];
      for (int k = 0; k < j; ++k) v -= L[i * R + k] * L[j * R + k];
      L[i * R + j] = v / L[j * R + j];
    }
  }
  for (int j = 0; j < R; ++j) {   // column j: G c = H e_j
    double y[3], cj[3];
    if (ok) {
      for (int i = 0; i < R; ++i) {
        double v = H[i * R + j];
        for (int k = 0; k < i; ++k) v -= L[i * R + k] * y[k];
        y[i] = v / L[i * R + i];
      }
      for (int i = R - 1; i >= 0; --i) {
        double v = y[i];
        for (int k = i + 1; k < R; ++k) v -= L[k * R + i] * cj[k];
        cj[i] = v / L[i * R + i];
      }
    } else {
      for (int i = 0; i < R; ++i) cj[i] = 0.0;
      const double gj = G[j * R + j];
      cj[j] = gj > 0.0 && isfinite(H[j * R + j] / gj) ? H[j * R + j] / gj : 0.0;
    }
    for (int i = 0; i < R; ++i) c[i * R + j] = isfinite(cj[i]) ? cj[i] : 0.0;
  }
  for (int i = 0; i < R * R; ++i) coefs[i] = c[i];
}

// x_j <- sum_i c_ij x_i, r_j <- b_j - sum_i c_ij q_i (in place: every right-hand side of one
// entry is read before any is written; r may alias b or q), |r_j|^2 partials [rhs][blk]
__global__ void __launch_bounds__(kThreads) k_brr_apply(double2* x, double2* r, const double2* b, const double2* q,
                                                        int R, long long n, FastDiv fdNh, long long field,
                                                        const double* coefs, double* partial, int ld) {
  __shared__ double red[32];
  double c[9];
  for (int i = 0; i < R * R; ++i) c[i] = coefs[i];
  double acc[3] = {0.0, 0.0, 0.0};
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e % field);
    const double w = k - fdNh.div(k) * (int)fdNh.d == 0 ? 1.0 : 2.0;
    double2 xv[3], qv[3], bv[3];
    for (int i = 0; i < R; ++i) {
      xv[i] = x[(long long)i * n + e];
      qv[i] = q[(long long)i * n + e];
      bv[i] = b[(long long)i * n + e];
    }
    for (int j = 0; j < R; ++j) {
      double2 xn = make_double2(0.0, 0.0), rn = bv[j];
      for (int i = 0; i < R; ++i) {
        const double cij = c[i * R + j];
        xn.x = fma(cij, xv[i].x, xn.x);
        xn.y = fma(cij, xv[i].y, xn.y);
        rn.x = fma(-cij, qv[i].x, rn.x);
        rn.y = fma(-cij, qv[i].y, rn.y);
      }
      x[(long long)j * n + e] = xn;
      r[(long long)j * n + e] = rn;
      acc[j] += w * (rn.x * rn.x + rn.y * rn.y);
    }
  }
  for (int j = 0; j < R; ++j) {
    const double s = block_sum(acc[j], red);
    if (threadIdx.x == 0) partial[(long long)j * ld + blockIdx.x] = s;
  }
}

cudaError_t launch_block_rayleigh_ritz(double2* x, double2* r, const double2* b, const double2* q, int R, int C,
                                       long long field, int Nh, double* part, double* coefs, double* partial,
                                       int nblk, cudaStream_t s) {
  if (R < 1 || R > 3 || (long long)C * field >= (1LL << 31)) return cudaErrorInvalidValue;
  const FastDiv fd((uint32_t)Nh);
  // <b_a, x_c> and <x_a, q_c> (the energy identity's pair sums with r = q)
  k_energy_identity_part<<<nblk, kThreads, 0, s>>>(b, x, q, R, C, field, fd, part);
  k_brr_solve<<<1, kThreads, 0, s>>>(part, nblk, R, coefs);
  k_brr_apply<<<nblk, kThreads, 0, s>>>(x, r, b, q, R, (long long)C * field, fd, field, coefs, partial, nblk);
  return cudaGetLastError();
}

cudaError_t launch_energy_reduce(const double* partial, int nblk, int nrr, double* out,
                                 cudaStream_t s) {
  k_energy_reduce<<<1, kThreads, 0, s>>>(partial, nblk, nrr, out);
  return cudaGetLastError();
}

cudaError_t launch_energy_identity(const double2* b, const double2* x, const double2* r, int R, int C,
                                   long long field, int Nh, const double* coef, int ncomp, long long grid,
                                   double* part, int nblk, double* cpart, int cblk, double* out, cudaStream_t s) {
  if (R < 1 || R > 3 || C > 3) return cudaErrorInvalidValue;
  k_energy_identity_part<<<nblk, kThreads, 0, s>>>(b, x, r, R, C, field, FastDiv((uint32_t)Nh), part);
  k_coef_sum_part<<<cblk, kThreads, 0, s>>>(coef, ncomp, grid, cpart);
  const int d = C;
  k_energy_identity_finish<<<1, kThreads, 0, s>>>(part, nblk, cpart, cblk, R, d, ncomp, (double)grid, out);
  return cudaGetLastError();
}

cudaError_t launch_affine(double* x, long long n, double a, double b, double c, cudaStream_t s) {
  long long blocks = (n + kThreads - 1) / kThreads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_affine<<<(int)blocks, kThreads, 0, s>>>(x, n, a, b, c);
  return cudaGetLastError();
}

cudaError_t launch_convert_d2f(const double* in, float* out, long long n, cudaStream_t s) {
  long long blocks = (n + kThreads - 1) / kThreads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_convert_d2f<<<(int)blocks, kThreads, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_convert_d2f_ff(const double* in, float* out, ffloat* off, long long n, cudaStream_t s) {
  long long blocks = (n + kThreads - 1) / kThreads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_convert_d2f_ff<<<(int)blocks, kThreads, 0, s>>>(in, out, off, n);
  return cudaGetLastError();
}

// explicit instantiations
#define HOMB_INST(T)                                                                             \
  template cudaError_t launch_rhs<T>(const SpecArgs&, int, int, int, const int*, void*, double*,  \
                                     int, cudaStream_t, const double2*);                         \
  template cudaError_t launch_cg_update<T>(void*, void*, const void*, const void*, int, int,     \
                                           long long, int, CgScalars*, double*, int,             \
                                           const double*, int, int, cudaStream_t);               \
  template cudaError_t launch_project_promote<T>(const void*, double2*, int, int, int, int, int, \
                                                 const double*, int, cudaStream_t);
HOMB_INST(double)
HOMB_INST(float)

}  // namespace homb
