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

#include "kernels.cuh"

namespace homb {

constexpr int kThreads = 256;
constexpr size_t kSmemBudget = 96 * 1024;
constexpr size_t kSmemMax = 220 * 1024;

template <typename T>
__device__ __forceinline__ void load_twiddles(cpx<T>* Ws, const void* W, int M) {
  const cpx<T>* w = reinterpret_cast<const cpx<T>*>(W);
  for (int t = threadIdx.x; t < M; t += blockDim.x) Ws[t] = w[t];
}

// ---------------------------------------------------------------------------------
// pencil pass along y or z (one component slab per CTA, XC contiguous positions)
// ---------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_pencil(PencilArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int M = a.plan.M;
  cpx<T>* Ws = reinterpret_cast<cpx<T>*>(smem);
  cpx<T>* A = Ws + M;
  cpx<T>* B = A + (size_t)a.XC * M;
  const int s = blockIdx.y;
  const int x0 = blockIdx.x * a.XC;
  const int rhs = s / a.slabs_per_rhs;
  if (a.cg != nullptr && !a.cg->active[rhs]) return;
  const int comp = (s / a.slabs_per_comp) % a.C;
  const int XC = min(a.XC, a.X - x0);
  load_twiddles<T>(Ws, a.W, M);
  const bool pad = a.dir > 0 && a.Pin != M;
  if (pad) {
    for (int t = threadIdx.x; t < XC * M; t += blockDim.x) A[t] = mk<T>(T(0), T(0));
    __syncthreads();
  }
  cpx<T>* pin = const_cast<cpx<T>*>(reinterpret_cast<const cpx<T>*>(a.in)) + (long long)s * a.in_slab;
  const T beta = a.prologue == 1 ? T(a.cg->beta[rhs]) : T(0);
  for (int t = threadIdx.x; t < a.Pin * XC; t += blockDim.x) {
    const int p = t / XC;
    const int xx = t - p * XC;
    const long long gi = (long long)p * a.X + x0 + xx;
    cpx<T> v = pin[gi];
    if (a.prologue == 1) {
      const cpx<T> r = reinterpret_cast<const cpx<T>*>(a.aux)[(long long)s * a.in_slab + gi];
      v = mk<T>(fma(beta, v.x, r.x), fma(beta, v.y, r.y));
      pin[gi] = v;
    } else if (a.prologue == 2) {
      if (comp == rhs && p == 0 && x0 + xx == 0) v.x += T(1);
    }
    int pos = p;
    if (pad) {
      const int k = sfreq(p, a.Nlog);
      pos = k < 0 ? k + M : k;
    }
    A[xx * M + pos] = v;
  }
  __syncthreads();
  cpx<T>* res = fft_pencils<T>(A, B, XC, M, a.plan, Ws, a.dir);
  cpx<T>* out = reinterpret_cast<cpx<T>*>(a.out) + (long long)s * a.out_slab;
  const bool trunc = a.dir < 0 && a.Pout != M;
  for (int t = threadIdx.x; t < a.Pout * XC; t += blockDim.x) {
    const int i = t / XC;
    const int xx = t - i * XC;
    int pos = i;
    if (trunc) {
      const int k = sfreq(i, a.Nlog);
      pos = k < 0 ? k + M : k;
    }
    out[(long long)i * a.X + x0 + xx] = res[xx * M + pos];
  }
}

// ---------------------------------------------------------------------------------
// final forward pass + truncation + projection (+ CG partial p.q)
// ---------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_final(FinalArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int M = a.M;
  const int C = a.C;
  cpx<T>* Ws = reinterpret_cast<cpx<T>*>(smem);
  cpx<T>* A = Ws + M;
  cpx<T>* B = A + (size_t)C * a.XC * M;
  double* red = reinterpret_cast<double*>(B + (size_t)C * a.XC * M);
  const int rhs = blockIdx.y;
  if (a.cg != nullptr && !a.cg->active[rhs]) return;
  const int x0 = blockIdx.x * a.XC;
  const int XC = min(a.XC, a.X - x0);
  load_twiddles<T>(Ws, a.W, M);
  const cpx<T>* in = reinterpret_cast<const cpx<T>*>(a.in) + (long long)rhs * C * a.in_comp;
  const int per = M * XC;
  for (int t = threadIdx.x; t < C * per; t += blockDim.x) {
    const int g = t / per;
    const int rem = t - g * per;
    const int p = rem / XC;
    const int xx = rem - p * XC;
    A[(g * XC + xx) * M + p] = in[(long long)g * a.in_comp + (long long)p * a.X + x0 + xx];
  }
  __syncthreads();
  cpx<T>* res = fft_pencils<T>(A, B, C * XC, M, a.plan, Ws, -1);
  cpx<T>* out = reinterpret_cast<cpx<T>*>(a.out) + (long long)rhs * C * a.out_comp;
  const cpx<T>* pdir = (a.cg && a.aux) ? reinterpret_cast<const cpx<T>*>(a.aux) + (long long)rhs * C * a.out_comp
                                       : nullptr;
  const cpx<T>* bsub = a.bsub ? reinterpret_cast<const cpx<T>*>(a.bsub) + (long long)rhs * C * a.out_comp
                              : nullptr;
  double acc = 0.0;
  for (int t = threadIdx.x; t < a.Nlog * XC; t += blockDim.x) {
    const int i = t / XC;
    const int xx = t - i * XC;
    const int kl = sfreq(i, a.Nlog);
    const int pos = kl < 0 ? kl + M : kl;
    const int x = x0 + xx;
    int kx, ky, kz;
    if (a.d == 3) {
      const int iy = x / a.Nh;
      kx = x - iy * a.Nh;
      ky = sfreq(iy, a.Ny);
      kz = kl;
    } else {
      kx = x;
      ky = kl;
      kz = 0;
    }
    cpx<T> u[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = c < C ? res[(c * XC + xx) * M + pos] : mk<T>(T(0), T(0));
    if (a.project) {
      const T xi[3] = {T(kx * a.invY[0]), T(ky * a.invY[1]), T(kz * a.invY[2])};
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
    const long long oi = (long long)i * a.X + x;
    if (bsub) {
      double s = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (c < C) {
          u[c] = sub<T>(bsub[(long long)c * a.out_comp + oi], u[c]);
          s += (double)u[c].x * (double)u[c].x + (double)u[c].y * (double)u[c].y;
        }
      acc += (kx == 0 ? 1.0 : 2.0) * s;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < C) out[(long long)c * a.out_comp + oi] = u[c];
    if (pdir) {
      const double w = kx == 0 ? 1.0 : 2.0;
      double s = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (c < C) {
          const cpx<T> pv = pdir[(long long)c * a.out_comp + oi];
          s += (double)pv.x * (double)u[c].x + (double)pv.y * (double)u[c].y;
        }
      acc += w * s;
    }
  }
  if (a.partial) {
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) a.partial[rhs * a.partial_ld + blockIdx.x] = s;
  }
}

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

template <typename T>
__global__ void __launch_bounds__(kThreads) k_xpass(XArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int M = a.M;
  const int p0 = blockIdx.x * a.YB;
  const int YB = min(a.YB, a.planes - p0);
  int rhs = 0, comp0 = 0, rpp;
  if (a.mode == 0) {
    rhs = blockIdx.y;
    rpp = a.C;
    if (a.cg != nullptr && !a.cg->active[rhs]) return;
  } else if (a.mode == 1) {
    rpp = a.R * a.C;
  } else {
    comp0 = blockIdx.y;
    rpp = 1;
  }
  const int nrow = YB * rpp;
  const int npair = (nrow + 1) / 2;
  const int bufsz = npair * (M + 1);
  cpx<T>* Ws = reinterpret_cast<cpx<T>*>(smem);
  cpx<T>* A = Ws + M;
  cpx<T>* B = A + bufsz;
  double* red = reinterpret_cast<double*>(B + bufsz);
  const int Nin = a.Nin;
  const cpx<T>* in = reinterpret_cast<const cpx<T>*>(a.in);
  auto row_off = [&](int row) -> long long {
    const int yy = row / rpp;
    const int rem = row - yy * rpp;
    const int f = a.mode == 0 ? rhs * a.C + rem : (a.mode == 1 ? rem : comp0);
    return (long long)f * a.comp_stride + (long long)(p0 + yy) * Nin;
  };
  // stage the rows
  for (int t = threadIdx.x; t < nrow * Nin; t += blockDim.x) {
    const int row = t / Nin;
    const int k = t - row * Nin;
    B[t] = in[row_off(row) + k];
  }
  load_twiddles<T>(Ws, a.W, M);
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
  cpx<T>* res = fft_pencils<T>(A, B, npair, M, a.plan, Ws, +1);
  cpx<T>* oth = res == A ? B : A;
  const T* coef = reinterpret_cast<const T*>(a.coef);
  const long long cstride = (long long)a.planes * M;
  if (a.mode == 0) {
    const int C = a.C;
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
      apply_coef<T>(coef, (long long)(p0 + yy) * M + x, cstride, a.ncomp, C, u, v, T(a.scale));
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (c < C) {
          const int row = yy * C + c;
          if (row & 1) res[(row >> 1) * M + x].y = v[c];
          else res[(row >> 1) * M + x].x = v[c];
        }
    }
    __syncthreads();
    cpx<T>* r2 = fft_pencils<T>(res, oth, npair, M, a.plan, Ws, -1);
    cpx<T>* out = reinterpret_cast<cpx<T>*>(a.out);
    const int Nout = a.Nout;
    for (int t = threadIdx.x; t < nrow * Nout; t += blockDim.x) {
      const int row = t / Nout;
      const int k = t - row * Nout;
      const int pp = row >> 1;
      const cpx<T> zk = r2[pp * M + k];
      const cpx<T> zm = r2[pp * M + (k == 0 ? 0 : M - k)];
      cpx<T> X;
      if ((row & 1) == 0) {
        X = mk<T>(T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y));
      } else {
        X = mk<T>(T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x));
      }
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
      for (int s = 0; s < 3; ++s)
        if (s < R) {
          T v[3];
          apply_coef<T>(coef, (long long)(p0 + yy) * M + x, cstride, a.ncomp, C, u[s], v, T(1));
#pragma unroll
          for (int r = 0; r < 3; ++r)
            if (r < R) {
              double e = 0.0;
#pragma unroll
              for (int c = 0; c < 3; ++c)
                if (c < C) e += (double)u[r][c] * (double)v[c];
              acc[r * 3 + s] += e;
            }
        }
    }
    for (int r = 0; r < R; ++r)
      for (int s = 0; s < R; ++s) {
        const double v = block_sum(acc[r * 3 + s], red);
        if (threadIdx.x == 0) a.partial[(long long)blockIdx.x * R * R + r * R + s] = v;
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

// ---------------------------------------------------------------------------------
// closed-form Fourier coefficients of the matrix-inclusion coefficient
// ---------------------------------------------------------------------------------
// (sin q - q cos q) / q^3, with its Taylor series near 0
__device__ __forceinline__ double ball_radial(double q) {
  if (q < 0.1) {
    const double q2 = q * q;
    return 1.0 / 3.0 + q2 * (-1.0 / 30.0 + q2 * (1.0 / 840.0 + q2 * (-1.0 / 45360.0 + q2 / 3991680.0)));
  }
  double s, c;
  sincos(q, &s, &c);
  return (s - q * c) / (q * q * q);
}

// J1(q) / q, with its Taylor series near 0
__device__ __forceinline__ double disk_radial(double q) {
  if (q < 1e-3) return 0.5 - q * q / 16.0;
  return j1(q) / q;
}

__device__ void ahat_eval(const SpecArgs& a, const int* ni, const int* ns, double2* out) {
  for (int q = 0; q < a.ncomp; ++q) out[q] = make_double2(0.0, 0.0);
  if (ns[0] == 0 && ns[1] == 0 && ns[2] == 0)
    for (int q = 0; q < a.ncomp; ++q) out[q].x = a.A0p[q];
  double rad = 0.0;
  for (int j = 0; j < a.nincl; ++j) {
    const DevIncl& I = a.incl[j];
    double f;
    if (I.shape == 0) {
      f = a.invVol;
      for (int al = 0; al < a.d; ++al) f *= a.sinc[((long long)j * 3 + al) * a.Mmax + ni[al]];
    } else {
      if (!I.same_as_prev) {
        double xi2 = 0.0;
        for (int al = 0; al < a.d; ++al) {
          const double xi = ns[al] * a.invY[al];
          xi2 += xi * xi;
        }
        const double R = I.h[0];
        const double q = 2.0 * M_PI * R * sqrt(xi2);
        rad = a.d == 3 ? 4.0 * M_PI * R * R * R * ball_radial(q) : 2.0 * M_PI * R * R * disk_radial(q);
      }
      f = rad * a.invVol;
    }
    double2 ph = a.phase[((long long)j * 3 + 0) * a.Mmax + ni[0]];
    for (int al = 1; al < a.d; ++al) {
      const double2 t = a.phase[((long long)j * 3 + al) * a.Mmax + ni[al]];
      ph = make_double2(ph.x * t.x - ph.y * t.y, ph.x * t.y + ph.y * t.x);
    }
    for (int q = 0; q < a.ncomp; ++q) {
      const double s = f * I.dA[q];
      out[q].x = fma(s, ph.x, out[q].x);
      out[q].y = fma(s, ph.y, out[q].y);
    }
  }
}

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

__device__ __forceinline__ int sym_index(int d, int al, int be) {
  if (al == be) return al;
  const int lo = al < be ? al : be, hi = al < be ? be : al;
  if (d == 2) return 2;
  if (lo == 1 && hi == 2) return 3;
  if (lo == 0 && hi == 2) return 4;
  return 5;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_rhs(SpecArgs a, int side, int Nh, int N1, int N2,
                                                   cpx<T>* b, double* partial, int ld) {
  __shared__ double red[32];
  const int r = blockIdx.y;
  const int C = a.d;
  const long long field = (long long)Nh * N1 * N2;
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < field;
       e += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(e % Nh);
    const int iy = (int)((e / Nh) % N1);
    const int iz = (int)(e / ((long long)Nh * N1));
    const int ns[3] = {kx, sfreq(iy, N1), a.d == 3 ? sfreq(iz, N2) : 0};
    const int ni[3] = {kx, ns[1] < 0 ? ns[1] + a.M[1] : ns[1], ns[2] < 0 ? ns[2] + a.M[2] : ns[2]};
    double2 Ah[6];
    ahat_eval(a, ni, ns, Ah);
    double2 v[3];
    for (int c = 0; c < C; ++c) {
      if (a.ncomp == 1) v[c] = c == r ? Ah[0] : make_double2(0.0, 0.0);
      else v[c] = Ah[sym_index(a.d, c, r)];
    }
    double xi[3], n2 = 0.0;
    double2 dot = make_double2(0.0, 0.0);
    for (int c = 0; c < C; ++c) {
      xi[c] = ns[c] * a.invY[c];
      n2 += xi[c] * xi[c];
      dot.x += xi[c] * v[c].x;
      dot.y += xi[c] * v[c].y;
    }
    const double w = kx == 0 ? 1.0 : 2.0;
    for (int c = 0; c < C; ++c) {
      double2 g = make_double2(0.0, 0.0);
      if (n2 > 0.0) {
        const double2 ge = make_double2(xi[c] * dot.x / n2, xi[c] * dot.y / n2);
        g = side == 0 ? ge : make_double2(v[c].x - ge.x, v[c].y - ge.y);
      }
      const cpx<T> bv = mk<T>(T(-g.x), T(-g.y));
      b[((long long)r * C + c) * field + e] = bv;
      acc += w * ((double)bv.x * bv.x + (double)bv.y * bv.y);
    }
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partial[r * ld + blockIdx.x] = s;
}

// ---------------------------------------------------------------------------------
// CG vector update and scalar kernels (one CTA), deterministic reductions
// ---------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_cg_update(cpx<T>* x, cpx<T>* r, const cpx<T>* p,
                                                         const cpx<T>* q, int C, long long field,
                                                         int Nh, CgScalars* cg, double* partial,
                                                         int ld) {
  __shared__ double red[32];
  const int rhs = blockIdx.y;
  if (!cg->active[rhs]) return;
  const T al = T(cg->alpha[rhs]);
  const long long n = (long long)C * field;
  const long long base = (long long)rhs * n;
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const cpx<T> pv = p[base + e], qv = q[base + e];
    cpx<T> xv = x[base + e], rv = r[base + e];
    xv = mk<T>(fma(al, pv.x, xv.x), fma(al, pv.y, xv.y));
    rv = mk<T>(fma(-al, qv.x, rv.x), fma(-al, qv.y, rv.y));
    x[base + e] = xv;
    r[base + e] = rv;
    const double w = (e % Nh) == 0 ? 1.0 : 2.0;
    acc += w * ((double)rv.x * rv.x + (double)rv.y * rv.y);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partial[rhs * ld + blockIdx.x] = s;
}

__device__ double reduce_row(const double* v, int n, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
  s = block_sum(s, red);
  return s;  // thread 0
}

__global__ void k_cg_init(CgScalars* cg, const double* partial, int ld, int nblk, int nrhs,
                          double tol2_abs, double rel2, int guard) {
  __shared__ double red[32];
  for (int r = 0; r < 3; ++r) {
    double s = 0.0;
    if (r < nrhs) s = reduce_row(partial + (long long)r * ld, nblk, red);
    __syncthreads();
    if (threadIdx.x == 0) {
      const double t2 = fmax(tol2_abs, rel2 * s);
      cg->tol2[r] = t2;
      cg->beta[r] = 0.0;
      cg->alpha[r] = 0.0;
      cg->iters[r] = 0;
      cg->rr[r] = s;
      cg->rr_min[r] = s;
      cg->min_iter[r] = 0;
      cg->guard = guard;
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

__global__ void k_cg_alpha(CgScalars* cg, const double* partial, int ld, int nblk, int nrhs) {
  __shared__ double red[32];
  for (int r = 0; r < nrhs; ++r) {
    if (!cg->active[r]) continue;
    const double pq = reduce_row(partial + (long long)r * ld, nblk, red);
    __syncthreads();
    if (threadIdx.x == 0) {
      cg->pq[r] = pq;
      if (!(pq > 0.0) || !isfinite(pq)) {
        cg->active[r] = 0;
        cg->status[r] = cg->guard ? 2 : -2;
      } else {
        cg->alpha[r] = cg->rr[r] / pq;
      }
    }
    __syncthreads();
  }
}

__global__ void k_cg_beta(CgScalars* cg, const double* partial, int ld, int nblk, int nrhs) {
  __shared__ double red[32];
  for (int r = 0; r < nrhs; ++r) {
    if (!cg->active[r]) continue;
    const double rr = reduce_row(partial + (long long)r * ld, nblk, red);
    __syncthreads();
    if (threadIdx.x == 0) {
      cg->iters[r] += 1;
      if (!isfinite(rr)) {
        cg->active[r] = 0;
        cg->status[r] = cg->guard ? 2 : -2;
      } else if (rr <= cg->tol2[r]) {
        cg->active[r] = 0;
        cg->status[r] = 0;
        cg->rr[r] = rr;
      } else if (cg->guard && (rr > 1e4 * cg->rr_min[r] || cg->iters[r] - cg->min_iter[r] > 40)) {
        // FP32 inner solve diverging or stagnating at its accuracy floor: stop, keep x
        cg->active[r] = 0;
        cg->status[r] = 2;
        cg->rr[r] = rr;
      } else {
        cg->beta[r] = rr / cg->rr[r];
        cg->rr[r] = rr;
        if (rr < cg->rr_min[r]) {
          cg->rr_min[r] = rr;
          cg->min_iter[r] = cg->iters[r];
        }
      }
    }
    __syncthreads();
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
                                                      long long field, int Nh, const CgScalars* outer,
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
    const double wt = (e % Nh) == 0 ? 1.0 : 2.0;
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

template <typename T>
__global__ void k_project_promote(const cpx<T>* x, double2* x64, int nrhs, int d, int Ny, int Nz,
                                  int Nh, double iy0, double iy1, double iy2, int side) {
  const long long field = (long long)Nh * Ny * Nz;
  const double invY[3] = {iy0, iy1, iy2};
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nrhs * field;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t / field);
    const long long e = t - r * field;
    const int kx = (int)(e % Nh);
    const int iy = (int)((e / Nh) % Ny);
    const int iz = (int)(e / ((long long)Nh * Ny));
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
    for (int c = 0; c < d; ++c) {
      double2 g = make_double2(0.0, 0.0);
      if (n2 > 0.0) {
        const double2 ge = make_double2(xi[c] * dot.x / n2, xi[c] * dot.y / n2);
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

__global__ void k_convert_d2f(const double* in, float* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fft_batch(const cpx<T>* in, cpx<T>* out, int M,
                                                         int howmany, int G, int dir, const void* W,
                                                         FftPlan plan) {
  extern __shared__ __align__(16) unsigned char smem[];
  cpx<T>* Ws = reinterpret_cast<cpx<T>*>(smem);
  cpx<T>* A = Ws + M;
  cpx<T>* B = A + (size_t)G * M;
  const int g0 = blockIdx.x * G;
  const int Ge = min(G, howmany - g0);
  load_twiddles<T>(Ws, W, M);
  for (int t = threadIdx.x; t < Ge * M; t += blockDim.x) A[t] = in[(long long)g0 * M + t];
  __syncthreads();
  cpx<T>* res = fft_pencils<T>(A, B, Ge, M, plan, Ws, dir);
  for (int t = threadIdx.x; t < Ge * M; t += blockDim.x) out[(long long)g0 * M + t] = res[t];
}

// ---------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------
static int current_device() {
  int dev = 0;
  cudaGetDevice(&dev);
  return dev;
}

template <typename F>
static cudaError_t ensure_smem(F* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  static thread_local size_t done[64][4] = {};
  static thread_local const void* fns[64] = {};
  const int dev = current_device() & 3;
  int slot = -1;
  for (int i = 0; i < 64; ++i) {
    if (fns[i] == (const void*)fn) { slot = i; break; }
    if (fns[i] == nullptr) { fns[i] = (const void*)fn; slot = i; break; }
  }
  if (slot >= 0 && done[slot][dev] >= bytes) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && slot >= 0) done[slot][dev] = bytes;
  return e;
}

template <typename T> int pencil_xc(int M, int X, int C) {
  const size_t sz = sizeof(cpx<T>);
  const size_t fixed = M * sz + 512;
  const size_t per = 2 * (size_t)C * M * sz;
  long long xc = (long long)((kSmemBudget > fixed ? kSmemBudget - fixed : 0) / per);
  if (xc < 1) xc = (fixed + per <= kSmemMax) ? 1 : 0;
  if (xc > 32) xc = 32;
  if (xc > X) xc = X;
  return (int)xc;
}

template <typename T> int xpass_yb(int M, int rpp, int planes) {
  const size_t sz = sizeof(cpx<T>);
  const size_t fixed = M * sz + 512;
  const long long npmax = (long long)((kSmemBudget - fixed) / (2 * (size_t)(M + 1) * sz));
  long long yb = (2 * npmax) / rpp;
  if (yb < 1) {
    const size_t need = fixed + 2 * (size_t)((rpp + 1) / 2) * (M + 1) * sz;
    yb = need <= kSmemMax ? 1 : 0;
  }
  if (yb > 32) yb = 32;
  if (yb > planes) yb = planes;
  return (int)yb;
}

template <typename T> cudaError_t launch_pencil(const PencilArgs& a, cudaStream_t s) {
  const size_t smem = (size_t)a.plan.M * sizeof(cpx<T>) * (1 + 2 * (size_t)a.XC);
  cudaError_t e = ensure_smem(k_pencil<T>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.X + a.XC - 1) / a.XC, a.nslab);
  k_pencil<T><<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_final(const FinalArgs& a, cudaStream_t s) {
  const size_t smem = (size_t)a.M * sizeof(cpx<T>) * (1 + 2 * (size_t)a.C * a.XC) + 32 * sizeof(double);
  cudaError_t e = ensure_smem(k_final<T>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.X + a.XC - 1) / a.XC, a.nrhs);
  k_final<T><<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_xpass(const XArgs& a, int grid_y, cudaStream_t s) {
  const int rpp = a.mode == 0 ? a.C : (a.mode == 1 ? a.R * a.C : 1);
  const int npair = (a.YB * rpp + 1) / 2;
  const size_t smem = (size_t)a.M * sizeof(cpx<T>) + 2 * (size_t)npair * (a.M + 1) * sizeof(cpx<T>) +
                      32 * sizeof(double);
  cudaError_t e = ensure_smem(k_xpass<T>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.planes + a.YB - 1) / a.YB, grid_y);
  k_xpass<T><<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_axis_tables(int nincl, int d, const int* M, int Mmax, const double* invY,
                               const DevIncl* incl, double2* phase, double* sinc, cudaStream_t s) {
  if (nincl == 0) return cudaSuccess;
  const long long total = (long long)nincl * 3 * Mmax;
  const int blocks = (int)((total + kThreads - 1) / kThreads);
  k_axis_tables<<<blocks, kThreads, 0, s>>>(nincl, d, M[0], M[1], M[2], Mmax, invY[0], invY[1],
                                            invY[2], incl, phase, sinc);
  return cudaGetLastError();
}

cudaError_t launch_spectrum(const SpecArgs& a, double2* out, cudaStream_t s) {
  const long long total = (long long)a.len[0] * a.len[1] * a.len[2];
  long long blocks = (total + kThreads - 1) / kThreads;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_spectrum<<<(int)blocks, kThreads, 0, s>>>(a, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rhs(const SpecArgs& a, int side, int nrhs, int Nh, const int* N, void* b,
                       double* partial, int nblk, cudaStream_t s) {
  dim3 grid(nblk, nrhs);
  k_rhs<T><<<grid, kThreads, 0, s>>>(a, side, Nh, N[1], N[2], reinterpret_cast<cpx<T>*>(b),
                                     partial, nblk);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_update(void* x, void* r, const void* p, const void* q, int nrhs, int C,
                             long long field, int Nh, CgScalars* cg, double* partial, int nblk,
                             cudaStream_t s) {
  dim3 grid(nblk, nrhs);
  k_cg_update<T><<<grid, kThreads, 0, s>>>(
      reinterpret_cast<cpx<T>*>(x), reinterpret_cast<cpx<T>*>(r), reinterpret_cast<const cpx<T>*>(p),
      reinterpret_cast<const cpx<T>*>(q), C, field, Nh, cg, partial, nblk);
  return cudaGetLastError();
}

cudaError_t launch_cg_init(CgScalars* cg, const double* partial, int ld, int nblk, int nrhs,
                           double tol2_abs, double rel2, int guard, cudaStream_t s) {
  k_cg_init<<<1, kThreads, 0, s>>>(cg, partial, ld, nblk, nrhs, tol2_abs, rel2, guard);
  return cudaGetLastError();
}
cudaError_t launch_outer_check(CgScalars* cg, const double* partial, int ld, int nblk, int nrhs,
                               double shrink2, cudaStream_t s) {
  k_outer_check<<<1, kThreads, 0, s>>>(cg, partial, ld, nblk, nrhs, shrink2);
  return cudaGetLastError();
}
cudaError_t launch_demote(const double2* r64, float2* r32, int nrhs, int C, long long field, int Nh,
                          const CgScalars* outer, double* partial, int nblk, cudaStream_t s) {
  dim3 grid(nblk, nrhs);
  k_demote<<<grid, kThreads, 0, s>>>(r64, r32, C, field, Nh, outer, partial, nblk);
  return cudaGetLastError();
}
cudaError_t launch_promote_add(const float2* x32, double2* x64, long long n, cudaStream_t s) {
  long long blocks = (n + kThreads - 1) / kThreads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_promote_add<<<(int)blocks, kThreads, 0, s>>>(x32, x64, n);
  return cudaGetLastError();
}
cudaError_t launch_cg_alpha(CgScalars* cg, const double* partial, int ld, int nblk, int nrhs,
                            cudaStream_t s) {
  k_cg_alpha<<<1, kThreads, 0, s>>>(cg, partial, ld, nblk, nrhs);
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
  const long long total = (long long)nrhs * Nh * Ny * Nz;
  long long blocks = (total + kThreads - 1) / kThreads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_project_promote<T><<<(int)blocks, kThreads, 0, s>>>(reinterpret_cast<const cpx<T>*>(x), x64, nrhs,
                                                        d, Ny, Nz, Nh, invY[0], invY[1], invY[2], side);
  return cudaGetLastError();
}

cudaError_t launch_energy_reduce(const double* partial, int nblk, int nrr, double* out,
                                 cudaStream_t s) {
  k_energy_reduce<<<1, kThreads, 0, s>>>(partial, nblk, nrr, out);
  return cudaGetLastError();
}

cudaError_t launch_convert_d2f(const double* in, float* out, long long n, cudaStream_t s) {
  long long blocks = (n + kThreads - 1) / kThreads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_convert_d2f<<<(int)blocks, kThreads, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fft_batch(const void* in, void* out, int M, int howmany, int dir, const void* W,
                             const FftPlan& plan, cudaStream_t s) {
  int G = pencil_xc<T>(M, howmany, 1);
  if (G < 1) return cudaErrorInvalidValue;
  const size_t smem = (size_t)M * sizeof(cpx<T>) * (1 + 2 * (size_t)G);
  cudaError_t e = ensure_smem(k_fft_batch<T>, smem);
  if (e != cudaSuccess) return e;
  const int blocks = (howmany + G - 1) / G;
  k_fft_batch<T><<<blocks, kThreads, smem, s>>>(reinterpret_cast<const cpx<T>*>(in),
                                                reinterpret_cast<cpx<T>*>(out), M, howmany, G, dir, W,
                                                plan);
  return cudaGetLastError();
}

// explicit instantiations
#define HOMB_INST(T)                                                                             \
  template cudaError_t launch_pencil<T>(const PencilArgs&, cudaStream_t);                        \
  template cudaError_t launch_final<T>(const FinalArgs&, cudaStream_t);                          \
  template cudaError_t launch_xpass<T>(const XArgs&, int, cudaStream_t);                         \
  template int pencil_xc<T>(int, int, int);                                                      \
  template int xpass_yb<T>(int, int, int);                                                       \
  template cudaError_t launch_rhs<T>(const SpecArgs&, int, int, int, const int*, void*, double*, \
                                     int, cudaStream_t);                                         \
  template cudaError_t launch_cg_update<T>(void*, void*, const void*, const void*, int, int,     \
                                           long long, int, CgScalars*, double*, int,             \
                                           cudaStream_t);                                        \
  template cudaError_t launch_project_promote<T>(const void*, double2*, int, int, int, int, int, \
                                                 const double*, int, cudaStream_t);              \
  template cudaError_t launch_fft_batch<T>(const void*, void*, int, int, int, const void*,       \
                                           const FftPlan&, cudaStream_t);
HOMB_INST(double)
HOMB_INST(float)

}  // namespace homb
