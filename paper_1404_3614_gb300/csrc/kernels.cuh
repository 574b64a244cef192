// Launch interface between the C-ABI layer (api.cu) and the kernels (kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace homb {

// Pencil pass along a strided axis: data[slab][P][X] with X contiguous.
// dir = +1: input holds Nlog frequencies in FFT order, zero-padded to M, inverse
//           transform, M outputs (Pout == M).
// dir = -1: input holds M grid values, forward transform, the Nlog kept
//           frequencies are written in FFT order (Pout == Nlog).
// prologue: 0 none; 1 CG direction update p = r + beta p (in = p, aux = r, writes p);
//           2 add the constant field e_rhs at k = 0 (energy fields u = e + x).
struct PencilArgs {
  const void* in;
  void* out;
  const void* aux;
  long long in_slab, out_slab;
  int nslab, X, XC, Pin, Pout, Nlog, dir;
  int slabs_per_rhs, slabs_per_comp, C;
  int prologue;
  const void* W;
  FftPlan plan;
  CgScalars* cg;   // may be null: no skipping
  int pgrid;       // > 0: the persistent pipelined z pass with this many CTAs (zpipe_pad_grid)
  int in64;        // float-float passes: `in` holds FP64 (double2) data, converted on load
  FastDiv fd_XC;   // divides by XC (set by the launcher)
};

// Last forward pass (z in 3D, y in 2D) over all C components of one field:
// in [rhs][c][M][X] -> out [rhs][c][N][X], then Gamma^E / Gamma^J (project = 1 / 2),
// none (0), and with `cg` the CG partial sums p.q (aux = p).
struct FinalArgs {
  const void* in;
  void* out;
  const void* aux;
  long long in_comp, out_comp;   // element stride between components
  int nrhs, C, X, XC, M, Nlog;
  int project;                   // 0 none, 1 Gamma^E, 2 Gamma^J
  int d, Ny, Nh;                 // frequency decoding (3D: X = Ny*Nh; 2D: X = Nh)
  double invY[3];
  const void* W;
  FftPlan plan;
  CgScalars* cg;
  double* partial;               // [rhs][gridDim.x]
  int partial_ld;
  const void* bsub;              // residual mode: out = bsub - Gamma(...), partial |out|^2
  int pgrid;                     // > 0: the persistent pipelined z pass with this many CTAs
                                 // (zpipe_final_grid; partial sums [rhs][pgrid])
  int pxc;                       // its positions per chunk: 8 or 16
  FastDiv fd_XC, fd_per, fd_Nh;  // set by the launcher
};

// Row pass along x (the contiguous axis) on rows of Nin complex values (k1 >= 0):
// mode 0 (matvec): c2r, v = (A u) * scale per grid point, r2c, keep Nout values;
// mode 1 (energy): c2r, partial sums of u_r . A u_s over the rows;
// mode 2 (c2r):    c2r only, real rows written to out_real.
struct XArgs {
  const void* in;
  void* out;           // mode 0: complex rows (may equal in); mode 2: real rows
  const void* coef;    // real [ncomp][planes][M]
  int mode;
  int planes;          // rows per component (Mz*My)
  int YB;              // planes per CTA
  int Nin, Nout, M;
  int R, C, ncomp, d;
  long long comp_stride;  // elements between components of the row storage
  double scale;
  const void* W;
  FftPlan plan;
  CgScalars* cg;
  double* partial;        // mode 1: [gridDim.x][R*R]
  FastDiv fd_Nin, fd_Nout, fd_rpp;   // set by the launcher
};

// fused y-x-y slab pass (3D, isotropic coefficient, M = R * R on x and y)
struct SlabArgs {
  const void* in;       // [nrc][Mz][Ny][Nh] half spectra after the z inverse transform
  void* out;            // same layout (may equal in)
  const void* coef;     // real [Mz][M][M]
  const void* W;        // twiddles w_M^j, j < M
  const CgScalars* cg;  // skip right-hand sides that have converged (may be NULL)
  int nrc, C, Mz, M, Ny, Nh;
  double scale;         // 1 / |M|
  int warps;            // warps per CTA, 0: automatic
  int* fault;           // set to 1 when a staged input copy did not complete (may be NULL)
};

struct DevIncl {
  int shape;       // 0 box, 1 ball / disk
  int same_as_prev;// 1 when shape and size equal the previous inclusion's (radial reuse)
  double c[3];
  double h[3];     // box sides, or radius in h[0]
  double dA[6];    // increment of this side's coefficient, packed symmetric
};

struct SpecArgs {
  int d, ncomp, nincl;
  int M[3];        // double grid (1 for unused axes)
  int len[3];      // stored extents of the output index set (x is the half range)
  int Nmod[3];     // modulus for signed decoding of y/z storage indices
  double invY[3];
  double invVol;
  double A0p[6];
  const DevIncl* incl;
  const double2* phase;   // [nincl][3][Mmax]
  const double* sinc;     // [nincl][3][Mmax]
  int Mmax;
  const double* bitmap;   // pixel image ([P3][P2][P1], x fastest) or NULL
  int P[3];
  int invert;             // dual side of an image: 1 / a
  int closed;             // GaNi sampling: boundary points belong to the inclusion
  // Radial factors of the balls / disks, [group][n] for n = |k|^2 = 0 .. radlen - 1 (integer
  // frequencies, cells with one side length on every axis); a group is a ball and the equal
  // balls after it (same_as_prev). NULL: evaluated per frequency.
  const double* radtab = nullptr;
  int radlen = 0;
};

// One batched 2D task: a (problem, side) pair solved entirely by one CTA of the
// persistent batch kernel (coefficient build, CG on both right-hand sides, FP64 energies).
struct BTask {
  int prob, side, ncomp, nincl, incl_off;
  int N0, N1, M0, M1, Nh, Nxs;
  double invY[2];
  double invVol;
  double C0p[3];
  int tw0, tw1;            // offsets of the length-M0 / M1 tables in the twiddle pools
  FftPlan plan0, plan1;
};

struct BArgs {
  const BTask* tasks;
  int ntasks;
  int* counter;            // queue head of the cooperative tasks (zero before launch)
  int* counter2;           // queue head of the single-CTA tasks (zero before launch)
  int ncoop;               // tasks [0, ncoop) are worked on by whole clusters
  const DevIncl* incl;
  const double2* tw64;
  const float2* tw32;
  unsigned char* slots;    // per-CTA scratch, slot_bytes each
  long long slot_bytes;
  double* energy;          // [ntasks][4]: W[r][s] / |M|
  int* iters;              // [ntasks][2]
  int* status;             // [ntasks][2]: 0 converged, 1 max_iter, 2 stopped by the FP32 guard, -2 breakdown
  double* resid;           // [ntasks][2]: final recursive residual norm
  double tol2;
  int max_iter;
  int cap;                 // shared-memory chunk capacity (complex FP64 elements)
  int M0max, M1max;
  const void* x0;          // optional starting fields [prob][side][rhs][comp][N1][Nh] (working precision)
  void* fields;            // optional final CG fields, same layout
  int wpass;               // FP32: warp-owned pencil passes for 2N-1 in {45, 125, 225, 405}
};

// bytes of one batch scratch slot for a task (same formula on host and device)
__host__ __device__ inline long long batch_slot_bytes(const BTask& t, int elem) {
  auto al = [](long long b) { return (b + 255) & ~255LL; };
  const long long fld = (long long)t.N1 * t.Nh;
  const int Mmax = t.M0 > t.M1 ? t.M0 : t.M1;
  long long work = (long long)t.ncomp * t.M1 * t.Nxs;
  if (4LL * t.M1 * t.Nh > work) work = 4LL * t.M1 * t.Nh;
  long long b = 0;
  b += al((long long)t.ncomp * t.M1 * t.M0 * 8);          // coef64
  b += al((long long)t.ncomp * t.M1 * t.M0 * (elem / 2)); // coefT
  b += al((long long)(t.nincl > 0 ? t.nincl : 1) * 3 * Mmax * 16);  // phase
  b += al((long long)(t.nincl > 0 ? t.nincl : 1) * 3 * Mmax * 8);   // sinc
  b += al(work * 16);                                      // work area (FP64 complex)
  b += 4 * al(4 * fld * elem);                             // x r p q
  b += al(4 * fld * 16);                                   // x64
  return b;
}

// dynamic shared memory of the batch kernel for working precision of `elem` bytes per complex
inline size_t batch_smem_bytes(int M0max, int M1max, int cap, int elem) {
  const size_t tw = ((size_t)(M0max + M1max) * (16 + elem) + 15) & ~(size_t)15;
  return tw + 2 * (size_t)cap * 16;
}
// threads per CTA: 256 (two CTAs per SM), 512 or 1024 (one CTA per SM); cluster: CTAs per
// thread-block cluster (1, 2, 4 or 8; nblocks a multiple of it)
template <typename T>
cudaError_t launch_batch(const BArgs& a, int nblocks, size_t smem, int threads, int cluster, cudaStream_t s);
// CTAs that can be resident at once on the device for a launch of this configuration
template <typename T> int batch_max_blocks(size_t smem, int threads, int cluster);

// launchers (return cudaGetLastError())
template <typename T> cudaError_t launch_pencil(const PencilArgs& a, cudaStream_t s);
template <typename T> cudaError_t launch_final(const FinalArgs& a, cudaStream_t s);
template <typename T> cudaError_t launch_xpass(const XArgs& a, int grid_y, cudaStream_t s);
template <typename T> int pencil_xc(int M, int X, int C);   // chunk that fits shared memory
// Persistent pipelined z passes of the FP32 3D operator at M = 225 (zpipe.cuh): their CTA
// counts on a device with `sms` SMs, 0 where they do not apply (another length, a transform
// that is not the zero-padded inverse / truncating forward one of the operator)
int zpipe_pad_grid(int M, int Pin, int Pout, int Nlog, int dir, int X, int nslab, int sms);
int zpipe_final_grid(int M, int Nlog, int d, int C, int X, int nrhs, int sms, int xc = 8);
template <typename T> int xpass_yb(int M, int rows_per_plane, int planes);
// fused y-x-y slab pass; cudaErrorNotSupported when the length or size does not apply
template <typename T> cudaError_t launch_slab(const SlabArgs& a, cudaStream_t s);
template <typename T> int slab_warps(int M, int Nh);   // 0: slab pass not applicable

cudaError_t launch_axis_tables(int nincl, int d, const int* M, int Mmax, const double* invY,
                               const DevIncl* incl, double2* phase, double* sinc, cudaStream_t s);
// Fourier coefficients of the side's coefficient on the half index set of Z_M,
// out [ncomp][Mz][My][(Mx+1)/2] complex FP64.
cudaError_t launch_spectrum(const SpecArgs& a, double2* out, cudaStream_t s);
// a.radtab (writable) from the inclusions: entries of each ball group for n = 0 .. radlen - 1
cudaError_t launch_radial_table(const SpecArgs& a, double* radtab, int groups, cudaStream_t s);
// The closed-form spectrum in float-float arithmetic from float-float copies of a's tables
// (phase_ff, sinc_ff: nincl x 3 x Mmax entries; rad_ff: the nrad entries of a.radtab, which
// every ball needs); at most 128 inclusions. Written in FP64 like launch_spectrum.
cudaError_t launch_spectrum_ff(const SpecArgs& a, long long nrad, ffloat2* phase_ff, ffloat* sinc_ff, ffloat* rad_ff,
                               double2* out, cudaStream_t s);
// b_r(k) = -Gamma(k) A_hat(k) e_r on Z_N (half), FP64 or FP32, plus |b|^2 partials; A_hat(k)
// from the closed form, or read from `hat` ([ncomp][N2][N1][Nh]) when it is given.
template <typename T>
cudaError_t launch_rhs(const SpecArgs& a, int side, int nrhs, int Nh, const int* N, void* b,
                       double* partial, int nblk, cudaStream_t s, const double2* hat = nullptr);
// alpha from the operator pass's p.Cp partials pq_part[rhs][pq_nblk] (row stride pq_ld), then
// x += alpha p, r -= alpha Cp and the |r|^2 partials into `partial` (a different buffer)
template <typename T>
cudaError_t launch_cg_update(void* x, void* r, const void* p, const void* q, int nrhs, int C,
                             long long field, int Nh, CgScalars* cg, double* partial, int nblk,
                             const double* pq_part, int pq_ld, int pq_nblk, cudaStream_t s);
// r.r from the partials; tol2[r] = max(tol2_abs, rel2 * r.r); guard as given.
// With drift > 0 (an FP32 inner solve), the absolute target is raised from tol2_abs toward
// tol2_hi: (sqrt(tol2_hi) - drift |r0|)^2 when that is larger, drift |r0| bounding how far the
// recursive residual may end up from the true one.
cudaError_t launch_cg_init(CgScalars* cg, const double* partial, int ld, int nblk, int nrhs,
                           double tol2_abs, double rel2, int guard, cudaStream_t s, double tol2_hi = 0.0,
                           double drift = 0.0);
// outer refinement step: r.r_new from the partials; converged when <= tol2[r]; stalled
// (status 1, stop) when r.r_new > shrink2 * r.r.
cudaError_t launch_outer_check(CgScalars* cg, const double* partial, int ld, int nblk, int nrhs,
                               double shrink2, cudaStream_t s);
// r32 = (float) r64 for active outer rhs (0 otherwise), plus |r32|^2 partials
cudaError_t launch_demote(const double2* r64, float2* r32, int nrhs, int C, long long field, int Nh,
                          const CgScalars* outer, double* partial, int nblk, cudaStream_t s);
// x64 += (double) x32
cudaError_t launch_promote_add(const float2* x32, double2* x64, long long n, cudaStream_t s);
cudaError_t launch_cg_beta(CgScalars* cg, const double* partial, int ld, int nblk, int nrhs,
                           cudaStream_t s);
// GaNi coefficient sampled at the grid points of the M = N grid (a.M = N), packed symmetric
cudaError_t launch_sample_coef(const SpecArgs& a, double* coef, cudaStream_t s);
// pixel image: D = a (or 1 / a) as complex, n values
cudaError_t launch_bitmap_load(const double* bmp, double2* D, long long n, int invert, cudaStream_t s);
// FMA-rate probe: `blocks` CTAs of 512 threads, 8 chains x `iters` FMAs per thread
cudaError_t launch_fma_probe(int precision_fp64, int blocks, int iters, cudaStream_t s);
// the local average of a pixel image (Sec. 7.3), periodic, out-of-place
cudaError_t launch_bitmap_smooth(const double* raw, double* out, int d, const int P[3], cudaStream_t s);
// out[a][c][b] = in[c][b][a] for an [P2][P1][P0] array (the next axis becomes contiguous)
cudaError_t launch_rotate3(const double2* in, double2* out, int P0, int P1, int P2, cudaStream_t s);
// spectrum of a pixel image on the half of Z_M (layout of launch_spectrum, one component) from
// the unnormalised DFT D of the image values ([P3][P2][P1], x fastest)
cudaError_t launch_bitmap_spectrum(const SpecArgs& a, const double2* D, double2* S, cudaStream_t s);
// S(n) = scale * D(n mod N) on the half of Z_M (N-periodic extension of an N-point DFT)
cudaError_t launch_periodic_spectrum(const SpecArgs& a, const double2* D, double2* S, const int* N, double scale,
                                     cudaStream_t s);
// r = -r with |r|^2 partials [nrhs][nblk]
template <typename T>
cudaError_t launch_negate_norm(void* r, int nrhs, int C, long long field, int Nh, double* partial, int nblk,
                               cudaStream_t s);
// Rayleigh-Ritz on span{x} per right-hand side (q = C x given): s = (x.b)/(x.C x), x = s x,
// r = b - s q (r may alias b), |r|^2 partials [nrhs][nblk]; rrpart holds [nrhs][2][nblk]
template <typename T>
cudaError_t launch_rayleigh_ritz(void* x, void* r, const void* b, const void* q, int nrhs, int C, long long field,
                                 int Nh, double* rrpart, double* partial, int nblk, cudaStream_t s);
struct Coef3 { double v[9]; };   // 3 x 3 row-major coefficients passed by value
// u_b = sum_a c[b*3+a] (e_a + x_a) in place over nrhs FP64 fields of d components
cudaError_t launch_combine_fields(double2* x, int nrhs, int d, long long field, const double* c,
                                  cudaStream_t s);
// half-spectrum fields [count][Nz][Ny][(Nx+1)/2] of grid `from` onto grid `to` (same d)
template <typename T>
cudaError_t launch_resample(const void* in, void* out, long long count, int d, const int* from, const int* to,
                            cudaStream_t s);
// x64 = Gamma (double) x_T (in place allowed for T = double)
template <typename T>
cudaError_t launch_project_promote(const void* x, double2* x64, int nrhs, int d, int Ny, int Nz,
                                   int Nh, const double* invY, int side, cudaStream_t s);
// The bound energies of a side from x (in the range of Gamma), its residual r = b - C x and b
// (FP64 half spectra [R][C][field]) and the FP64 double-grid coefficient (its grid sum gives
// the cell mean): out[a R + c] in the energy pass's convention (grid sums). part needs
// nblk * 2 R^2 doubles, cpart cblk * ncomp; three launches.
cudaError_t launch_energy_identity(const double2* b, const double2* x, const double2* r, int R, int C,
                                   long long field, int Nh, const double* coef, int ncomp, long long grid,
                                   double* part, int nblk, double* cpart, int cblk, double* out, cudaStream_t s);
// Block Rayleigh-Ritz start of one side from R FP64 starting fields x (in place), q = C x, the
// right-hand sides b; writes x, r = b - C x and |r|^2 partials [rhs][nblk]. part: nblk * 18
// doubles; coefs: 9 doubles. Three launches.
cudaError_t launch_block_rayleigh_ritz(double2* x, double2* r, const double2* b, const double2* q, int R, int C,
                                       long long field, int Nh, double* part, double* coefs, double* partial,
                                       int nblk, cudaStream_t s);
cudaError_t launch_energy_reduce(const double* partial, int nblk, int nrr, double* out,
                                 cudaStream_t s);
cudaError_t launch_convert_d2f(const double* in, float* out, long long n, cudaStream_t s);
// FP64 -> FP32 (out) and float-float (off) in one pass
cudaError_t launch_convert_d2f_ff(const double* in, float* out, ffloat* off, long long n, cudaStream_t s);
// x = c + b (x - a) for n doubles
cudaError_t launch_affine(double* x, long long n, double a, double b, double c, cudaStream_t s);
template <typename T>
cudaError_t launch_fft_batch(const void* in, void* out, int M, int howmany, int dir, const void* W,
                             const FftPlan& plan, cudaStream_t s);

}  // namespace homb
