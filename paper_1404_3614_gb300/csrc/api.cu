// C ABI (include/homb.h): problem validation, plans, workspace layout and the
// orchestration of the guaranteed-bounds pipeline on one GPU.
//
// Pipeline per side (Algorithm of Sec. 6.2, with the exact double-grid operator of
// Lemma double-grid inside CG as the Galerkin method without numerical integration):
//   1. closed-form Fourier coefficients on Z_{2N-1} (Lemma bounds_for_matrix-inclusion)
//      -> inverse FFT -> A_{2N-1}(x_j) (Eq. MBA_GA), once per problem;
//   2. d right-hand sides b = -Gamma A_hat(k) e_a (Eq. linear_system_primal / _dual),
//      solved together by d independent CG recurrences sharing every operator pass;
//   3. FP64 re-projection of the fields and the exact double-grid energies
//      (Def. upper_lower_bounds) -> upper = A_bar, lower = inv(B_bar).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/homb.h"
#include "kernels.cuh"
#include "net.cuh"

using namespace homb;

struct hom_ctx {
  int device = 0;
  std::string err;
  CgScalars* host_cg = nullptr;        // pinned staging for convergence polls
  double* host_e = nullptr;            // pinned staging for energies
  std::string prof_family;
  std::vector<cudaEvent_t> ev;         // start/stop pairs
  size_t ev_used = 0;
  // kernel timing inside captured graphs: event pairs recorded by the graph's own nodes,
  // read after each replay and summed here
  std::vector<cudaEvent_t>* capture_events = nullptr;
  double graph_prof_ms = 0;
  long long graph_prof_n = 0;
  bool graph_prof_off = false;
  long long launches = 0;              // kernels launched (since the call began)
  long long h2d = 0, d2h = 0;          // bytes copied
  // batched path: pinned staging, captured graph and autotuned chunk capacities
  unsigned char* pin_in = nullptr;
  size_t pin_in_bytes = 0;
  unsigned char* pin_out = nullptr;
  size_t pin_out_bytes = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  // network: DFT bases already uploaded to this workspace for this grid / mode count
  const void* net_bases_ws = nullptr;
  int net_bases_N = 0, net_bases_modes = 0, net_bases_d = 0;
  // single-problem paths: tables already at the front of this workspace for this problem
  std::vector<unsigned char> tables_key;
  // CG iteration blocks captured as graphs (private capture stream, replayed on the caller's)
  cudaStream_t cap_stream = nullptr;
  struct CgGraph {
    std::vector<unsigned char> key;
    cudaGraphExec_t exec;
    long long launches;
    std::vector<cudaEvent_t> events;   // timing pairs of the profiled kernel family, if any
  };
  std::vector<CgGraph> cg_graphs;
  bool graphs_off = false;
  bool slab_on = true;   // fused y-x-y slab pass where it applies
  int zpipe_mask = 1;    // persistent pipelined FP32 z passes where they apply: 1 last pass, 2 z inverse
  double inner_drift = 0.0;   // drift coefficient of the FP32 inner target (0: default)
  double inner_floor = 0.0;   // relative floor of the FP32 inner target (0: default)
  int refine_arith = 0;       // arithmetic of the mixed residual: 0 default, 1 FP64, 2 float-float
  int sms = 0;           // SMs of the device (set at creation)
  int slab_warps = 0;     // warps per slab CTA chosen by the caller (0: automatic)
  int ypass_xc = 0;       // pencils per CTA of the operator's y passes (0: automatic)
  int xpass_yb = 0;       // planes per CTA of the operator's row pass (0: automatic)
  std::vector<long long> graph_key;
  struct Tuned { long long key; int cap, threads, sched, cluster, coopM; };
  std::vector<Tuned> tuned_cap;
  int batch_threads = 0;   // threads per batched CTA set by the caller (0: tuned / default)
  int graph_launched[6] = {0, 0, 0, 0, 0, 0};   // launch configuration inside the batch graph
  int batch_cluster = 0;   // cluster size set by the caller (0: tuned / default)
  int batch_wpass = 1;     // FP32 batched iterations: warp-owned pencil passes where they apply
  int batch_coopM = 0;     // with batch_cluster: cells at least this large are cooperative
  // tensor-core GEMMs: this context's timeout flag and the test limit on barrier polls
  int gemm_slot = 0;
  long long gemm_spin = 0;
  int net_chunk = 0;        // cells per network forward of a batch's learned start (0: by bytes)
  // learned warm start: the network parameters already uploaded to this workspace offset
  unsigned long long net_params_id = 0;
  const void* net_params_at = nullptr;
  std::vector<unsigned char> net_params_tables;   // tables_key when they were uploaded
};

// A warm-start network loaded from a file: config and FP32 parameters on the host.
struct hom_net {
  hom_net_config cfg;
  std::vector<float> params;
  unsigned long long id;   // unique per loaded object: keys the parameter upload to a workspace
};

namespace {

constexpr double kInnerDrift = 100.0;   // default drift coefficient of the FP32 inner target
constexpr double kInnerFloor = 1e-5;    // default relative floor of the FP32 inner target
constexpr bool kRefineFF = true;         // default arithmetic of the mixed residual: float-float (measured faster)
constexpr double kFFResidRel = 2e-14;    // rounding of a float-float operator application relative
                                         // to its output (measured 1.1e-14 on the 16-ball cell)
constexpr int kVecBlocks = 304;   // 2 x 152 SMs for the elementwise CG kernels

#define CK(expr)                                                                               \
  do {                                                                                         \
    cudaError_t _e = (expr);                                                                   \
    if (_e != cudaSuccess) {                                                                   \
      char _b[256];                                                                            \
      snprintf(_b, sizeof _b, "%s:%d: %s (%s)", __FILE__, __LINE__, cudaGetErrorString(_e), #expr); \
      ctx->err = _b;                                                                           \
      return HOM_ERR_CUDA;                                                                     \
    }                                                                                          \
  } while (0)

// a kernel launch: checked and counted
#define KL(expr)          \
  do {                    \
    CK(expr);             \
    ++ctx->launches;      \
  } while (0)
// a launcher that starts n kernels
#define KLN(expr, n)          \
  do {                        \
    CK(expr);                 \
    ctx->launches += (n);     \
  } while (0)

#define CKS(expr)                                                                              \
  do {                                                                                         \
    hom_status _s = (expr);                                                                    \
    if (_s != HOM_OK) return _s;                                                               \
  } while (0)

cudaError_t h2d_copy(hom_ctx* ctx, void* dst, const void* src, size_t bytes, cudaStream_t st) {
  ctx->h2d += (long long)bytes;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
}
cudaError_t d2h_copy(hom_ctx* ctx, void* dst, const void* src, size_t bytes, cudaStream_t st) {
  ctx->d2h += (long long)bytes;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st);
}

hom_status fail(hom_ctx* ctx, hom_status s, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return s;
}

// ---------------------------------------------------------------------------------
// geometry / validation
// ---------------------------------------------------------------------------------
struct Geometry {
  int d = 2;
  int N[3] = {1, 1, 1};
  int M[3] = {1, 1, 1};
  int Nh = 1;       // (N1 + 1)/2: the stored x frequencies 0..Nh-1 (an even N1 has no Nyquist column)
  bool even = false;   // some axis has an even N (general grids, Def. FD_proj_E)
  int Nxs = 1;      // (M1 + 1)/2 = N1: half range of the coefficient spectrum
  double Y[3] = {1, 1, 1};
  double invY[3] = {1, 1, 1};
  int ncomp = 1;
  long long field = 0;   // Nz*Ny*Nh
  long long planes = 0;  // Mz*My
  long long grid = 0;    // Mz*My*Mx
  long long spec = 0;    // Mz*My*Nxs
  double A0[3][3];
  std::vector<hom_inclusion> incl;
  FftPlan plan[3];
  // pixel image of an isotropic conductivity ([P2][P1] or [P3][P2][P1], x fastest), or empty
  std::vector<double> bitmap;
  int P[3] = {1, 1, 1};
  FftPlan pplan[3];            // DFT plans of the image lengths
  uint64_t bitmap_hash = 0;
  int smooth = 0;              // replace the image by its local average (Sec. 7.3) on the device
  int closed = 0;              // GaNi: boundary grid points belong to the inclusion (Eq. S2)
  // GaNi on the double grid (an N without a fast FFT length): the GaNi matrix as the Galerkin
  // operator of the periodized sample spectrum; nplan are the N-point DFT plans of the samples
  bool gani_dg = false;
  FftPlan nplan[3];
  long long nsamp() const { return (long long)N[0] * N[1] * N[2]; }
  long long npix() const { return (long long)P[0] * P[1] * P[2]; }
};

bool spd(const double* A, int d) {
  // symmetric (relative to the largest entry) and Cholesky-positive (leading dim 3)
  double amax = 0.0;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      if (!std::isfinite(A[3 * i + j])) return false;
      amax = std::max(amax, std::fabs(A[3 * i + j]));
    }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < i; ++j)
      if (std::fabs(A[3 * i + j] - A[3 * j + i]) > 1e-12 * amax) return false;
  double L[3][3] = {};
  for (int i = 0; i < d; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = A[3 * i + j];
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      if (i == j) {
        if (!(s > 0)) return false;
        L[i][i] = std::sqrt(s);
      } else {
        L[i][j] = s / L[j][j];
      }
    }
  return true;
}

bool isotropic(const double* A, int d) {
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      if (i != j ? A[3 * i + j] != 0.0 : A[3 * i + i] != A[0]) return false;
  return true;
}

void inv3(const double* A, int d, double* out) {  // leading dim 3
  if (d == 2) {
    const double det = A[0] * A[4] - A[1] * A[3];
    out[0] = A[4] / det; out[1] = -A[1] / det; out[3] = -A[3] / det; out[4] = A[0] / det;
    return;
  }
  const double a = A[0], b = A[1], c = A[2], e = A[3], f = A[4], g = A[5], h = A[6], i = A[7], k = A[8];
  const double det = a * (f * k - g * i) - b * (e * k - g * h) + c * (e * i - f * h);
  out[0] = (f * k - g * i) / det; out[1] = (c * i - b * k) / det; out[2] = (b * g - c * f) / det;
  out[3] = (g * h - e * k) / det; out[4] = (a * k - c * h) / det; out[5] = (c * e - a * g) / det;
  out[6] = (e * i - f * h) / det; out[7] = (b * h - a * i) / det; out[8] = (a * f - b * e) / det;
}

double pdist(double a, double b, double Y) {
  double t = std::fabs(a - b);
  t = std::fmod(t, Y);
  return std::min(t, Y - t);
}

bool overlap(const hom_inclusion& p, const hom_inclusion& q, const double* Y, int d) {
  double dist[3];
  for (int a = 0; a < d; ++a) dist[a] = pdist(p.center[a], q.center[a], Y[a]);
  if (p.shape == HOM_BOX && q.shape == HOM_BOX) {
    for (int a = 0; a < d; ++a)
      if (!(dist[a] < 0.5 * (p.size[a] + q.size[a]))) return false;
    return true;
  }
  if (p.shape == HOM_BALL && q.shape == HOM_BALL) {
    double s = 0;
    for (int a = 0; a < d; ++a) s += dist[a] * dist[a];
    return std::sqrt(s) < p.size[0] + q.size[0];
  }
  const hom_inclusion& bx = p.shape == HOM_BOX ? p : q;
  const hom_inclusion& bl = p.shape == HOM_BOX ? q : p;
  double s = 0;
  for (int a = 0; a < d; ++a) {
    const double o = std::max(pdist(bx.center[a], bl.center[a], Y[a]) - 0.5 * bx.size[a], 0.0);
    s += o * o;
  }
  return std::sqrt(s) < bl.size[0];
}

void make_plan(int M, FftPlan& p) {
  p.M = M;
  p.nrad = 0;
  p.sched = 0;
  int m = M;
  const int small[] = {5, 3, 7, 11, 13, 2};   // 2 only for image lengths (the double grid is odd)
  for (int r : small)
    while (m % r == 0 && p.nrad < kMaxRadices) { p.radix[p.nrad++] = r; m /= r; }
  for (int r = 17; m > 1 && r <= m; r += 2)
    while (m % r == 0 && p.nrad < kMaxRadices) { p.radix[p.nrad++] = r; m /= r; }
}

// Smallest odd M >= m whose prime factors are all radices with butterflies (3, 5, 7, 11,
// 13). The double-grid quadrature (Lemma double-grid) stays exact on any odd M >= 2N - 1:
// the Galerkin entries need A_hat(k - j) for |k - j| <= N - 1, all inside Z_M without
// aliasing, and the grid of M points integrates A_M u v exactly. A length like 809 (prime)
// would otherwise run as one O(M^2) generic radix.
int smooth_odd_at_least(int m) {
  for (int c = m | 1;; c += 2) {
    int r = c;
    for (int p : {3, 5, 7, 11, 13})
      while (r % p == 0) r /= p;
    if (r == 1) return c;
  }
}

// smooth_M: the whole-pipeline calls (hom_bounds, hom_bounds_batched) take the smallest
// smooth odd double grid >= 2N - 1; the step-level calls keep M = 2N - 1 (their coefficient
// and grid layouts are part of the ABI).
hom_status build_geometry(hom_ctx* ctx, const hom_problem* P, Geometry& g, bool smooth_M = false) {
  if (!P) return fail(ctx, HOM_ERR_INVALID_ARG, "problem is NULL");
  if (P->d != 2 && P->d != 3) return fail(ctx, HOM_ERR_INVALID_ARG, "d must be 2 or 3");
  g.d = P->d;
  for (int a = 0; a < 3; ++a) {
    g.N[a] = a < g.d ? P->N[a] : 1;
    g.Y[a] = a < g.d ? P->Y[a] : 1.0;
    if (a < g.d) {
      if (g.N[a] < 1) return fail(ctx, HOM_ERR_INVALID_ARG, "grid sizes N must be >= 1");
      if (g.N[a] % 2 == 0) g.even = true;
      if (g.N[a] > 2049) return fail(ctx, HOM_ERR_INVALID_ARG, "grid size N too large (max 2049)");
      if (!(g.Y[a] > 0) || !std::isfinite(g.Y[a])) return fail(ctx, HOM_ERR_INVALID_ARG, "cell sizes Y must be > 0");
    }
    g.M[a] = 2 * g.N[a] - 1;
    if (smooth_M && a < g.d) g.M[a] = smooth_odd_at_least(g.M[a]);
    g.invY[a] = 1.0 / g.Y[a];
  }
  g.Nh = (g.N[0] + 1) / 2;
  g.Nxs = (g.M[0] + 1) / 2;
  if (P->closed != 0 && P->closed != 1) return fail(ctx, HOM_ERR_INVALID_ARG, "closed must be 0 or 1");
  g.closed = P->closed;
  if (P->smooth != 0 && P->smooth != 1) return fail(ctx, HOM_ERR_INVALID_ARG, "smooth must be 0 or 1");
  if (P->smooth && !P->bitmap) return fail(ctx, HOM_ERR_INVALID_ARG, "smooth applies to pixel images only");
  g.smooth = P->smooth;
  if (P->bitmap) {
    if (P->n_incl != 0) return fail(ctx, HOM_ERR_INVALID_ARG, "a pixel image excludes inclusions");
    long long n = 1;
    for (int a = 0; a < 3; ++a) {
      g.P[a] = a < g.d ? P->bitmap_n[a] : 1;
      if (g.P[a] < 1 || g.P[a] > 4096) return fail(ctx, HOM_ERR_INVALID_ARG, "image sizes must be in [1, 4096]");
      n *= g.P[a];
    }
    if (n > (1LL << 27)) return fail(ctx, HOM_ERR_INVALID_ARG, "image too large (max 2^27 pixels)");
    g.bitmap.assign(P->bitmap, P->bitmap + n);
    uint64_t h = 1469598103934665603ull;   // FNV-1a over the bytes of the image
    for (long long i = 0; i < n; ++i) {
      if (!(g.bitmap[i] > 0) || !std::isfinite(g.bitmap[i]))
        return fail(ctx, HOM_ERR_INVALID_ARG, "image values must be finite and > 0");
      uint64_t bits;
      memcpy(&bits, &g.bitmap[i], 8);
      for (int k = 0; k < 8; ++k) {
        h ^= (bits >> (8 * k)) & 0xff;
        h *= 1099511628211ull;
      }
    }
    g.bitmap_hash = h;
    for (int a = 0; a < 3; ++a) make_plan(g.P[a], g.pplan[a]);
    double mean = 0.0;
    for (long long i = 0; i < n; ++i) mean += g.bitmap[i];
    mean /= (double)n;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) g.A0[i][j] = (i == j && i < g.d) ? mean : 0.0;
  } else if (!spd(P->A0, g.d)) {
    return fail(ctx, HOM_ERR_INVALID_ARG, "A0 is not symmetric positive definite");
  }
  if (P->n_incl < 0 || (P->n_incl > 0 && !P->incl)) return fail(ctx, HOM_ERR_INVALID_ARG, "bad inclusion list");
  if (P->n_incl > 4096) return fail(ctx, HOM_ERR_INVALID_ARG, "too many inclusions (max 4096)");
  g.incl.assign(P->incl, P->incl + P->n_incl);
  bool iso = P->bitmap ? true : isotropic(P->A0, g.d);
  double minY = g.Y[0];
  for (int a = 1; a < g.d; ++a) minY = std::min(minY, g.Y[a]);
  for (size_t j = 0; j < g.incl.size(); ++j) {
    const hom_inclusion& I = g.incl[j];
    if (I.shape != HOM_BOX && I.shape != HOM_BALL) return fail(ctx, HOM_ERR_INVALID_ARG, "unknown inclusion shape");
    if (!spd(I.A, g.d)) return fail(ctx, HOM_ERR_INVALID_ARG, "inclusion phase is not SPD");
    if (I.shape == HOM_BOX) {
      for (int a = 0; a < g.d; ++a)
        if (!(I.size[a] > 0) || I.size[a] > g.Y[a]) return fail(ctx, HOM_ERR_INVALID_ARG, "box side must be in (0, Y]");
    } else if (!(I.size[0] > 0) || 2 * I.size[0] > minY) {
      return fail(ctx, HOM_ERR_INVALID_ARG, "ball radius must be in (0, min(Y)/2]");
    }
    for (int a = 0; a < g.d; ++a)
      if (!std::isfinite(I.center[a])) return fail(ctx, HOM_ERR_INVALID_ARG, "inclusion centre not finite");
    iso = iso && isotropic(I.A, g.d);
    for (size_t k = 0; k < j; ++k)
      if (overlap(I, g.incl[k], g.Y, g.d)) return fail(ctx, HOM_ERR_INVALID_ARG, "inclusions overlap");
  }
  g.ncomp = iso ? 1 : g.d * (g.d + 1) / 2;
  if (!P->bitmap)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) g.A0[i][j] = P->A0[3 * i + j];
  g.field = (long long)g.Nh * g.N[1] * g.N[2];
  g.planes = (long long)g.M[1] * g.M[2];
  g.grid = g.planes * g.M[0];
  g.spec = g.planes * g.Nxs;
  for (int a = 0; a < 3; ++a) make_plan(g.M[a], g.plan[a]);
  return HOM_OK;
}

void pack_sym(const double* A, int d, int ncomp, double* out) {  // A leading dim 3
  if (ncomp == 1) { out[0] = A[0]; return; }
  if (d == 2) { out[0] = A[0]; out[1] = A[4]; out[2] = A[1]; return; }
  out[0] = A[0]; out[1] = A[4]; out[2] = A[8]; out[3] = A[5]; out[4] = A[2]; out[5] = A[1];
}

// ---------------------------------------------------------------------------------
// workspace layout
// ---------------------------------------------------------------------------------
struct Layout {
  size_t tw64[3], tw32[3], twff[3], incl, phase, sinc, coef64, coef32, x, r, p, q, x64, b64, r64, t1, t2,
      cg[2], cgo[2], partial, epart, eout, total;
  size_t bmp = 0, bmpD[2] = {0, 0}, bmptw[3] = {0, 0, 0};   // pixel image, its DFT buffers, twiddles
  size_t rrpart = 0;                                         // Rayleigh-Ritz partial sums
  size_t gs = 0, gD[2] = {0, 0}, gtw[3] = {0, 0, 0};         // GaNi samples, their DFT, twiddles
  int Mmax, maxblk, nblk_energy;
  size_t radtab = 0;            // radial factors of the ball groups (0 bytes: evaluated per frequency)
  size_t coefff = 0;            // float-float coefficient of the mixed residual (0: none)
  size_t phaseff = 0, sincff = 0, radff = 0;   // float-float spectrum tables (mixed path; 0: none)
  int radgroups = 0, radlen = 0;
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  }
};

int final_xc_elem(const Geometry& g, size_t elem) {
  const int M = g.d == 3 ? g.M[2] : g.M[1];
  const int X = g.d == 3 ? g.N[1] * g.Nh : g.Nh;
  return elem == 16 ? pencil_xc<double>(M, X, g.d) : pencil_xc<float>(M, X, g.d);
}

// mode: 0 = hom_bounds (CG vectors in `elem`), 1 = step-level calls
Layout make_layout(const Geometry& g, int R, size_t elem, int mode) {
  Layout L{};
  L.Mmax = std::max(g.M[0], std::max(g.M[1], g.M[2]));
  for (int a = 0; a < 3; ++a) {
    L.tw64[a] = L.take((size_t)g.M[a] * 16);
    L.tw32[a] = L.take((size_t)g.M[a] * 8);
    L.twff[a] = L.take((size_t)g.M[a] * 16);
  }
  const size_t ni = std::max<size_t>(g.incl.size(), 1);
  L.incl = L.take(2 * ni * sizeof(DevIncl));
  L.phase = L.take(ni * 3 * L.Mmax * sizeof(double2));
  L.sinc = L.take(ni * 3 * L.Mmax * sizeof(double));
  {
    // radial factors of the balls / disks on integer |k|^2 when the cell has one side length
    // (then |xi|^2 = |k|^2 / Y^2): one table per group of equal consecutive balls
    bool same_y = true;
    for (int a = 1; a < g.d; ++a) same_y = same_y && g.Y[a] == g.Y[0];
    int groups = 0;
    for (size_t j = 0; j < g.incl.size(); ++j) {
      const hom_inclusion& I = g.incl[j];
      if (I.shape == HOM_BALL && !(j > 0 && g.incl[j - 1].shape == HOM_BALL && I.size[0] == g.incl[j - 1].size[0]))
        ++groups;
    }
    long long len = 1;
    for (int a = 0; a < g.d; ++a) len += (long long)((g.M[a] - 1) / 2) * ((g.M[a] - 1) / 2);
    if (g.bitmap.empty() && same_y && groups > 0 && (long long)groups * len * 8 <= (32LL << 20)) {
      L.radgroups = groups;
      L.radlen = (int)len;
      L.radtab = L.take((size_t)groups * len * sizeof(double));
    }
  }
  if (!g.bitmap.empty()) {
    L.bmp = L.take((size_t)g.npix() * 8);
    L.bmpD[0] = L.take((size_t)g.npix() * 16);
    L.bmpD[1] = L.take((size_t)g.npix() * 16);
    for (int a = 0; a < 3; ++a) L.bmptw[a] = L.take((size_t)g.P[a] * 16);
  }
  if (g.gani_dg) {
    L.gs = L.take((size_t)g.ncomp * g.nsamp() * 8);
    L.gD[0] = L.take((size_t)g.nsamp() * 16);
    L.gD[1] = L.take((size_t)g.nsamp() * 16);
    for (int a = 0; a < 3; ++a) L.gtw[a] = L.take((size_t)g.N[a] * 16);
  }
  const long long RC = (long long)R * g.d;
  const size_t spec_b = (size_t)g.ncomp * g.spec * 16;
  const size_t t1_b = g.d == 3 ? (size_t)RC * g.M[2] * g.N[1] * g.Nh * 16 : 0;
  const size_t t2_b = (size_t)RC * g.planes * g.Nh * 16;
  L.t1 = L.take(std::max(t1_b, spec_b));
  L.t2 = L.take(std::max(t2_b, spec_b));
  if (mode == 0) {
    L.coef64 = L.take((size_t)g.ncomp * g.grid * 8);
    L.coef32 = elem == 8 ? L.take((size_t)g.ncomp * g.grid * 4) : 0;
    L.coefff = elem == 8 ? L.take((size_t)g.ncomp * g.grid * 8) : 0;
    if (elem == 8 && g.bitmap.empty() && !g.incl.empty() && g.incl.size() <= 128) {
      L.phaseff = L.take(g.incl.size() * 3 * L.Mmax * sizeof(ffloat2));
      L.sincff = L.take(g.incl.size() * 3 * L.Mmax * sizeof(ffloat));
      L.radff = L.take(std::max<size_t>((size_t)L.radgroups * L.radlen, 1) * sizeof(ffloat));
    }
    const size_t fb = (size_t)RC * g.field * elem;
    L.x = L.take(fb);
    L.r = L.take(fb);
    L.p = L.take(fb);
    L.q = L.take(fb);
    L.x64 = elem == 8 ? L.take((size_t)RC * g.field * 16) : L.x;
    L.b64 = elem == 8 ? L.take((size_t)RC * g.field * 16) : 0;
    L.r64 = elem == 8 ? L.take((size_t)RC * g.field * 16) : 0;
  }
  L.cg[0] = L.take(sizeof(CgScalars));
  L.cg[1] = L.take(sizeof(CgScalars));
  L.cgo[0] = L.take(sizeof(CgScalars));
  L.cgo[1] = L.take(sizeof(CgScalars));
  const int X = g.d == 3 ? g.N[1] * g.Nh : g.Nh;
  const int xcff = pencil_xc<ffloat>(g.d == 3 ? g.M[2] : g.M[1], X, g.d);
  const int xc = std::max(1, std::min(std::min(final_xc_elem(g, 16), final_xc_elem(g, 8)), xcff > 0 ? xcff : 1 << 30));
  L.maxblk = std::max(kVecBlocks, (X + xc - 1) / xc);
  L.partial = L.take((size_t)3 * L.maxblk * sizeof(double));
  L.rrpart = L.take((size_t)6 * kVecBlocks * sizeof(double));
  L.nblk_energy = (int)g.planes;   // upper bound of the energy pass grid
  // the energy pass's per-block 3x3 sums, or the Fourier-side identity's (kVecBlocks blocks
  // of 2 x 9 sums and of up to 6 coefficient sums)
  L.epart = L.take(std::max((size_t)L.nblk_energy * 9, (size_t)kVecBlocks * 24) * sizeof(double));
  L.eout = L.take(2 * 9 * sizeof(double));
  L.total = L.off;
  return L;
}

void twiddles(int M, std::vector<double2>& w64, std::vector<float2>& w32, std::vector<ffloat2>* wff = nullptr) {
  w64.resize(M);
  w32.resize(M);
  if (wff) wff->resize(M);
  auto split = [](long double v) {   // nearest float-float: hi = fl32(v), lo = fl32(v - hi)
    const float h = (float)v;
    return ffloat(h, (float)(v - (long double)h));
  };
  for (int j = 0; j < M; ++j) {
    const long double ang = -2.0L * 3.14159265358979323846264338327950288L * (long double)j / (long double)M;
    const long double c = std::cos(ang), s = std::sin(ang);
    w64[j] = make_double2((double)c, (double)s);
    w32[j] = make_float2((float)c, (float)s);
    if (wff) (*wff)[j] = ffloat2{split(c), split(s)};
  }
}

// ---------------------------------------------------------------------------------
// per-call runner
// ---------------------------------------------------------------------------------
struct Prof {
  hom_ctx* ctx;
  cudaStream_t s;
  bool on;
  cudaEvent_t stop_ev = nullptr;
  bool ext = false;
  Prof(hom_ctx* c, const char* fam, cudaStream_t st) : ctx(c), s(st), on(false) {
    if (c->prof_family.empty() || c->prof_family != fam) return;
    if (c->capture_events) {   // being captured: the pair becomes two event-record nodes
      cudaEvent_t a, b;
      if (cudaEventCreate(&a) != cudaSuccess) return;
      if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return;
      }
      c->capture_events->push_back(a);
      c->capture_events->push_back(b);
      ext = on = true;
      cudaEventRecordWithFlags(a, s, cudaEventRecordExternal);
      stop_ev = b;
      return;
    }
    if (c->ev_used + 2 > c->ev.size()) {
      for (int i = 0; i < 256; ++i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        c->ev.push_back(e);
      }
    }
    on = true;
    cudaEventRecord(c->ev[c->ev_used], s);
    stop_ev = c->ev[c->ev_used + 1];
    c->ev_used += 2;
  }
  ~Prof() {
    if (on && ext) cudaEventRecordWithFlags(stop_ev, s, cudaEventRecordExternal);
    else if (on) cudaEventRecord(stop_ev, s);
  }
};

// a caller's chunk size (hom_set_pass_chunks) within the shared-memory maximum
static int chunk(int automatic, int requested) {
  return requested > 0 && automatic > 0 ? std::min(automatic, requested) : automatic;
}

struct Runner {
  hom_ctx* ctx;
  const Geometry& g;
  Layout L;
  unsigned char* base;
  cudaStream_t st;
  int R;
  bool gani = false;   // GaNi: g is the N grid (M = N), coefficient sampled at the grid points
  int coef_side = -1;  // side whose double-grid coefficient build_coefficient left in L.coef64
  bool spec_ff = false;  // closed-form spectrum in float-float (the mixed path)

  template <typename X> X* at(size_t off) const { return reinterpret_cast<X*>(base + off); }

  // Twiddle and inclusion tables at the front of the workspace. They are uploaded once per
  // (workspace, problem) and kept across calls on the same context; other layouts that
  // use a workspace (batched, network) clear the record.
  hom_status upload_tables() {
    std::vector<unsigned char> key;
    auto push = [&](const void* p, size_t n) {
      const unsigned char* b = static_cast<const unsigned char*>(p);
      key.insert(key.end(), b, b + n);
    };
    const void* wsp = base;
    push(&wsp, sizeof wsp);
    push(&g.d, sizeof g.d);
    push(g.N, sizeof g.N);
    push(g.Y, sizeof g.Y);
    push(g.A0, sizeof g.A0);
    push(&g.ncomp, sizeof g.ncomp);
    push(&g.closed, sizeof g.closed);
    push(&g.gani_dg, sizeof g.gani_dg);
    push(g.M, sizeof g.M);
    if (!g.incl.empty()) push(g.incl.data(), g.incl.size() * sizeof(hom_inclusion));
    if (!g.bitmap.empty()) {
      push(&g.bitmap_hash, sizeof g.bitmap_hash);
      push(g.P, sizeof g.P);
      push(&g.smooth, sizeof g.smooth);
    }
    if (key == ctx->tables_key) return HOM_OK;
    ctx->tables_key.clear();
    if (!g.bitmap.empty()) {
      if (g.smooth) {   // raw image into the DFT scratch, its local average into the image slot
        CK(h2d_copy(ctx, base + L.bmpD[1], g.bitmap.data(), (size_t)g.npix() * 8, st));
        KL(launch_bitmap_smooth(at<double>(L.bmpD[1]), at<double>(L.bmp), g.d, g.P, st));
      } else {
        CK(h2d_copy(ctx, base + L.bmp, g.bitmap.data(), (size_t)g.npix() * 8, st));
      }
      for (int a = 0; a < 3; ++a) {
        std::vector<double2> w64;
        std::vector<float2> w32;
        twiddles(g.P[a], w64, w32);
        CK(h2d_copy(ctx, base + L.bmptw[a], w64.data(), w64.size() * sizeof(double2), st));
      }
    }
    if (g.gani_dg)
      for (int a = 0; a < 3; ++a) {
        std::vector<double2> w64;
        std::vector<float2> w32;
        twiddles(g.N[a], w64, w32);
        CK(h2d_copy(ctx, base + L.gtw[a], w64.data(), w64.size() * sizeof(double2), st));
      }
    std::vector<double2> w64;
    std::vector<float2> w32;
    std::vector<ffloat2> wff;
    for (int a = 0; a < 3; ++a) {
      twiddles(g.M[a], w64, w32, &wff);
      CK(h2d_copy(ctx, base + L.tw64[a], w64.data(), w64.size() * sizeof(double2), st));
      CK(h2d_copy(ctx, base + L.tw32[a], w32.data(), w32.size() * sizeof(float2), st));
      CK(h2d_copy(ctx, base + L.twff[a], wff.data(), wff.size() * sizeof(ffloat2), st));
    }
    // inclusion tables for both sides: [side][j]
    const size_t n = g.incl.size();
    std::vector<DevIncl> di(2 * std::max<size_t>(n, 1));
    double B0[9] = {};
    double A0f[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) A0f[3 * i + j] = g.A0[i][j];
    inv3(A0f, g.d, B0);
    for (int side = 0; side < 2; ++side)
      for (size_t j = 0; j < n; ++j) {
        const hom_inclusion& I = g.incl[j];
        DevIncl& D = di[side * n + j];
        memset(&D, 0, sizeof D);
        D.shape = I.shape == HOM_BOX ? 0 : 1;
        D.same_as_prev = 0;
        if (j > 0 && I.shape == HOM_BALL && g.incl[j - 1].shape == HOM_BALL && I.size[0] == g.incl[j - 1].size[0])
          D.same_as_prev = 1;
        for (int a = 0; a < 3; ++a) {
          D.c[a] = I.center[a];
          D.h[a] = I.size[a];
        }
        double dA[9] = {};
        if (side == 0) {
          for (int k = 0; k < 9; ++k) dA[k] = I.A[k] - A0f[k];
        } else {
          double Bi[9] = {};
          inv3(I.A, g.d, Bi);
          for (int k = 0; k < 9; ++k) dA[k] = Bi[k] - B0[k];
        }
        pack_sym(dA, g.d, g.ncomp, D.dA);
      }
    CK(h2d_copy(ctx, base + L.incl, di.data(), di.size() * sizeof(DevIncl), st));
    ctx->tables_key = key;
    return HOM_OK;
  }

  bool has_balls() const {
    for (const hom_inclusion& I : g.incl)
      if (I.shape == HOM_BALL) return true;
    return false;
  }

  SpecArgs spec_args(int side) const {
    SpecArgs a{};
    a.d = g.d;
    a.ncomp = g.ncomp;
    a.nincl = (int)g.incl.size();
    for (int k = 0; k < 3; ++k) {
      a.M[k] = g.M[k];
      a.invY[k] = g.invY[k];
    }
    a.len[0] = g.Nxs;
    a.len[1] = g.M[1];
    a.len[2] = g.M[2];
    a.Nmod[0] = g.M[0];
    a.Nmod[1] = g.M[1];
    a.Nmod[2] = g.M[2];
    a.invVol = 1.0 / (g.Y[0] * g.Y[1] * g.Y[2]);
    a.closed = g.closed;
    double C0[9], A0f[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) A0f[3 * i + j] = g.A0[i][j];
    if (side == 0) memcpy(C0, A0f, sizeof C0);
    else inv3(A0f, g.d, C0);
    pack_sym(C0, g.d, g.ncomp, a.A0p);
    a.incl = at<DevIncl>(L.incl) + side * g.incl.size();
    if (!g.bitmap.empty()) {
      a.bitmap = at<double>(L.bmp);
      for (int k = 0; k < 3; ++k) a.P[k] = g.P[k];
      a.invert = side;
    }
    a.phase = at<double2>(L.phase);
    a.sinc = at<double>(L.sinc);
    a.Mmax = L.Mmax;
    a.radtab = L.radlen > 0 ? at<double>(L.radtab) : nullptr;
    a.radlen = L.radlen;
    return a;
  }

  // Double-grid coefficient of one side into `coef` (FP64, real). Uses t1/t2.
  // Unnormalised DFT of the pixel image (or of 1 / a) into L.bmpD[0], layout [P3][P2][P1]:
  // a transform along the contiguous axis, then a rotation that makes the next axis
  // contiguous, three times.
  // Unnormalised forward DFT of a [P2][P1][P0] complex grid (x fastest) in place in D0:
  // along x, then two axis rotations with the next axis' DFT, a third rotation back.
  hom_status dft3(double2* D0, double2* D1, const int* P, const FftPlan* plans, const size_t* tw) {
    double2* const out = D0;
    int P0 = P[0], P1 = P[1], P2 = P[2];
    const long long n = (long long)P0 * P1 * P2;
    for (int step = 0; step < 3; ++step) {
      if (P0 > 1) KL(launch_fft_batch<double>(D0, D0, P0, P1 * P2, -1, base + tw[step], plans[step], st));
      KL(launch_rotate3(D0, D1, P0, P1, P2, st));
      std::swap(D0, D1);
      const int t = P0;
      P0 = P1;
      P1 = P2;
      P2 = t;
    }
    if (D0 != out)   // three swaps: the result is in the other buffer
      CK(cudaMemcpyAsync(out, D0, (size_t)n * 16, cudaMemcpyDeviceToDevice, st));
    return HOM_OK;
  }

  hom_status bitmap_dft(int side) {
    KL(launch_bitmap_load(at<double>(L.bmp), at<double2>(L.bmpD[0]), g.npix(), side, st));
    return dft3(at<double2>(L.bmpD[0]), at<double2>(L.bmpD[1]), g.P, g.pplan, L.bmptw);
  }

  // One material in the inclusions of an isotropic cell (scalar phases a0, a1): the double-grid
  // coefficient is A_M = a0 + (a1 - a0) F_M with F_M the double-grid interpolant of the
  // inclusions' indicator sum, the same F_M on both sides (the dual side's pointwise inverse is
  // 1/a0 + (1/a1 - 1/a0) sum f_j), so the dual coefficient is an affine map of the primal one.
  bool one_material(double* a0, double* a1) const {
    if (g.ncomp != 1 || !g.bitmap.empty() || g.incl.empty()) return false;
    for (const hom_inclusion& I : g.incl)
      for (int k = 0; k < 9; ++k)
        if (I.A[k] != g.incl[0].A[k]) return false;
    *a0 = g.A0[0][0];
    *a1 = g.incl[0].A[0];
    return *a1 != *a0;
  }

  hom_status build_coefficient(int side, double* coef) {
    Prof pr(ctx, "coef", st);
    double a0 = 0.0, a1 = 0.0;
    if (side == 1 && coef_side == 0 && coef == at<double>(L.coef64) && one_material(&a0, &a1)) {
      // A^-1_M = 1/a0 + (1/a1 - 1/a0) F_M = 1/a0 + b (A_M - a0), b = (1/a1 - 1/a0) / (a1 - a0)
      KL(launch_affine(coef, (long long)g.grid, a0, (1.0 / a1 - 1.0 / a0) / (a1 - a0), 1.0 / a0, st));
      coef_side = 1;
      return HOM_OK;
    }
    coef_side = coef == at<double>(L.coef64) ? side : -1;
    SpecArgs sa = spec_args(side);
    double2* S = at<double2>(L.t1);
    if (!g.bitmap.empty()) {
      CKS(bitmap_dft(side));
      KL(launch_bitmap_spectrum(sa, at<double2>(L.bmpD[0]), S, st));
    } else {
      KL(launch_axis_tables(sa.nincl, g.d, g.M, L.Mmax, g.invY, sa.incl, at<double2>(L.phase), at<double>(L.sinc),
                            st));
      if (L.radlen > 0) KL(launch_radial_table(sa, at<double>(L.radtab), L.radgroups, st));
      if (spec_ff && L.phaseff != 0 && (!has_balls() || L.radlen > 0))
        KLN(launch_spectrum_ff(sa, (long long)L.radgroups * L.radlen, at<ffloat2>(L.phaseff), at<ffloat>(L.sincff),
                              at<ffloat>(L.radff), S, st), 2);
      else
        KL(launch_spectrum(sa, S, st));
    }
    return coefficient_from_spectrum(coef);
  }

  // GaNi matrix on the double grid: K_N[l, k] = A_hat_N(l - k mod N) (Lemma FD_of_GaNi) with
  // A_hat_N the N-point DFT (1/|N|) of the grid samples; for |l - k| <= N - 1 and an odd
  // M >= 2N - 1 these are the Galerkin entries of the coefficient whose spectrum on Z_M is
  // the N-periodic extension of A_hat_N, so the double-grid passes apply the GaNi operator
  // exactly, with fast lengths M even when N is prime.
  hom_status gani_coefficient_dg(int side, double* coef) {
    Prof pr(ctx, "coef", st);
    SpecArgs sn = spec_args(side);
    for (int k = 0; k < 3; ++k) sn.M[k] = k < g.d ? g.N[k] : 1;
    KL(launch_sample_coef(sn, at<double>(L.gs), st));
    const SpecArgs sa = spec_args(side);
    double2* S = at<double2>(L.t1);
    const long long total = (long long)sa.len[0] * sa.len[1] * sa.len[2];
    const double scale = 1.0 / (double)g.nsamp();
    for (int q = 0; q < g.ncomp; ++q) {
      KL(launch_bitmap_load(at<double>(L.gs) + q * g.nsamp(), at<double2>(L.gD[0]), g.nsamp(), 0, st));
      CKS(dft3(at<double2>(L.gD[0]), at<double2>(L.gD[1]), g.N, g.nplan, L.gtw));
      KL(launch_periodic_spectrum(sa, at<double2>(L.gD[0]), S + q * total, g.N, scale, st));
    }
    return coefficient_from_spectrum(coef);
  }

  // A_M(x) = sum over Z_M of the half spectrum in t1 (inverse passes z, y, then the rows)
  hom_status coefficient_from_spectrum(double* coef) {
    double2* S = at<double2>(L.t1);
    // 3D: z pass t1 -> t2, y pass t2 -> t1, rows from t1; 2D: y pass t1 -> t2, rows from t2
    const void* cur = S;
    void* nxt = at<void>(L.t2);
    if (g.d == 3) {
      PencilArgs z{};
      z.in = cur; z.out = nxt; z.aux = nullptr;
      z.in_slab = z.out_slab = g.spec;
      z.nslab = g.ncomp; z.X = g.M[1] * g.Nxs;
      z.XC = pencil_xc<double>(g.M[2], z.X, 1);
      z.Pin = z.Pout = z.Nlog = g.M[2]; z.dir = +1;
      z.slabs_per_rhs = z.nslab; z.slabs_per_comp = 1; z.C = 1; z.prologue = 0;
      z.W = base + L.tw64[2]; z.plan = g.plan[2]; z.cg = nullptr;
      if (z.XC < 1) return fail(ctx, HOM_ERR_INVALID_ARG, "grid too large for the shared-memory FFT");
      KL(launch_pencil<double>(z, st));
      cur = at<void>(L.t2);
      nxt = at<void>(L.t1);
    }
    PencilArgs y{};
    y.in = cur; y.out = nxt; y.aux = nullptr;
    y.in_slab = y.out_slab = (long long)g.M[1] * g.Nxs;
    y.nslab = g.ncomp * g.M[2]; y.X = g.Nxs;
    y.XC = pencil_xc<double>(g.M[1], y.X, 1);
    y.Pin = y.Pout = y.Nlog = g.M[1]; y.dir = +1;
    y.slabs_per_rhs = y.nslab; y.slabs_per_comp = 1; y.C = 1; y.prologue = 0;
    y.W = base + L.tw64[1]; y.plan = g.plan[1]; y.cg = nullptr;
    if (y.XC < 1) return fail(ctx, HOM_ERR_INVALID_ARG, "grid too large for the shared-memory FFT");
    KL(launch_pencil<double>(y, st));
    XArgs x{};
    x.in = nxt; x.out = coef; x.coef = nullptr; x.mode = 2;
    x.planes = (int)g.planes; x.YB = xpass_yb<double>(g.M[0], 1, (int)g.planes);
    x.Nin = g.Nxs; x.Nout = 0; x.M = g.M[0]; x.R = 1; x.C = 1; x.ncomp = g.ncomp; x.d = g.d;
    x.comp_stride = g.planes * g.Nxs; x.scale = 1.0;
    x.W = base + L.tw64[0]; x.plan = g.plan[0]; x.cg = nullptr; x.partial = nullptr;
    if (x.YB < 1) return fail(ctx, HOM_ERR_INVALID_ARG, "grid too large for the shared-memory FFT");
    KL(launch_xpass<double>(x, g.ncomp, st));
    return HOM_OK;
  }

  // Operator passes on R fields: out = Gamma^{side} P F (A/|M|) F^{-1} Pad(in).
  // cgmode: first pass updates p = r + beta p (in = p, aux = r), last pass writes p.q partials.
  // project: 0 none, 1 Gamma^E, 2 Gamma^J.  addE: energy-style constant added (not used here).
  template <typename T>
  hom_status matvec(const void* in, void* out, const void* coef, int project, CgScalars* cg,
                    const void* r_aux, const void* p_aux, int prologue, const void* bsub = nullptr) {
    constexpr bool ff = is_ff<T>::value;   // float-float: in and out FP64, passes in FP32 pairs
    auto W = [&](int a) -> const void* { return base + (ff ? L.twff[a] : sizeof(T) == 8 ? L.tw64[a] : L.tw32[a]); };
    const int C = g.d;
    const int Mx = g.M[0], My = g.M[1], Mz = g.M[2];
    const int Ny = g.N[1], Nz = g.N[2], Nh = g.Nh;
    void* T1 = at<void>(L.t1);
    void* T2 = at<void>(L.t2);
    const void* ycur = in;
    if (g.d == 3) {
      Prof pr(ctx, "zpass", st);
      PencilArgs z{};
      z.in = in; z.out = T1; z.aux = r_aux;
      z.in_slab = (long long)Nz * Ny * Nh; z.out_slab = (long long)Mz * Ny * Nh;
      z.nslab = R * C; z.X = Ny * Nh; z.XC = pencil_xc<T>(Mz, z.X, 1);
      z.Pin = Nz; z.Pout = Mz; z.Nlog = Nz; z.dir = +1;
      z.slabs_per_rhs = C; z.slabs_per_comp = 1; z.C = C; z.prologue = prologue;
      z.W = W(2); z.plan = g.plan[2]; z.cg = cg; z.in64 = ff;
      if (sizeof(T) == 4 && (ctx->zpipe_mask & 2))
        z.pgrid = zpipe_pad_grid(Mz, z.Pin, z.Pout, z.Nlog, z.dir, z.X, z.nslab, ctx->sms);
      if (z.XC < 1) return fail(ctx, HOM_ERR_INVALID_ARG, "grid too large for the shared-memory FFT");
      KL(launch_pencil<T>(z, st));
      ycur = T1;
    }
    const void* fin = T2;
    bool use_slab = false;
    if constexpr (!ff)
      use_slab = g.d == 3 && g.ncomp == 1 && g.M[0] == g.M[1] && ctx->slab_on && slab_warps<T>(g.M[0], Nh) > 0;
    if (use_slab) {
      // fused inverse y, x row pass and forward y on each (rhs, comp, z) slab of T1
      if constexpr (!ff) {
        Prof pr(ctx, "slab", st);
        SlabArgs sl{};
        sl.in = T1; sl.out = T1; sl.coef = coef; sl.W = W(0); sl.cg = cg;
        sl.nrc = R * C; sl.C = C; sl.Mz = Mz; sl.M = Mx; sl.Ny = Ny; sl.Nh = Nh;
        sl.scale = 1.0 / (double)g.grid;
        sl.warps = ctx->slab_warps;
        sl.fault = cg ? &cg->fault : nullptr;
        KL(launch_slab<T>(sl, st));
        fin = T1;
      }
    } else {
    {
      Prof pr(ctx, "ypass", st);
      PencilArgs y{};
      y.in = ycur; y.out = T2; y.aux = g.d == 3 ? nullptr : r_aux;
      y.in_slab = (long long)Ny * Nh; y.out_slab = (long long)My * Nh;
      y.nslab = R * C * Mz; y.X = Nh; y.XC = chunk(pencil_xc<T>(My, Nh, 1), ctx->ypass_xc);
      y.Pin = Ny; y.Pout = My; y.Nlog = Ny; y.dir = +1;
      y.slabs_per_rhs = C * Mz; y.slabs_per_comp = Mz; y.C = C;
      y.prologue = g.d == 3 ? 0 : prologue;
      y.W = W(1); y.plan = g.plan[1]; y.cg = cg; y.in64 = ff && g.d == 2;
      if (y.XC < 1) return fail(ctx, HOM_ERR_INVALID_ARG, "grid too large for the shared-memory FFT");
      KL(launch_pencil<T>(y, st));
    }
    {
      Prof pr(ctx, "xpass", st);
      XArgs x{};
      x.in = T2; x.out = T2; x.coef = coef; x.mode = 0;
      x.planes = (int)g.planes; x.YB = chunk(xpass_yb<T>(Mx, C, (int)g.planes), ctx->xpass_yb);
      x.Nin = Nh; x.Nout = Nh; x.M = Mx; x.R = R; x.C = C; x.ncomp = g.ncomp; x.d = g.d;
      x.comp_stride = g.planes * Nh; x.scale = 1.0 / (double)g.grid;
      x.W = W(0); x.plan = g.plan[0]; x.cg = cg; x.partial = nullptr;
      if (x.YB < 1) return fail(ctx, HOM_ERR_INVALID_ARG, "grid too large for the shared-memory FFT");
      KL(launch_xpass<T>(x, R, st));
    }
    if (g.d == 3) {
      Prof pr(ctx, "ypass", st);
      PencilArgs y{};
      y.in = T2; y.out = T1; y.aux = nullptr;
      y.in_slab = (long long)My * Nh; y.out_slab = (long long)Ny * Nh;
      y.nslab = R * C * Mz; y.X = Nh; y.XC = chunk(pencil_xc<T>(My, Nh, 1), ctx->ypass_xc);
      y.Pin = My; y.Pout = Ny; y.Nlog = Ny; y.dir = -1;
      y.slabs_per_rhs = C * Mz; y.slabs_per_comp = Mz; y.C = C; y.prologue = 0;
      y.W = W(1); y.plan = g.plan[1]; y.cg = cg;
      KL(launch_pencil<T>(y, st));
      fin = T1;
    }
    }
    {
      Prof pr(ctx, "final", st);
      FinalArgs f{};
      f.in = fin; f.out = out; f.aux = p_aux;
      const int Mlast = g.d == 3 ? Mz : My;
      const int Nlast = g.d == 3 ? Nz : Ny;
      f.X = g.d == 3 ? Ny * Nh : Nh;
      f.in_comp = (long long)Mlast * f.X; f.out_comp = (long long)Nlast * f.X;
      f.nrhs = R; f.C = C; f.XC = pencil_xc<T>(Mlast, f.X, C); f.M = Mlast; f.Nlog = Nlast;
      f.project = project; f.d = g.d; f.Ny = Ny; f.Nh = Nh;
      for (int k = 0; k < 3; ++k) f.invY[k] = g.invY[k];
      f.W = W(g.d == 3 ? 2 : 1); f.plan = g.plan[g.d == 3 ? 2 : 1];
      f.cg = cg; f.partial_ld = L.maxblk; f.bsub = bsub;
      f.partial = ((cg && p_aux) || bsub) ? at<double>(L.partial) : nullptr;
      if (sizeof(T) == 4 && !bsub) {
        f.pgrid = final_pipe_grid();
        f.pxc = final_pipe_xc();
      }
      if (f.XC < 1) return fail(ctx, HOM_ERR_INVALID_ARG, "grid too large for the shared-memory FFT");
      KL(launch_final<T>(f, st));
    }
    return HOM_OK;
  }

  // CTAs of the persistent FP32 last pass (0: the chunked pass runs), at most one partial
  // sum slot per CTA and right-hand side
  int final_pipe_grid() const {
    if (!(ctx->zpipe_mask & 1)) return 0;
    const int pg = zpipe_final_grid(g.d == 3 ? g.M[2] : g.M[1], g.d == 3 ? g.N[2] : g.N[1], g.d, g.d,
                                    g.d == 3 ? g.N[1] * g.Nh : g.Nh, R, ctx->sms, final_pipe_xc());
    return std::min(pg, L.maxblk);
  }
  int final_pipe_xc() const { return (ctx->zpipe_mask & 4) ? 16 : 8;
  }

  // CTAs (partial sums per right-hand side) of the float-float last pass
  int final_blocks_ff() const {
    const int M = g.d == 3 ? g.M[2] : g.M[1];
    const int X = g.d == 3 ? g.N[1] * g.Nh : g.Nh;
    const int xc = pencil_xc<ffloat>(M, X, g.d);
    return xc > 0 ? (X + xc - 1) / xc : 0;
  }

  int final_blocks(size_t elem) const {
    if (elem == 8 && final_pipe_grid() > 0) return final_pipe_grid();
    const int X = g.d == 3 ? g.N[1] * g.Nh : g.Nh;
    const int xc = final_xc_elem(g, elem);
    return (X + xc - 1) / xc;
  }

  // Energy matrix of the R FP64 fields x64 (u = e_r + x_r when addE) -> eout[slot*9 ...]
  hom_status energy(const double* coef, const double2* x64, int addE, int slot) {
    Prof pr(ctx, "energy", st);
    const int C = g.d;
    const int My = g.M[1], Mz = g.M[2];
    const int Ny = g.N[1], Nz = g.N[2], Nh = g.Nh;
    void* T1 = at<void>(L.t1);
    void* T2 = at<void>(L.t2);
    const void* ycur = x64;
    if (g.d == 3) {
      PencilArgs z{};
      z.in = x64; z.out = T1; z.aux = nullptr;
      z.in_slab = (long long)Nz * Ny * Nh; z.out_slab = (long long)Mz * Ny * Nh;
      z.nslab = R * C; z.X = Ny * Nh; z.XC = pencil_xc<double>(Mz, z.X, 1);
      z.Pin = Nz; z.Pout = Mz; z.Nlog = Nz; z.dir = +1;
      z.slabs_per_rhs = C; z.slabs_per_comp = 1; z.C = C; z.prologue = addE ? 2 : 0;
      z.W = base + L.tw64[2]; z.plan = g.plan[2]; z.cg = nullptr;
      KL(launch_pencil<double>(z, st));
      ycur = T1;
    }
    PencilArgs y{};
    y.in = ycur; y.out = T2; y.aux = nullptr;
    y.in_slab = (long long)Ny * Nh; y.out_slab = (long long)My * Nh;
    y.nslab = R * C * Mz; y.X = Nh; y.XC = pencil_xc<double>(My, Nh, 1);
    y.Pin = Ny; y.Pout = My; y.Nlog = Ny; y.dir = +1;
    y.slabs_per_rhs = C * Mz; y.slabs_per_comp = Mz; y.C = C;
    y.prologue = (g.d == 2 && addE) ? 2 : 0;
    y.W = base + L.tw64[1]; y.plan = g.plan[1]; y.cg = nullptr;
    KL(launch_pencil<double>(y, st));
    XArgs x{};
    x.in = T2; x.out = nullptr; x.coef = coef; x.mode = 1;
    x.planes = (int)g.planes; x.YB = xpass_yb<double>(g.M[0], R * C, (int)g.planes);
    if (x.YB < 1) return fail(ctx, HOM_ERR_INVALID_ARG, "grid too large for the shared-memory FFT");
    x.Nin = Nh; x.Nout = 0; x.M = g.M[0]; x.R = R; x.C = C; x.ncomp = g.ncomp; x.d = g.d;
    x.comp_stride = g.planes * Nh; x.scale = 1.0;
    x.W = base + L.tw64[0]; x.plan = g.plan[0]; x.cg = nullptr; x.partial = at<double>(L.epart);
    KL(launch_xpass<double>(x, 1, st));
    const int nblk = (int)((g.planes + x.YB - 1) / x.YB);
    KL(launch_energy_reduce(at<double>(L.epart), nblk, R * R, at<double>(L.eout) + slot * 9, st));
    return HOM_OK;
  }

  // One CG iteration on R right-hand sides (operator with the p update in its first pass
  // and p.Cp in its last, alpha, x/r update with r.r, beta), enqueued on `st`.
  template <typename T>
  hom_status cg_iteration(CgScalars* cg, const void* coefT, int side, int nfin) {
    CKS(matvec<T>(base + L.p, base + L.q, coefT, side + 1, cg, base + L.r, base + L.p, 1));
    Prof pr(ctx, "cg", st);
    // alpha inside the update (from the last pass's p.Cp partials in L.partial), the |r|^2
    // partials into L.rrpart (the update's CTAs still read L.partial while others write)
    KL(launch_cg_update<T>(base + L.x, base + L.r, base + L.p, base + L.q, R, g.d, g.field, g.Nh, cg,
                           at<double>(L.rrpart), kVecBlocks, at<double>(L.partial), L.maxblk, nfin, st));
    KL(launch_cg_beta(cg, at<double>(L.rrpart), kVecBlocks, kVecBlocks, R, st));
    return HOM_OK;
  }

  // K iterations: replayed from a captured graph (captured once per workspace, problem,
  // side, precision and K on the context's private stream), or launched one by one when
  // graphs are off or kernel timing is on.
  template <typename T>
  hom_status cg_block(CgScalars* cg, const void* coefT, int side, int nfin, int K, bool graphs) {
    const bool prof = !ctx->prof_family.empty();
    if (!graphs || ctx->graphs_off || (prof && ctx->graph_prof_off) || K <= 0) {
      for (int k = 0; k < K; ++k) CKS((cg_iteration<T>(cg, coefT, side, nfin)));
      return HOM_OK;
    }
    std::vector<unsigned char> key = ctx->tables_key;
    const long long extra[13] = {(long long)side, (long long)sizeof(T), K, (long long)(uintptr_t)coefT,
                                 (long long)(uintptr_t)cg, (long long)L.total, R, nfin, ctx->ypass_xc,
                                 ctx->xpass_yb, (long long)ctx->slab_on, ctx->slab_warps,
                                 (long long)ctx->zpipe_mask};
    const unsigned char* eb = reinterpret_cast<const unsigned char*>(extra);
    key.insert(key.end(), eb, eb + sizeof extra);
    key.insert(key.end(), ctx->prof_family.begin(), ctx->prof_family.end());
    for (auto& gr : ctx->cg_graphs)
      if (gr.key == key) {
        CK(cudaGraphLaunch(gr.exec, st));
        ctx->launches += gr.launches;
        return collect_graph_timing(gr);
      }
    if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    const cudaStream_t saved = st;
    const long long l0 = ctx->launches;
    std::vector<cudaEvent_t> events;
    st = ctx->cap_stream;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    ctx->capture_events = &events;
    hom_status s = HOM_OK;
    for (int k = 0; k < K && s == HOM_OK; ++k) s = cg_iteration<T>(cg, coefT, side, nfin);
    ctx->capture_events = nullptr;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &graph);
    st = saved;
    const long long per = ctx->launches - l0;
    ctx->launches = l0;
    if (s != HOM_OK || e != cudaSuccess)
      for (cudaEvent_t ev : events) cudaEventDestroy(ev);
    if (s != HOM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    cudaGraphExec_t exec = nullptr;
    cudaError_t ei = e;
    if (e == cudaSuccess) {
      ei = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
    }
    if (ei != cudaSuccess) {   // capture not possible here: launch this context's kernels directly
      cudaGetLastError();
      if (e == cudaSuccess)
        for (cudaEvent_t ev : events) cudaEventDestroy(ev);
      if (prof) ctx->graph_prof_off = true;
      else ctx->graphs_off = true;
      for (int k = 0; k < K; ++k) CKS((cg_iteration<T>(cg, coefT, side, nfin)));
      return HOM_OK;
    }
    if (ctx->cg_graphs.size() >= 8) {
      cudaGraphExecDestroy(ctx->cg_graphs.front().exec);
      for (cudaEvent_t ev : ctx->cg_graphs.front().events) cudaEventDestroy(ev);
      ctx->cg_graphs.erase(ctx->cg_graphs.begin());
    }
    ctx->cg_graphs.push_back({key, exec, per, std::move(events)});
    CK(cudaGraphLaunch(exec, st));
    ctx->launches += per;
    return collect_graph_timing(ctx->cg_graphs.back());
  }

  // Timing pairs recorded by a replayed graph: wait for the replay, sum the pairs into the
  // context's kernel timing (the next replay reuses the same events).
  hom_status collect_graph_timing(const hom_ctx::CgGraph& gr) {
    if (gr.events.empty()) return HOM_OK;
    CK(cudaStreamSynchronize(st));
    for (size_t i = 0; i + 1 < gr.events.size(); i += 2) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, gr.events[i], gr.events[i + 1]) != cudaSuccess) {
        cudaGetLastError();
        ctx->graph_prof_off = true;   // no timing from graph nodes here: profile without graphs
        return HOM_OK;
      }
      ctx->graph_prof_ms += ms;
      ctx->graph_prof_n += 1;
    }
    return HOM_OK;
  }

  // Start of the dual CG from the primal minimisers (Remark "Avoiding the solution of
  // dual formulation", Eq. FD_superposition_odd_A): for each b, u_b = sum_a E_a (e_a +
  // e^(a)) with E = inv(Abar) e_b (Abar = the primal energy matrix, the upper bound), and
  // j0_b = Gamma^J P_N F_M (A_M/|M|) F_M^{-1} Pad(u_b) with the primal coefficient. Needs
  // the re-projected primal fields in x64, the primal coefficient in coef64 and the primal
  // energies in eout[0..]; writes the FP64 starts to `out`. *ok = false (and nothing
  // written) when the primal energy matrix is not SPD.
  hom_status dual_start(double2* out, bool* ok, int* matvecs) {
    *ok = false;
    CK(d2h_copy(ctx, ctx->host_e, at<double>(L.eout), 9 * sizeof(double), st));
    CK(cudaStreamSynchronize(st));
    const int d = g.d;
    const double invM = 1.0 / (double)g.grid;
    double A[9] = {}, Ai[9] = {};
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) A[3 * i + j] = 0.5 * (ctx->host_e[d * i + j] + ctx->host_e[d * j + i]) * invM;
    if (!spd(A, d)) return HOM_OK;
    inv3(A, d, Ai);
    double c[9] = {};   // c[b][a] = (inv(Abar) e_b)_a
    for (int b = 0; b < R; ++b)
      for (int a = 0; a < d; ++a) c[3 * b + a] = Ai[3 * a + b];
    double2* x64 = at<double2>(L.x64);
    KL(launch_combine_fields(x64, R, d, g.field, c, st));
    CKS(matvec<double>(x64, out, at<double>(L.coef64), 2, nullptr, nullptr, nullptr, 0));
    ++*matvecs;
    *ok = true;
    return HOM_OK;
  }

  // GaNi coefficient: the side's coefficient sampled at the grid points (Def. GaNi)
  hom_status sample_coefficient(int side, double* coef) {
    if (g.gani_dg) return gani_coefficient_dg(side, coef);
    Prof pr(ctx, "coef", st);
    KL(launch_sample_coef(spec_args(side), coef, st));
    return HOM_OK;
  }

  template <typename T>
  hom_status solve_side(int side, const hom_opts& o, hom_report* rep, int* matvecs,
                        const double2* x0 = nullptr, bool user_start = false) {
    const size_t elem = sizeof(T) * 2;
    double* coef64 = at<double>(L.coef64);
    if (gani) CKS(sample_coefficient(side, coef64));
    else CKS(build_coefficient(side, coef64));
    const void* coefT = coef64;
    if (sizeof(T) == 4) {
      KL(launch_convert_d2f(coef64, at<float>(L.coef32), (long long)g.ncomp * g.grid, st));
      coefT = at<float>(L.coef32);
    }
    const size_t fb = (size_t)R * g.d * g.field * elem;
    CK(cudaMemsetAsync(base + L.x, 0, fb, st));
    CK(cudaMemsetAsync(base + L.p, 0, fb, st));
    CgScalars* cg = at<CgScalars>(L.cg[side]);
    SpecArgs sa = spec_args(side);
    const int N3[3] = {g.N[0], g.N[1], g.N[2]};
    if (gani || !g.bitmap.empty()) {
      // b = -Gamma F (A E) (Eq. linear_system_primal; with the GaNi matrix for GaNi, with the
      // double-grid coefficient for a pixel image): the operator applied to the constant
      // field E = e_r (x = 0 here), negated
      CKS(matvec<T>(base + L.x, base + L.r, coefT, side + 1, nullptr, nullptr, nullptr, 2));
      ++*matvecs;
      KL(launch_negate_norm<T>(base + L.r, R, g.d, g.field, g.Nh, at<double>(L.partial), kVecBlocks, st));
    } else {
      KL(launch_rhs<T>(sa, side, R, g.Nh, N3, base + L.r, at<double>(L.partial), kVecBlocks, st));
    }
    const double tol = o.tol > 0 ? o.tol : 1e-8;
    const int nfin = final_blocks(elem);
    if (x0 && sizeof(T) == 8 && user_start) {
      // a caller's start: the Galerkin solution of each right-hand side in the span of the R
      // projected starts Gamma x0 (block Rayleigh-Ritz: never a larger energy error than the
      // per-right-hand-side scaling or than x = 0), r = b - C x
      KL(launch_project_promote<double>(x0, at<double2>(L.x), R, g.d, g.N[1], g.N[2], g.Nh, g.invY, side, st));
      CKS(matvec<T>(base + L.x, base + L.q, coefT, side + 1, nullptr, nullptr, nullptr, 0));
      ++*matvecs;
      double* ep = at<double>(L.epart);
      KLN(launch_block_rayleigh_ritz(at<double2>(L.x), at<double2>(L.r), at<double2>(L.r), at<double2>(L.q), R, g.d,
                                    g.field, g.Nh, ep, ep + (size_t)kVecBlocks * 18, at<double>(L.partial),
                                    kVecBlocks, st), 3);
      KL(launch_cg_init(cg, at<double>(L.partial), kVecBlocks, kVecBlocks, R, tol * tol, 0.0, 0, st));
    } else if (x0 && sizeof(T) == 8) {   // x = x0 (after b, which GaNi forms from x = 0); r0 = b - C x0
      CK(cudaMemcpyAsync(base + L.x, x0, fb, cudaMemcpyDeviceToDevice, st));
      CKS(matvec<T>(base + L.x, base + L.r, coefT, side + 1, nullptr, nullptr, nullptr, 0, base + L.r));
      ++*matvecs;
      KL(launch_cg_init(cg, at<double>(L.partial), L.maxblk, nfin, R, tol * tol, 0.0, 0, st));
    } else {
      KL(launch_cg_init(cg, at<double>(L.partial), kVecBlocks, kVecBlocks, R, tol * tol, 0.0, 0, st));
    }
    // with a caller's start, max_iter = 0 is taken literally: bounds of the projected start
    const int maxit = o.max_iter > 0 ? o.max_iter : ((o.max_iter == 0 && x0 && user_start) ? 0 : 10000);
    const int every = o.check_every > 0 ? o.check_every : 8;
    // an initial poll avoids work when b = 0 (homogeneous cells)
    CK(d2h_copy(ctx, ctx->host_cg, cg, sizeof(CgScalars), st));
    CK(cudaStreamSynchronize(st));
    bool any = false;
    for (int r = 0; r < R; ++r) any = any || ctx->host_cg->active[r];
    const bool graphs = o.graph >= 0;
    for (int it = 0; any && it < maxit;) {
      const int K = std::min(every, maxit - it);
      CKS((cg_block<T>(cg, coefT, side, nfin, K, graphs)));
      *matvecs += K;
      it += K;
      CK(d2h_copy(ctx, ctx->host_cg, cg, sizeof(CgScalars), st));
      CK(cudaStreamSynchronize(st));
      any = false;
      for (int r = 0; r < R; ++r) any = any || ctx->host_cg->active[r];
    }
    CK(d2h_copy(ctx, ctx->host_cg, cg, sizeof(CgScalars), st));
    CK(cudaStreamSynchronize(st));
    if (ctx->host_cg->fault) return fail(ctx, HOM_ERR_TIMEOUT, "an operator pass gave up waiting for its staged input");
    hom_status result = HOM_OK;
    for (int r = 0; r < R; ++r) {
      const CgScalars& h = *ctx->host_cg;
      int stt = h.status[r] == 1 ? 1 : h.status[r];
      if (rep) {
        rep->iters[side][r] = h.iters[r];
        rep->resid[side][r] = std::sqrt(std::max(h.rr[r], 0.0));
        rep->status[side][r] = stt;
      }
      if (stt == -2) result = fail(ctx, HOM_ERR_BREAKDOWN, "CG breakdown (non-finite value or p.Cp <= 0)");
      else if (stt == 1 && result == HOM_OK) result = HOM_WARN_NOT_CONVERGED;
    }
    if (result == HOM_ERR_BREAKDOWN) return result;
    // FP64 re-projection (and promotion for the mixed path), then the exact energies
    KL(launch_project_promote<T>(base + L.x, at<double2>(L.x64), R, g.d, g.N[1], g.N[2], g.Nh, g.invY, side, st));
    CKS(energy(coef64, at<double2>(L.x64), 1, side));
    return result;
  }
};

// Mixed precision (FP32 inner CG, FP64 outer): iterative refinement on the FP64 residual.
// r64 = b - C x64 in FP64; each inner FP32 CG solves C d = r64 to
// max(tol/2, eta |r64|), stopping early when FP32 accuracy runs out; x64 += d. The CG
// scalars (alpha, beta, r.r, p.Cp) are FP64 reductions of FP32 products. The outer loop
// stops at |r64| <= tol |E| or when a step fails to halve |r64|; any field is a valid
// conforming test field after the FP64 re-projection, so the bounds stay guaranteed.
hom_status Runner_solve_mixed(Runner& run, int side, const hom_opts& o, hom_report* rep, int* matvecs,
                              bool warm = false, bool user_start = false) {
  hom_ctx* ctx = run.ctx;
  const Geometry& g = run.g;
  const Layout& L = run.L;
  const int R = run.R;
  cudaStream_t st = run.st;
  unsigned char* base = run.base;
  double* coef64 = run.at<double>(L.coef64);
  // the closed-form spectrum in float-float unless the caller asked for FP64 residuals
  run.spec_ff = ctx->refine_arith != 1;
  if (run.gani) CKS(run.sample_coefficient(side, coef64));
  else CKS(run.build_coefficient(side, coef64));
  // the residual b - C x64 of every refinement step in float-float (FP64 data, FP32-pair
  // arithmetic) or in FP64
  bool ffres = (ctx->refine_arith == 0 ? kRefineFF : ctx->refine_arith == 2) && L.coefff != 0;
  if (ffres)
    KL(launch_convert_d2f_ff(coef64, run.at<float>(L.coef32), run.at<ffloat>(L.coefff), (long long)g.ncomp * g.grid,
                             st));
  else
    KL(launch_convert_d2f(coef64, run.at<float>(L.coef32), (long long)g.ncomp * g.grid, st));
  const float* coef32 = run.at<float>(L.coef32);
  const long long n = (long long)R * g.d * g.field;
  double2* b64 = run.at<double2>(L.b64);
  double2* r64 = run.at<double2>(L.r64);
  double2* x64 = run.at<double2>(L.x64);
  CgScalars* inner = run.at<CgScalars>(L.cg[side]);
  CgScalars* outer = run.at<CgScalars>(L.cgo[side]);
  SpecArgs sa = run.spec_args(side);
  const int N3[3] = {g.N[0], g.N[1], g.N[2]};
  double* partial = run.at<double>(L.partial);
  const double tol = o.tol > 0 ? o.tol : 1e-8;
  const int nfin32 = run.final_blocks(8), nfin64 = run.final_blocks(16), nfinff = run.final_blocks_ff();
  // b in FP64: closed form, or for a pixel image and for GaNi the operator applied to the
  // constant field (x = 0 taken from `zero`), negated
  auto form_rhs = [&](double2* zero) -> hom_status {
    if (g.bitmap.empty() && !run.gani) {
      const double2* hat = nullptr;
      if (run.spec_ff && L.phaseff != 0 && (L.radlen > 0 || !run.has_balls())) {
        // A_hat at the N-grid frequencies in float-float (the coefficient's tables), into the
        // second pass buffer, which nothing holds before the solve
        SpecArgs sn = sa;
        sn.len[0] = g.Nh; sn.len[1] = g.N[1]; sn.len[2] = g.d == 3 ? g.N[2] : 1;
        sn.Nmod[1] = g.N[1]; sn.Nmod[2] = g.d == 3 ? g.N[2] : 1;
        double2* h = run.at<double2>(L.t2);
        KLN(launch_spectrum_ff(sn, (long long)L.radgroups * L.radlen, run.at<ffloat2>(L.phaseff),
                              run.at<ffloat>(L.sincff), run.at<ffloat>(L.radff), h, st), 2);
        hat = h;
      }
      KL(launch_rhs<double>(sa, side, R, g.Nh, N3, b64, partial, kVecBlocks, st, hat));
    } else {
      CK(cudaMemsetAsync(zero, 0, n * sizeof(double2), st));
      CKS(run.matvec<double>(zero, b64, coef64, side + 1, nullptr, nullptr, nullptr, 2));
      ++*matvecs;
      KL(launch_negate_norm<double>(b64, R, g.d, g.field, g.Nh, partial, kVecBlocks, st));
    }
    return HOM_OK;
  };
  if (warm && user_start) {   // a caller's start in b64: block Rayleigh-Ritz over its projection, r64 = b - C x64
    KL(launch_project_promote<double>(b64, x64, R, g.d, g.N[1], g.N[2], g.Nh, g.invY, side, st));
    CKS(form_rhs(r64));
    CKS(run.matvec<double>(x64, r64, coef64, side + 1, nullptr, nullptr, nullptr, 0));
    ++*matvecs;
    double* ep = run.at<double>(L.epart);
    KLN(launch_block_rayleigh_ritz(x64, r64, b64, r64, R, g.d, g.field, g.Nh, ep, ep + (size_t)kVecBlocks * 18,
                                  partial, kVecBlocks, st), 3);
    KL(launch_cg_init(outer, partial, kVecBlocks, kVecBlocks, R, tol * tol, 0.0, 0, st));
  } else if (warm) {   // the start is in b64 (Runner::dual_start): x64 = start, r64 = b - C x64
    CK(cudaMemcpyAsync(x64, b64, n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    CKS(form_rhs(r64));
    CKS(run.matvec<double>(x64, r64, coef64, side + 1, nullptr, nullptr, nullptr, 0, b64));
    ++*matvecs;
    KL(launch_cg_init(outer, partial, L.maxblk, nfin64, R, tol * tol, 0.0, 0, st));
  } else {
    CKS(form_rhs(x64));
    KL(launch_cg_init(outer, partial, kVecBlocks, kVecBlocks, R, tol * tol, 0.0, 0, st));
    CK(cudaMemcpyAsync(r64, b64, n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(x64, 0, n * sizeof(double2), st));
  }
  const int maxit = o.max_iter > 0 ? o.max_iter : ((o.max_iter == 0 && warm && user_start) ? 0 : 10000);
  const int every = o.check_every > 0 ? o.check_every : 8;
  const double eta = ctx->inner_floor > 0.0 ? ctx->inner_floor : kInnerFloor;
  // The recursive FP32 residual of an inner solve (restarted from the FP64 residual) stays
  // within a few eps_32 |r_k| per step of the true one (measured on the 16-ball cell at
  // contrast 1000: equal to four digits); the inner solve aims at tol less c eps_32 |r0|
  // (at least tol / 2), so that the FP64 check after it passes without another refinement step.
  const double drift = (ctx->inner_drift > 0.0 ? ctx->inner_drift : kInnerDrift) * 5.9604644775390625e-8;
  int used = 0;
  int inner_iters[3] = {0, 0, 0};
  for (int outer_it = 0; outer_it < 30; ++outer_it) {
    CK(d2h_copy(ctx, ctx->host_cg, outer, sizeof(CgScalars), st));
    CK(cudaStreamSynchronize(st));
    if (outer_it == 0 && ffres && ctx->refine_arith == 0) {
      // the default keeps float-float residuals only while their rounding, about
      // kFFResidRel |C x64| ~ kFFResidRel |b|, stays a hundredth of the tolerance: the first
      // residual of a cold start is b itself; a warm start does not know |b| and keeps FP64
      double b2 = 0.0;
      for (int r = 0; r < R; ++r) b2 = std::max(b2, ctx->host_cg->rr[r]);
      const double lim = 100.0 * kFFResidRel;
      ffres = !warm && tol * tol >= lim * lim * b2;
    }
    bool any = false;
    for (int r = 0; r < R; ++r) any = any || ctx->host_cg->active[r];
    if (!any || used >= maxit) break;
    // inner FP32 CG on the current FP64 residual, from zero (a restart: keeping the last
    // search direction with the replaced residual made the recursive residual drift from the
    // true one, and so cost another refinement step)
    KL(launch_demote(r64, run.at<float2>(L.r), R, g.d, g.field, g.Nh, outer, partial, kVecBlocks, st));
    CK(cudaMemsetAsync(base + L.x, 0, n * sizeof(float2), st));
    CK(cudaMemsetAsync(base + L.p, 0, n * sizeof(float2), st));
    KL(launch_cg_init(inner, partial, kVecBlocks, kVecBlocks, R, 0.25 * tol * tol, eta * eta, 1, st, tol * tol,
                      drift));
    CK(d2h_copy(ctx, ctx->host_cg, inner, sizeof(CgScalars), st));
    CK(cudaStreamSynchronize(st));
    bool ia = false;
    for (int r = 0; r < R; ++r) ia = ia || ctx->host_cg->active[r];
    while (ia && used < maxit) {
      const int K = std::min(every, maxit - used);
      CKS((run.cg_block<float>(inner, coef32, side, nfin32, K, o.graph >= 0)));
      *matvecs += K;
      used += K;
      CK(d2h_copy(ctx, ctx->host_cg, inner, sizeof(CgScalars), st));
      CK(cudaStreamSynchronize(st));
      ia = false;
      for (int r = 0; r < R; ++r) ia = ia || ctx->host_cg->active[r];
    }
    CK(d2h_copy(ctx, ctx->host_cg, inner, sizeof(CgScalars), st));
    CK(cudaStreamSynchronize(st));
    for (int r = 0; r < R; ++r) inner_iters[r] += ctx->host_cg->iters[r];
    if (ctx->host_cg->fault) return fail(ctx, HOM_ERR_TIMEOUT, "an operator pass gave up waiting for its staged input");
    // x64 += d, re-projected in FP64, then the exact FP64 residual r64 = b - C x64 (so that at
    // the end x64 lies in the range of Gamma and r64 is its residual: the bound energies follow
    // from them without another pass over the double grid)
    KL(launch_promote_add(run.at<float2>(L.x), x64, n, st));
    KL(launch_project_promote<double>(x64, x64, R, g.d, g.N[1], g.N[2], g.Nh, g.invY, side, st));
    if (ffres) CKS(run.matvec<ffloat>(x64, r64, run.at<ffloat>(L.coefff), side + 1, outer, nullptr, nullptr, 0, b64));
    else CKS(run.matvec<double>(x64, r64, coef64, side + 1, outer, nullptr, nullptr, 0, b64));
    // (the float-float last pass runs the warp FFTs on larger chunks: fewer partial sums)
    KL(launch_outer_check(outer, partial, L.maxblk, ffres ? nfinff : nfin64, R, 0.25, st));
    ++*matvecs;
  }
  CK(d2h_copy(ctx, ctx->host_cg, outer, sizeof(CgScalars), st));
  CK(cudaStreamSynchronize(st));
  hom_status result = HOM_OK;
  for (int r = 0; r < R; ++r) {
    const CgScalars& h = *ctx->host_cg;
    const int stt = h.status[r];
    if (rep) {
      rep->iters[side][r] = inner_iters[r];
      rep->resid[side][r] = std::sqrt(std::max(h.rr[r], 0.0));
      rep->status[side][r] = stt;
    }
    if (stt == -2) result = fail(ctx, HOM_ERR_BREAKDOWN, "non-finite FP64 residual");
    else if (stt == 1 && result == HOM_OK) result = HOM_WARN_NOT_CONVERGED;
  }
  if (result == HOM_ERR_BREAKDOWN) return result;
  if (run.gani) {   // the GaNi fields' energies are those of the Galerkin (double-grid) operator
    KL(launch_project_promote<double>(x64, x64, R, g.d, g.N[1], g.N[2], g.Nh, g.invY, side, st));
    CKS(run.energy(coef64, x64, 1, side));
    return result;
  }
  // a(E_b + x_b, E_a + x_a) = E_a.<A>E_b - <b_a, x_b> - <x_a, r_b> with the final x64 (in the
  // range of Gamma) and its FP64 residual r64 = b - C x64 (Def. upper_lower_bounds, Lemma
  // double-grid: C is the exactly integrated Galerkin operator)
  {
    Prof pr(ctx, "energy", st);
    double* part = run.at<double>(L.epart);
    KLN(launch_energy_identity(b64, x64, r64, R, g.d, g.field, g.Nh, coef64, g.ncomp, g.grid, part, kVecBlocks,
                              part + (size_t)kVecBlocks * 18, kVecBlocks, run.at<double>(L.eout) + side * 9, st), 3);
  }
  return result;
}

hom_status set_device(hom_ctx* ctx) {
  CK(cudaSetDevice(ctx->device));
  return HOM_OK;
}

bool sym_inv_spd(const double* B, int d, double* out) {  // leading dim d
  double A3[9] = {}, I3[9] = {};
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) A3[3 * i + j] = B[d * i + j];
  if (!spd(A3, d)) return false;
  inv3(A3, d, I3);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) out[d * i + j] = I3[3 * i + j];
  return true;
}

// ---------------------------------------------------------------------------------
// batched 2D path
// ---------------------------------------------------------------------------------
struct BatchPlan {
  std::vector<BTask> tasks;
  std::vector<DevIncl> incl;
  std::vector<double2> tw64;
  std::vector<float2> tw32;
  int M0max = 1, M1max = 1, Mmax = 1;
  long long slot_bytes = 0;
  int nslots_max = 0;
  // workspace offsets
  size_t o_tasks, o_incl, o_tw64, o_tw32, o_counter, o_energy, o_iters, o_status, o_resid, o_slots, total;
  size_t in_bytes;    // contiguous H2D region [o_tasks, o_counter)
  size_t out_bytes;   // contiguous D2H region [o_energy, o_slots)
};

int device_sms(int device) {
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n <= 0) n = 152;
  return n;
}

hom_status build_batch(hom_ctx* ctx, int n, const hom_problem* probs, const hom_opts* o, BatchPlan& bp) {
  if (n < 1 || !probs) return fail(ctx, HOM_ERR_INVALID_ARG, "batch needs n >= 1 problems");
  const size_t elem = o->precision == HOM_MIXED ? 8 : 16;
  std::vector<int> Ms;
  auto tw_off = [&](int M) -> int {
    int off = 0;
    for (int m : Ms) {
      if (m == M) return off;
      off += m;
    }
    Ms.push_back(M);
    std::vector<double2> w64;
    std::vector<float2> w32;
    twiddles(M, w64, w32);
    bp.tw64.insert(bp.tw64.end(), w64.begin(), w64.end());
    bp.tw32.insert(bp.tw32.end(), w32.begin(), w32.end());
    return off;
  };
  for (int i = 0; i < n; ++i) {
    Geometry g;
    CKS(build_geometry(ctx, &probs[i], g, true));
    if (g.d != 2) return fail(ctx, HOM_ERR_INVALID_ARG, "hom_bounds_batched handles two-dimensional cells (d = 2)");
    if (g.even) return fail(ctx, HOM_ERR_INVALID_ARG, "hom_bounds_batched handles odd grids");
    if (!g.bitmap.empty()) return fail(ctx, HOM_ERR_INVALID_ARG, "hom_bounds_batched takes inclusion cells, not images");
    double A0f[9], B0[9] = {};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) A0f[3 * a + b] = g.A0[a][b];
    inv3(A0f, 2, B0);
    for (int side = 0; side < 2; ++side) {
      BTask t;
      memset(&t, 0, sizeof t);
      t.prob = i;
      t.side = side;
      t.ncomp = g.ncomp;
      t.nincl = (int)g.incl.size();
      t.incl_off = (int)bp.incl.size();
      t.N0 = g.N[0];
      t.N1 = g.N[1];
      t.M0 = g.M[0];
      t.M1 = g.M[1];
      t.Nh = g.Nh;
      t.Nxs = g.Nxs;
      t.invY[0] = g.invY[0];
      t.invY[1] = g.invY[1];
      t.invVol = 1.0 / (g.Y[0] * g.Y[1]);
      pack_sym(side == 0 ? A0f : B0, 2, g.ncomp, t.C0p);
      t.tw0 = tw_off(g.M[0]);
      t.tw1 = tw_off(g.M[1]);
      t.plan0 = g.plan[0];
      t.plan1 = g.plan[1];
      for (size_t j = 0; j < g.incl.size(); ++j) {
        const hom_inclusion& I = g.incl[j];
        DevIncl D;
        memset(&D, 0, sizeof D);
        D.shape = I.shape == HOM_BOX ? 0 : 1;
        D.same_as_prev = (j > 0 && I.shape == HOM_BALL && g.incl[j - 1].shape == HOM_BALL &&
                          I.size[0] == g.incl[j - 1].size[0]) ? 1 : 0;
        for (int a = 0; a < 3; ++a) {
          D.c[a] = I.center[a];
          D.h[a] = I.size[a];
        }
        double dA[9] = {};
        if (side == 0) {
          for (int k = 0; k < 9; ++k) dA[k] = I.A[k] - A0f[k];
        } else {
          double Bi[9] = {};
          inv3(I.A, 2, Bi);
          for (int k = 0; k < 9; ++k) dA[k] = Bi[k] - B0[k];
        }
        pack_sym(dA, 2, g.ncomp, D.dA);
        bp.incl.push_back(D);
      }
      bp.M0max = std::max(bp.M0max, t.M0);
      bp.M1max = std::max(bp.M1max, t.M1);
      bp.slot_bytes = std::max(bp.slot_bytes, batch_slot_bytes(t, (int)elem));
      bp.tasks.push_back(t);
    }
  }
  bp.Mmax = std::max(bp.M0max, bp.M1max);
  if (bp.Mmax > 2047) return fail(ctx, HOM_ERR_INVALID_ARG, "batched grids are limited to N <= 1024");
  // largest grids first (longest tasks start first)
  std::stable_sort(bp.tasks.begin(), bp.tasks.end(), [](const BTask& a, const BTask& b) {
    return (long long)a.M0 * a.M1 > (long long)b.M0 * b.M1;
  });
  if (bp.incl.empty()) bp.incl.resize(1);
  const int nt = (int)bp.tasks.size();
  bp.nslots_max = std::min(nt, device_sms(ctx->device) * 4);
  Layout L{};
  bp.o_tasks = L.take(bp.tasks.size() * sizeof(BTask));
  bp.o_incl = L.take(bp.incl.size() * sizeof(DevIncl));
  bp.o_tw64 = L.take(bp.tw64.size() * sizeof(double2));
  bp.o_tw32 = L.take(bp.tw32.size() * sizeof(float2));
  bp.o_counter = L.take(2 * sizeof(int));
  bp.in_bytes = bp.o_counter - bp.o_tasks;
  bp.o_energy = L.take((size_t)nt * 4 * sizeof(double));
  bp.o_iters = L.take((size_t)nt * 2 * sizeof(int));
  bp.o_status = L.take((size_t)nt * 2 * sizeof(int));
  bp.o_resid = L.take((size_t)nt * 2 * sizeof(double));
  bp.o_slots = L.take(0);
  bp.out_bytes = bp.o_slots - bp.o_energy;
  L.off = bp.o_slots + (size_t)bp.nslots_max * (size_t)bp.slot_bytes;
  bp.total = L.off;
  return HOM_OK;
}

hom_status ensure_pinned(hom_ctx* ctx, unsigned char** buf, size_t* have, size_t need) {
  if (*have >= need) return HOM_OK;
  if (*buf) cudaFreeHost(*buf);
  *buf = nullptr;
  *have = 0;
  CK(cudaMallocHost((void**)buf, need));
  *have = need;
  return HOM_OK;
}

}  // namespace

// =====================================================================================
// C ABI
// =====================================================================================
extern "C" {

const char* hom_version(void) { return "homb 0.1"; }

hom_status hom_create(hom_ctx** out, int device) {
  if (!out) return HOM_ERR_INVALID_ARG;
  static std::atomic<int> created{0};
  hom_ctx* ctx = new hom_ctx();
  ctx->device = device;
  ctx->gemm_slot = created.fetch_add(1) % kGemmFlagSlots;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->host_cg, sizeof(CgScalars));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->host_e, 64 * sizeof(double));
  if (e != cudaSuccess) {
    delete ctx;
    *out = nullptr;
    return HOM_ERR_CUDA;
  }
  *out = ctx;
  return HOM_OK;
}

hom_status hom_destroy(hom_ctx* ctx) {
  if (!ctx) return HOM_OK;
  cudaSetDevice(ctx->device);
  for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
  if (ctx->host_cg) cudaFreeHost(ctx->host_cg);
  if (ctx->host_e) cudaFreeHost(ctx->host_e);
  if (ctx->pin_in) cudaFreeHost(ctx->pin_in);
  if (ctx->pin_out) cudaFreeHost(ctx->pin_out);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  for (auto& gr : ctx->cg_graphs) {
    cudaGraphExecDestroy(gr.exec);
    for (cudaEvent_t ev : gr.events) cudaEventDestroy(ev);
  }
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  delete ctx;
  return HOM_OK;
}

const char* hom_last_error(const hom_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

hom_status hom_problem_info(hom_ctx* ctx, const hom_problem* prob, int32_t* ncomp, int32_t M[3],
                            int64_t* field_elems, int64_t* grid_elems) {
  if (!ctx) return HOM_ERR_INVALID_ARG;
  Geometry g;
  CKS(build_geometry(ctx, prob, g));
  if (ncomp) *ncomp = g.ncomp;
  if (M)
    for (int a = 0; a < 3; ++a) M[a] = g.M[a];
  if (field_elems) *field_elems = g.field;
  if (grid_elems) *grid_elems = g.grid;
  return HOM_OK;
}

// the N-grid geometry of GaNi: transform lengths M = N, coefficient sampled on the N grid
// GaNi geometry: the N grid itself when every N_a factors into radices 2, 3, 5, 7, 11, 13;
// else the (smooth) double grid of g with the GaNi matrix built as a periodized spectrum
Geometry gani_geometry(const Geometry& g) {
  Geometry n = g;
  bool fast = true;
  for (int a = 0; a < g.d; ++a) {
    int r = g.N[a];
    for (int p : {2, 3, 5, 7, 11, 13})
      while (r % p == 0) r /= p;
    fast = fast && r == 1;
  }
  if (!fast) {
    n.gani_dg = true;
    for (int a = 0; a < 3; ++a) make_plan(a < g.d ? g.N[a] : 1, n.nplan[a]);
    return n;
  }
  for (int a = 0; a < 3; ++a) n.M[a] = a < g.d ? g.N[a] : 1;
  n.Nxs = (n.M[0] + 1) / 2;
  n.planes = (long long)n.M[1] * n.M[2];
  n.grid = n.planes * n.M[0];
  n.spec = n.planes * n.Nxs;
  for (int a = 0; a < 3; ++a) make_plan(n.M[a], n.plan[a]);
  return n;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Every shared-memory pass of the FP64 pipeline holds at least one pencil (the y and z
// transforms; the last pass with its d components) or one plane of rows (the x pass: one
// c2r row, d operator rows, and the energy pass's d^2 rows). Checked before any work, so
// that an oversize grid fails at once instead of at its first energy evaluation. The FP32
// passes of the mixed path are half the size and fit whenever these do.
static hom_status check_pass_fit(hom_ctx* ctx, const Geometry& g, bool energy) {
  bool ok = xpass_yb<double>(g.M[0], 1, 1) >= 1 && xpass_yb<double>(g.M[0], g.d, 1) >= 1 &&
            pencil_xc<double>(g.M[g.d - 1], 1, g.d) >= 1;
  if (energy) ok = ok && xpass_yb<double>(g.M[0], g.d * g.d, 1) >= 1;
  for (int a = 1; a < g.d; ++a) ok = ok && pencil_xc<double>(g.M[a], 1, 1) >= 1;
  if (!ok)
    return fail(ctx, HOM_ERR_INVALID_ARG,
                "grid too large for the shared-memory FFT (a pass cannot hold one pencil or plane of rows)");
  return HOM_OK;
}

// the learned warm start (defined with the network entry points below)
static hom_status net_cfg(hom_ctx* ctx, const hom_net_config* c, NetConfig* out);
static size_t net_ws_bytes(const NetConfig& c, int batch);
static hom_status net_prepare(hom_ctx* ctx, const NetConfig& c, int batch, void* d_ws, size_t ws_bytes,
                              cudaStream_t st, float** bases, float** rest);
static hom_status gemm_begin(hom_ctx* ctx, cudaStream_t st);
static hom_status gemm_end(hom_ctx* ctx, cudaStream_t st);
static size_t features_stage_bytes(int n, size_t n_incl);
static hom_status features_impl(hom_ctx* ctx, int32_t n, const hom_problem* probs, float* d_features, void* d_ws,
                                size_t ws_bytes, cudaStream_t st);

// Workspace region of the learned start, after the solver's own layout: the network
// parameters, the features of every cell and the prediction of one chunk of cells on the N
// grid, the half-spectrum start fields [cell][side][rhs][comp][(z)][y][kx], the feature
// staging and the network's own workspace (DFT bases and activations for one chunk).
struct LearnedPlan {
  NetConfig c{};
  long long n_params = 0;
  int n = 1, chunk = 1;   // cells, cells per network forward
  int x0_elem = 16;       // bytes per complex entry of the start fields
  size_t params = 0, feat = 0, pred = 0, x0 = 0, stage = 0, stage_bytes = 0, netws = 0, net_bytes = 0, end = 0;
};

// Network activations of one forward call are bounded by this many bytes: a batch of
// cells is run through the network in chunks of as many cells as fit.
constexpr size_t kNetChunkBytes = size_t(512) << 20;

// n cells sharing the geometry g's grid (the caller checks that), n_incl inclusions in all,
// start fields of x0_elem bytes per complex entry.
static hom_status plan_learned(hom_ctx* ctx, const Geometry& g, const hom_opts* o, size_t base, LearnedPlan& lp,
                               int n = 1, size_t n_incl = 0, int x0_elem = 16) {
  if (o->warm_start != 0 && o->warm_start != 1) return fail(ctx, HOM_ERR_INVALID_ARG, "warm_start must be 0 or 1");
  if (o->warm_start == 0) return HOM_OK;
  if (!o->net) return fail(ctx, HOM_ERR_INVALID_ARG, "warm_start = 1 needs a network (hom_net_load)");
  if (o->discretization != 0) return fail(ctx, HOM_ERR_INVALID_ARG, "the learned start is for the Galerkin discretization");
  if (!g.bitmap.empty()) return fail(ctx, HOM_ERR_INVALID_ARG, "the learned start takes inclusion cells, not images");
  for (int a = 1; a < g.d; ++a)
    if (g.N[a] != g.N[0]) return fail(ctx, HOM_ERR_INVALID_ARG, "the learned start needs one N on every axis");
  hom_net_config hc = o->net->cfg;
  hc.N = g.N[0];
  CKS(net_cfg(ctx, &hc, &lp.c));
  if (lp.c.d != g.d || lp.c.cin != 1 || lp.c.cout != 2 * g.d * g.d)
    return fail(ctx, HOM_ERR_INVALID_ARG, "the network's dimension / channels do not fit this cell");
  lp.n_params = net_offsets(lp.c).total;
  if ((long long)o->net->params.size() != lp.n_params)
    return fail(ctx, HOM_ERR_INVALID_ARG, "network parameter count does not match its config");
  const long long pts = (long long)g.N[0] * g.N[1] * g.N[2];
  lp.n = n;
  lp.x0_elem = x0_elem;
  lp.chunk = 1;
  if (ctx->net_chunk > 0) lp.chunk = std::min(n, ctx->net_chunk);
  else
    while (lp.chunk < n &&
           net_ws_bytes(lp.c, lp.chunk + 1) + (size_t)(lp.chunk + 1) * pts * lp.c.cout * 4 <= kNetChunkBytes)
      ++lp.chunk;
  size_t off = align256(base);
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align256(off + bytes);
    return at;
  };
  lp.params = take((size_t)lp.n_params * 4);
  lp.feat = take((size_t)n * pts * 4);
  lp.pred = take((size_t)lp.chunk * pts * lp.c.cout * 4);
  lp.x0 = take((size_t)n * 2 * g.d * g.d * g.field * x0_elem);
  lp.stage_bytes = features_stage_bytes(n, n == 1 ? g.incl.size() : n_incl);
  lp.stage = take(lp.stage_bytes);
  lp.net_bytes = net_ws_bytes(lp.c, lp.chunk);
  lp.netws = take(lp.net_bytes);
  lp.end = off;
  return HOM_OK;
}

// The learned start of lp.n cells into lp.x0 ([cell][side][rhs][comp] half spectra, FP64
// when lp.x0_elem is 16, else FP32): features, the network on the cells' grid in chunks of
// lp.chunk cells, half spectra of its outputs. The solver projects and scales them before CG.
static hom_status learned_start(hom_ctx* ctx, const hom_problem* prob, const hom_opts* o, const LearnedPlan& lp,
                                unsigned char* ws, cudaStream_t st) {
  float* params = reinterpret_cast<float*>(ws + lp.params);
  // still valid only if no call used the workspace otherwise since (every such call
  // changes or clears the table key)
  if (ctx->net_params_id != o->net->id || ctx->net_params_at != params || ctx->tables_key.empty() ||
      ctx->tables_key != ctx->net_params_tables) {
    CK(h2d_copy(ctx, params, o->net->params.data(), (size_t)lp.n_params * 4, st));
    ctx->net_params_id = o->net->id;
    ctx->net_params_at = params;
  }
  float* feat = reinterpret_cast<float*>(ws + lp.feat);
  float* pred = reinterpret_cast<float*>(ws + lp.pred);
  CKS(features_impl(ctx, lp.n, prob, feat, ws + lp.stage, lp.stage_bytes, st));
  float *bases, *rest;
  CKS(net_prepare(ctx, lp.c, lp.chunk, ws + lp.netws, lp.net_bytes, st, &bases, &rest));
  const long long pts = (long long)lp.c.N * lp.c.N * (lp.c.d == 3 ? lp.c.N : 1);
  const long long half = (long long)(lp.c.N + 1) / 2 * lp.c.N * (lp.c.d == 3 ? lp.c.N : 1);
  CKS(gemm_begin(ctx, st));
  for (int c0 = 0; c0 < lp.n; c0 += lp.chunk) {
    const int nb = std::min(lp.chunk, lp.n - c0);
    KL(net_forward(lp.c, params, bases, nb, feat + (size_t)c0 * pts, pred, rest, 0, st));
    KL(grid_to_half(lp.c.d, lp.c.N, nb, lp.c.cout, pred, ws + lp.x0 + (size_t)c0 * lp.c.cout * half * lp.x0_elem,
                    lp.x0_elem == 16 ? 1 : 0, st));
  }
  CKS(gemm_end(ctx, st));
  return HOM_OK;
}

hom_status hom_workspace_size(hom_ctx* ctx, const hom_problem* prob, const hom_opts* opts,
                              size_t* bytes) {
  if (!ctx || !opts || !bytes) return fail(ctx, HOM_ERR_INVALID_ARG, "NULL argument");
  Geometry g;
  CKS(build_geometry(ctx, prob, g, true));
  CKS(check_pass_fit(ctx, g, true));
  if (opts->discretization == 1) CKS(check_pass_fit(ctx, gani_geometry(g), false));
  const size_t elem = opts->precision == HOM_MIXED ? 8 : 16;
  *bytes = make_layout(g, g.d, elem, 0).total;
  if (opts->discretization == 1) *bytes = align256(*bytes) + make_layout(gani_geometry(g), g.d, elem, 0).total;
  LearnedPlan lp;
  CKS(plan_learned(ctx, g, opts, *bytes, lp));
  if (opts->warm_start == 1) *bytes = lp.end;
  return HOM_OK;
}

hom_status hom_step_workspace_size(hom_ctx* ctx, const hom_problem* prob, int32_t nrhs,
                                   size_t* bytes) {
  if (!ctx || !bytes || nrhs < 1 || nrhs > 3) return fail(ctx, HOM_ERR_INVALID_ARG, "bad argument");
  Geometry g;
  CKS(build_geometry(ctx, prob, g));
  if (nrhs > g.d) return fail(ctx, HOM_ERR_INVALID_ARG, "nrhs > d");
  *bytes = make_layout(g, nrhs, 16, 1).total;
  return HOM_OK;
}

static hom_status bounds_impl(hom_ctx* ctx, const hom_problem* prob, const hom_opts* opts, void* d_ws,
                              size_t ws_bytes, void* stream, double* upper, double* lower, double* mean,
                              double* D, hom_report* rep, const hom_field_io* io) {
  if (!ctx || !opts) return fail(ctx, HOM_ERR_INVALID_ARG, "NULL argument");
  const auto t0 = std::chrono::steady_clock::now();
  ctx->err.clear();
  ctx->launches = ctx->h2d = ctx->d2h = 0;
  CKS(set_device(ctx));
  Geometry g;
  CKS(build_geometry(ctx, prob, g, true));
  if (opts->precision != HOM_FP64 && opts->precision != HOM_MIXED)
    return fail(ctx, HOM_ERR_INVALID_ARG, "precision must be HOM_FP64 or HOM_MIXED");
  const size_t elem = opts->precision == HOM_MIXED ? 8 : 16;
  if (opts->discretization != 0 && opts->discretization != 1)
    return fail(ctx, HOM_ERR_INVALID_ARG, "discretization must be 0 (Ga) or 1 (GaNi)");
  const bool gani = opts->discretization == 1;
  if (gani && io && (io->d_x0 || io->d_fields))
    return fail(ctx, HOM_ERR_INVALID_ARG, "starting / output fields are for the Galerkin discretization");
  CKS(check_pass_fit(ctx, g, true));
  if (gani) CKS(check_pass_fit(ctx, gani_geometry(g), false));
  Runner run{ctx, g, make_layout(g, g.d, elem, 0), static_cast<unsigned char*>(d_ws),
             static_cast<cudaStream_t>(stream), g.d};
  const Geometry gn = gani ? gani_geometry(g) : g;
  const size_t gani_off = align256(run.L.total);
  Runner rn{ctx, gn, gani ? make_layout(gn, g.d, elem, 0) : Layout{}, static_cast<unsigned char*>(d_ws) + gani_off,
            static_cast<cudaStream_t>(stream), g.d};
  rn.gani = true;
  size_t need = gani ? gani_off + rn.L.total : run.L.total;
  LearnedPlan lp;
  CKS(plan_learned(ctx, g, opts, need, lp));
  const bool learned = opts->warm_start == 1;
  if (learned && io && io->d_x0) return fail(ctx, HOM_ERR_INVALID_ARG, "give either starting fields or warm_start");
  if (learned) need = lp.end;
  if (!d_ws || ws_bytes < need) return fail(ctx, HOM_ERR_WORKSPACE, "workspace too small");
  if (reinterpret_cast<uintptr_t>(d_ws) % 256) return fail(ctx, HOM_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  if (rep) memset(rep, 0, sizeof *rep);
  hom_field_io io_learned{nullptr, nullptr};
  if (learned) {   // the network's start, before the solver's tables (its bases share the key)
    CKS(learned_start(ctx, prob, opts, lp, static_cast<unsigned char*>(d_ws), run.st));
    io_learned.d_x0 = static_cast<unsigned char*>(d_ws) + lp.x0;
    io_learned.d_fields = io ? io->d_fields : nullptr;
    io = &io_learned;
  }
  CKS(run.upload_tables());
  if (learned) ctx->net_params_tables = ctx->tables_key;
  if (gani) CKS(rn.upload_tables());
  const int sides = opts->sides ? opts->sides : 3;
  int matvecs = 0;
  hom_status worst = HOM_OK;
  bool warm = false;
  for (int side = 0; side < 2; ++side) {
    if (!(sides & (1 << side))) continue;
    if (gani) {
      // the paper's algorithm (Sec. 6.2): GaNi minimisers on the N grid, then their exactly
      // integrated energies on the double grid (Eq. GaNi_bounds)
      double2* x0 = elem == 16 ? rn.at<double2>(rn.L.q) : rn.at<double2>(rn.L.b64);
      if (side == 1 && (sides & 3) == 3 && opts->dual_start == 1) CKS(rn.dual_start(x0, &warm, &matvecs));
      hom_status s = elem == 16 ? rn.solve_side<double>(side, *opts, rep, &matvecs, warm ? x0 : nullptr)
                                : Runner_solve_mixed(rn, side, *opts, rep, &matvecs, warm, false);
      if (s < 0) return s;
      if (s == HOM_WARN_NOT_CONVERGED) worst = s;
      double* coef64 = run.at<double>(run.L.coef64);
      CKS(run.build_coefficient(side, coef64));
      CKS(run.energy(coef64, rn.at<double2>(rn.L.x64), 1, side));
      continue;
    }
    const size_t side_bytes = (size_t)g.d * g.d * g.field * sizeof(double2);
    double2* x0 = elem == 16 ? run.at<double2>(run.L.q) : run.at<double2>(run.L.b64);
    const bool user = io && io->d_x0;
    warm = false;
    if (user) {
      const unsigned char* src = static_cast<const unsigned char*>(io->d_x0) + side * side_bytes;
      if (elem == 16) {
        x0 = reinterpret_cast<double2*>(const_cast<unsigned char*>(src));
      } else {
        CK(cudaMemcpyAsync(x0, src, side_bytes, cudaMemcpyDeviceToDevice, run.st));
      }
      warm = true;
    } else if (side == 1 && (sides & 3) == 3 && opts->dual_start == 1) {
      CKS(run.dual_start(x0, &warm, &matvecs));
    }
    hom_status s = elem == 16 ? run.solve_side<double>(side, *opts, rep, &matvecs, warm ? x0 : nullptr, user)
                              : Runner_solve_mixed(run, side, *opts, rep, &matvecs, warm, user);
    if (s < 0) return s;
    if (s == HOM_WARN_NOT_CONVERGED) worst = s;
    if (io && io->d_fields)   // the re-projected FP64 fields of this side
      CK(cudaMemcpyAsync(static_cast<unsigned char*>(io->d_fields) + side * side_bytes, run.at<double2>(run.L.x64),
                         side_bytes, cudaMemcpyDeviceToDevice, run.st));
  }
  if (gani && rep) {   // the GaNi homogenized matrices A_{H,N}, B_{H,N} (Cor. FD_GaNi)
    CK(d2h_copy(ctx, ctx->host_e, rn.at<double>(rn.L.eout), 18 * sizeof(double), run.st));
    CK(cudaStreamSynchronize(run.st));
    const double invN = 1.0 / (double)gn.grid;
    for (int sd = 0; sd < 2; ++sd)
      for (int i = 0; i < g.d; ++i)
        for (int j = 0; j < g.d; ++j)
          rep->gani[sd][g.d * i + j] =
              0.5 * (ctx->host_e[9 * sd + g.d * i + j] + ctx->host_e[9 * sd + g.d * j + i]) * invN;
  }
  CK(d2h_copy(ctx, ctx->host_e, run.at<double>(run.L.eout), 18 * sizeof(double), run.st));
  CK(cudaStreamSynchronize(run.st));
  const int d = g.d;
  const double invM = 1.0 / (double)g.grid;
  double Au[9] = {}, Bu[9] = {}, Lo[9] = {};
  // the bound matrices are symmetric bilinear forms (Eq. upper_lower_bounds): report the
  // symmetric part of the two energy matrices
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      Au[d * i + j] = 0.5 * (ctx->host_e[d * i + j] + ctx->host_e[d * j + i]) * invM;
      Bu[d * i + j] = 0.5 * (ctx->host_e[9 + d * i + j] + ctx->host_e[9 + d * j + i]) * invM;
    }
  if (sides & 1)
    if (upper) memcpy(upper, Au, sizeof(double) * d * d);
  if (sides & 2) {
    if (!sym_inv_spd(Bu, d, Lo)) return fail(ctx, HOM_ERR_NOT_SPD_RESULT, "dual energy matrix is not SPD");
    if (lower) memcpy(lower, Lo, sizeof(double) * d * d);
  }
  if ((sides & 3) == 3) {
    for (int i = 0; i < d * d; ++i) {
      if (mean) mean[i] = 0.5 * (Au[i] + Lo[i]);
      if (D) D[i] = 0.5 * (Au[i] - Lo[i]);
    }
    if (rep)   // entry intervals of A_H (Lemma bounds, Eqs. estimate_diagonal, estimate_nondiagonal)
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
          const int i = a * d + b;
          if (a == b) {
            rep->elem_lo[i] = Lo[i];
            rep->elem_hi[i] = Au[i];
          } else {
            const double m = 0.5 * (Au[i] + Lo[i]);
            const double r = 0.5 * (Au[a * d + a] - Lo[a * d + a]) + 0.5 * (Au[b * d + b] - Lo[b * d + b]);
            rep->elem_lo[i] = m - r;
            rep->elem_hi[i] = m + r;
          }
        }
  }
  if (rep) {
    rep->launches = ctx->launches;
    rep->h2d_bytes = ctx->h2d;
    rep->d2h_bytes = ctx->d2h;
    rep->matvecs = matvecs;
    rep->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return worst;
}

hom_status hom_bounds(hom_ctx* ctx, const hom_problem* prob, const hom_opts* opts, void* d_ws,
                      size_t ws_bytes, void* stream, double* upper, double* lower, double* mean,
                      double* D, hom_report* rep) {
  return bounds_impl(ctx, prob, opts, d_ws, ws_bytes, stream, upper, lower, mean, D, rep, nullptr);
}

hom_status hom_bounds_io(hom_ctx* ctx, const hom_problem* prob, const hom_opts* opts, void* d_ws,
                         size_t ws_bytes, void* stream, double* upper, double* lower, double* mean,
                         double* D, hom_report* rep, const hom_field_io* io) {
  return bounds_impl(ctx, prob, opts, d_ws, ws_bytes, stream, upper, lower, mean, D, rep, io);
}

hom_status hom_energy_bounds(hom_ctx* ctx, const hom_problem* prob, const hom_opts* opts, void* d_ws,
                             size_t ws_bytes, void* stream, const double* E, double* upper, double* lower,
                             hom_report* rep) {
  if (!ctx || !prob || !opts || !E || !upper || !lower) return fail(ctx, HOM_ERR_INVALID_ARG, "NULL argument");
  if (opts->sides != 0 && opts->sides != 3) return fail(ctx, HOM_ERR_INVALID_ARG, "energy bounds need both sides");
  double Au[9], Lo[9];
  const hom_status s = bounds_impl(ctx, prob, opts, d_ws, ws_bytes, stream, Au, Lo, nullptr, nullptr, rep, nullptr);
  if (s < 0) return s;
  const int d = prob->d;
  double eu = 0.0, el = 0.0;
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      eu += E[a] * Au[d * a + b] * E[b];
      el += E[a] * Lo[d * a + b] * E[b];
    }
  *upper = eu;
  *lower = el;
  return s;
}

// The learned start of a batch, after the batch's own layout: every cell on one square grid,
// start fields in the inner precision (the layout of hom_batch_io.d_x0).
static hom_status plan_learned_batch(hom_ctx* ctx, int n, const hom_problem* probs, const hom_opts* o,
                                     const BatchPlan& bp, LearnedPlan& lp) {
  if (o->warm_start != 1) return plan_learned(ctx, Geometry{}, o, bp.total, lp);
  Geometry g0;
  CKS(build_geometry(ctx, &probs[0], g0, true));
  size_t n_incl = 0;
  for (int i = 0; i < n; ++i) {
    Geometry g;
    CKS(build_geometry(ctx, &probs[i], g, true));
    if (g.N[0] != g0.N[0] || g.N[1] != g0.N[1])
      return fail(ctx, HOM_ERR_INVALID_ARG, "the learned start of a batch needs one grid N for every cell");
    n_incl += g.incl.size();
  }
  return plan_learned(ctx, g0, o, bp.total, lp, n, n_incl, o->precision == HOM_MIXED ? 8 : 16);
}

hom_status hom_batched_workspace_size(hom_ctx* ctx, int32_t n, const hom_problem* probs, const hom_opts* opts,
                                      size_t* bytes) {
  if (!ctx || !opts || !bytes) return fail(ctx, HOM_ERR_INVALID_ARG, "NULL argument");
  BatchPlan bp;
  CKS(build_batch(ctx, n, probs, opts, bp));
  LearnedPlan lp;
  CKS(plan_learned_batch(ctx, n, probs, opts, bp, lp));
  *bytes = opts->warm_start == 1 ? lp.end : bp.total;
  return HOM_OK;
}

hom_status hom_bounds_batched(hom_ctx* ctx, int32_t n, const hom_problem* probs, const hom_opts* opts, void* d_ws,
                              size_t ws_bytes, void* stream, double* upper, double* lower, int32_t* status,
                              int32_t* iters, hom_report* rep, const hom_batch_io* io) {
  if (!ctx || !opts) return fail(ctx, HOM_ERR_INVALID_ARG, "NULL argument");
  const auto t0 = std::chrono::steady_clock::now();
  ctx->err.clear();
  ctx->launches = ctx->h2d = ctx->d2h = 0;
  CKS(set_device(ctx));
  if (opts->precision != HOM_FP64 && opts->precision != HOM_MIXED)
    return fail(ctx, HOM_ERR_INVALID_ARG, "precision must be HOM_FP64 or HOM_MIXED");
  BatchPlan bp;
  CKS(build_batch(ctx, n, probs, opts, bp));
  LearnedPlan lp;
  CKS(plan_learned_batch(ctx, n, probs, opts, bp, lp));
  const bool learned = opts->warm_start == 1;
  if (learned && io && io->d_x0) return fail(ctx, HOM_ERR_INVALID_ARG, "give either starting fields or warm_start");
  if (!d_ws || ws_bytes < (learned ? lp.end : bp.total)) return fail(ctx, HOM_ERR_WORKSPACE, "workspace too small");
  ctx->tables_key.clear();
  ctx->net_bases_ws = nullptr;
  if (reinterpret_cast<uintptr_t>(d_ws) % 256) return fail(ctx, HOM_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  unsigned char* base = static_cast<unsigned char*>(d_ws);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  hom_batch_io io_learned{nullptr, nullptr};
  if (learned) {   // the network's start of every cell, in the layout of hom_batch_io.d_x0
    CKS(learned_start(ctx, probs, opts, lp, base, st));
    io_learned.d_x0 = base + lp.x0;
    io_learned.d_fields = io ? io->d_fields : nullptr;
    io = &io_learned;
  }
  const bool f32 = opts->precision == HOM_MIXED;
  const int nt = (int)bp.tasks.size();
  const bool has_io = io && (io->d_x0 || io->d_fields);
  if (has_io)
    for (const BTask& t : bp.tasks)
      if (t.N0 != bp.tasks[0].N0 || t.N1 != bp.tasks[0].N1)
        return fail(ctx, HOM_ERR_INVALID_ARG, "starting/final field pools need one grid N for the whole batch");
  // stage the tables in pinned memory (a captured graph reads them at replay)
  CKS(ensure_pinned(ctx, &ctx->pin_in, &ctx->pin_in_bytes, bp.in_bytes));
  CKS(ensure_pinned(ctx, &ctx->pin_out, &ctx->pin_out_bytes, bp.out_bytes));
  memset(ctx->pin_in, 0, bp.in_bytes);
  memcpy(ctx->pin_in + (bp.o_tasks - bp.o_tasks), bp.tasks.data(), bp.tasks.size() * sizeof(BTask));
  memcpy(ctx->pin_in + (bp.o_incl - bp.o_tasks), bp.incl.data(), bp.incl.size() * sizeof(DevIncl));
  memcpy(ctx->pin_in + (bp.o_tw64 - bp.o_tasks), bp.tw64.data(), bp.tw64.size() * sizeof(double2));
  memcpy(ctx->pin_in + (bp.o_tw32 - bp.o_tasks), bp.tw32.data(), bp.tw32.size() * sizeof(float2));
  const double tol = opts->tol > 0 ? opts->tol : 1e-8;
  const int sms = device_sms(ctx->device);
  const int elem = f32 ? 8 : 16;
  const int cap_min = 2 * (bp.Mmax + 1);
  // tasks whose larger double-grid extent is at least coopM go to whole clusters
  auto ncoop_for = [&](int cluster, int coopM) {
    if (cluster <= 1) return 0;
    int n_ = 0;
    while (n_ < nt && std::max(bp.tasks[n_].M0, bp.tasks[n_].M1) >= coopM) ++n_;
    return n_;
  };
  auto args_for = [&](int cap, int max_iter, int ncoop) {
    BArgs a{};
    a.tasks = reinterpret_cast<const BTask*>(base + bp.o_tasks);
    a.ntasks = nt;
    a.counter = reinterpret_cast<int*>(base + bp.o_counter);
    a.counter2 = a.counter + 1;
    a.ncoop = ncoop;
    a.incl = reinterpret_cast<const DevIncl*>(base + bp.o_incl);
    a.tw64 = reinterpret_cast<const double2*>(base + bp.o_tw64);
    a.tw32 = reinterpret_cast<const float2*>(base + bp.o_tw32);
    a.slots = base + bp.o_slots;
    a.slot_bytes = bp.slot_bytes;
    a.energy = reinterpret_cast<double*>(base + bp.o_energy);
    a.iters = reinterpret_cast<int*>(base + bp.o_iters);
    a.status = reinterpret_cast<int*>(base + bp.o_status);
    a.resid = reinterpret_cast<double*>(base + bp.o_resid);
    a.tol2 = tol * tol;
    a.max_iter = max_iter;
    a.cap = cap;
    a.M0max = bp.M0max;
    a.M1max = bp.M1max;
    a.x0 = io ? io->d_x0 : nullptr;
    a.fields = io ? io->d_fields : nullptr;
    a.wpass = ctx->batch_wpass;
    return a;
  };
  // CTAs of one launch: as many as fit at once (0 when the cluster shape cannot be placed),
  // at most one per scratch slot, a multiple of the cluster size
  auto grid_for = [&](int cap, int threads, int cluster, size_t* smem) {
    *smem = batch_smem_bytes(bp.M0max, bp.M1max, cap, elem);
    const int mx = f32 ? batch_max_blocks<float>(*smem, threads, cluster)
                       : batch_max_blocks<double>(*smem, threads, cluster);
    const int g_ = std::min(bp.nslots_max, mx);
    return (g_ / cluster) * cluster;
  };
  int launched[6] = {0, 0, 0, 0, 0, 0};   // threads, cap, schedule, cluster, coopM, CTAs
  auto enqueue = [&](int cap, int threads, int cluster, int coopM, int max_iter) -> hom_status {
    size_t smem = 0;
    int grid = grid_for(cap, threads, cluster, &smem);
    if (grid < cluster) {   // the cluster shape does not fit: single CTAs
      cluster = 1;
      grid = grid_for(cap, threads, 1, &smem);
    }
    if (grid < 1) return fail(ctx, HOM_ERR_INVALID_ARG, "batched kernel does not fit on the device");
    CK(h2d_copy(ctx, base + bp.o_tasks, ctx->pin_in, bp.in_bytes, st));
    CK(cudaMemsetAsync(base + bp.o_counter, 0, 2 * sizeof(int), st));
    const BArgs a = args_for(cap, max_iter, ncoop_for(cluster, coopM));
    launched[0] = threads;
    launched[1] = cap;
    launched[3] = cluster;
    launched[4] = cluster > 1 ? coopM : 0;
    launched[5] = grid;
    if (f32) KL(launch_batch<float>(a, grid, smem, threads, cluster, st));
    else KL(launch_batch<double>(a, grid, smem, threads, cluster, st));
    CK(d2h_copy(ctx, ctx->pin_out, base + bp.o_energy, bp.out_bytes, st));
    return HOM_OK;
  };
  // chunk capacity and threads per CTA: autotuned once per (grid extent, precision), or
  // the defaults; a thread count set on the context overrides both
  int cap = std::max(2048, cap_min);
  int threads = 256, sched = 0, cluster = 1, coopM = 0;
  // the radix schedule travels in the staged task table (both axes' plans of every task)
  auto set_sched = [&](int sc) {
    BTask* tk = reinterpret_cast<BTask*>(ctx->pin_in);
    for (long long k = 0; k < nt; ++k) tk[k].plan0.sched = tk[k].plan1.sched = sc;
  };
  const long long tkey = ((long long)bp.Mmax * 4 + (f32 ? 1 : 0)) * 2 + ctx->batch_wpass;
  bool tuned = false;
  for (auto& kv : ctx->tuned_cap)
    if (kv.key == tkey) {
      cap = std::max(kv.cap, cap_min);
      threads = kv.threads;
      sched = kv.sched;
      cluster = kv.cluster;
      coopM = kv.coopM;
      tuned = true;
    }
  if (opts->autotune && !tuned && ctx->batch_threads == 0) {
    // search over (threads per CTA, chunk capacity, radix schedule), each timed on this
    // batch with 3 CG iterations per task after an untimed run of the same configuration
    float best = 1e30f;
    int best_cap = cap, best_threads = threads, best_sched = 0;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int sc : {1, 2})
      for (int th : {256, 512, 1024})
        for (int c : {2048, 4096, 8192}) {
          if (c < cap_min || batch_smem_bytes(bp.M0max, bp.M1max, c, elem) > 200 * 1024) continue;
          set_sched(sc);
          CKS(enqueue(c, th, 1, 0, 3));
          CK(cudaEventRecord(e0, st));
          CKS(enqueue(c, th, 1, 0, 3));
          CK(cudaEventRecord(e1, st));
          CK(cudaEventSynchronize(e1));
          float ms = 0;
          CK(cudaEventElapsedTime(&ms, e0, e1));
          if (ms < best) { best = ms; best_cap = c; best_threads = th; best_sched = sc; }
        }
    cap = best_cap;
    threads = best_threads;
    sched = best_sched;
    set_sched(sched);
    // clusters for the largest cells: timed on whole solves of this batch, since they act
    // on the longest tasks at the end of the launch, which short probes do not see
    const int mtop = std::max(bp.tasks[0].M0, bp.tasks[0].M1);
    int msecond = 0;
    for (const BTask& tk : bp.tasks)
      if (std::max(tk.M0, tk.M1) < mtop) { msecond = std::max(tk.M0, tk.M1); break; }
    best = 1e30f;
    const int solve_iter = opts->max_iter > 0 ? opts->max_iter : 10000;
    struct Cand { int cl, m; };
    std::vector<Cand> cands = {{1, 0}, {2, mtop}, {4, mtop}, {8, mtop}};
    if (msecond > 0) {
      cands.push_back({4, msecond});
      cands.push_back({8, msecond});
    }
    for (const Cand& cd : cands) {
      size_t sm_ = 0;
      if (cd.cl > 1 && grid_for(cap, threads, cd.cl, &sm_) < cd.cl) continue;
      CK(cudaEventRecord(e0, st));
      CKS(enqueue(cap, threads, cd.cl, cd.m, solve_iter));
      CK(cudaEventRecord(e1, st));
      CK(cudaEventSynchronize(e1));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) { best = ms; cluster = cd.cl; coopM = cd.m; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tuned_cap.push_back({tkey, cap, threads, sched, cluster, coopM});
  }
  set_sched(sched);
  if (ctx->batch_threads) threads = ctx->batch_threads;
  if (ctx->batch_cluster) {
    cluster = ctx->batch_cluster;
    coopM = ctx->batch_coopM;
  }
  // with starting fields, max_iter = 0 is taken literally: bounds of the projected starts
  const int max_iter = opts->max_iter > 0 ? opts->max_iter : ((opts->max_iter == 0 && io && io->d_x0) ? 0 : 10000);
  if (opts->graph && st != nullptr) {
    size_t smem = 0;
    const int grid = grid_for(cap, threads, cluster, &smem);
    const std::vector<long long> key = {(long long)threads, (long long)cluster, (long long)coopM,
                                        (long long)(uintptr_t)d_ws, (long long)(uintptr_t)(io ? io->d_x0 : nullptr),
                                        (long long)(uintptr_t)(io ? io->d_fields : nullptr),
                                        (long long)bp.total, nt, grid, (long long)smem, cap,
                                        (long long)f32, max_iter, (long long)(tol * 1e18), (long long)ctx->pin_in_bytes,
                                        (long long)ctx->pin_out_bytes, bp.M0max, bp.M1max, bp.slot_bytes,
                                        (long long)ctx->batch_wpass};
    if (!ctx->graph_exec || ctx->graph_key != key) {
      if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
      if (ctx->graph) cudaGraphDestroy(ctx->graph);
      ctx->graph_exec = nullptr;
      ctx->graph = nullptr;
      CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      const hom_status s = enqueue(cap, threads, cluster, coopM, max_iter);
      cudaGraph_t g = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(st, &g);
      if (s != HOM_OK) return s;
      CK(ee);
      ctx->graph = g;
      CK(cudaGraphInstantiate(&ctx->graph_exec, g, 0));
      ctx->graph_key = key;
      for (int i = 0; i < 6; ++i) ctx->graph_launched[i] = launched[i];
    } else {
      ctx->h2d += bp.in_bytes;
      ctx->d2h += bp.out_bytes;
      ctx->launches += 1;
      for (int i = 0; i < 6; ++i) launched[i] = ctx->graph_launched[i];
    }
    CK(cudaGraphLaunch(ctx->graph_exec, st));
  } else {
    CKS(enqueue(cap, threads, cluster, coopM, max_iter));
  }
  CK(cudaStreamSynchronize(st));
  // results
  const double* E = reinterpret_cast<const double*>(ctx->pin_out);
  const int* IT = reinterpret_cast<const int*>(ctx->pin_out + (bp.o_iters - bp.o_energy));
  const int* ST = reinterpret_cast<const int*>(ctx->pin_out + (bp.o_status - bp.o_energy));
  const double* RS = reinterpret_cast<const double*>(ctx->pin_out + (bp.o_resid - bp.o_energy));
  std::vector<int> task_of(2 * n, -1);
  for (int k = 0; k < nt; ++k) task_of[2 * bp.tasks[k].prob + bp.tasks[k].side] = k;
  hom_status worst = HOM_OK;
  if (rep) memset(rep, 0, sizeof *rep);
  for (int i = 0; i < n; ++i) {
    const int kp = task_of[2 * i], kd = task_of[2 * i + 1];
    double Au[4], Bu[4], Lo[4];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        Au[2 * a + b] = 0.5 * (E[kp * 4 + 2 * a + b] + E[kp * 4 + 2 * b + a]);
        Bu[2 * a + b] = 0.5 * (E[kd * 4 + 2 * a + b] + E[kd * 4 + 2 * b + a]);
      }
    int stt = 0;
    for (int k : {kp, kd})
      for (int r = 0; r < 2; ++r) {
        const int v = ST[k * 2 + r];
        if (v == -2) stt = -2;
        else if (v != 0 && stt == 0) stt = 1;
      }
    if (!sym_inv_spd(Bu, 2, Lo)) {
      stt = -2;
      for (int q = 0; q < 4; ++q) Lo[q] = NAN;
    }
    if (upper) memcpy(upper + 4 * i, Au, sizeof Au);
    if (lower) memcpy(lower + 4 * i, Lo, sizeof Lo);
    if (status) status[i] = stt;
    if (iters)
      for (int side = 0; side < 2; ++side)
        for (int r = 0; r < 2; ++r) iters[4 * i + 2 * side + r] = IT[(side ? kd : kp) * 2 + r];
    if (stt == -2) worst = HOM_ERR_BREAKDOWN;
    else if (stt == 1 && worst == HOM_OK) worst = HOM_WARN_NOT_CONVERGED;
    if (rep)
      for (int side = 0; side < 2; ++side)
        for (int r = 0; r < 2; ++r) {
          const int k = side ? kd : kp;
          rep->iters[side][r] = std::max(rep->iters[side][r], IT[k * 2 + r]);
          rep->resid[side][r] = std::max(rep->resid[side][r], RS[k * 2 + r]);
        }
  }
  if (rep) {
    rep->launches = ctx->launches;
    rep->h2d_bytes = ctx->h2d;
    rep->d2h_bytes = ctx->d2h;
    rep->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    launched[2] = sched == 0 ? (f32 ? 2 : 1) : sched;
    for (int i = 0; i < 6; ++i) rep->batch_config[i] = launched[i];
  }
  if (worst == HOM_ERR_BREAKDOWN) ctx->err = "a batched solve broke down (see status[])";
  return worst == HOM_OK ? HOM_OK : HOM_WARN_NOT_CONVERGED;
}

hom_status hom_coefficient(hom_ctx* ctx, const hom_problem* prob, int32_t side, int32_t precision,
                           void* d_coef, void* d_ws, size_t ws_bytes, void* stream) {
  if (!ctx || !d_coef) return fail(ctx, HOM_ERR_INVALID_ARG, "NULL argument");
  if (side != 0 && side != 1) return fail(ctx, HOM_ERR_INVALID_ARG, "side must be 0 or 1");
  if (precision != HOM_FP64 && precision != HOM_FP32 && precision != HOM_FF)
    return fail(ctx, HOM_ERR_INVALID_ARG, "precision");
  CKS(set_device(ctx));
  Geometry g;
  CKS(build_geometry(ctx, prob, g));
  if (g.even && precision != HOM_FP64) return fail(ctx, HOM_ERR_INVALID_ARG, "even grids run in FP64");
  Runner run{ctx, g, make_layout(g, 1, 16, 1), static_cast<unsigned char*>(d_ws),
             static_cast<cudaStream_t>(stream), 1};
  if (!d_ws || ws_bytes < run.L.total) return fail(ctx, HOM_ERR_WORKSPACE, "workspace too small");
  CKS(run.upload_tables());
  if (precision == HOM_FP64) return run.build_coefficient(side, static_cast<double*>(d_coef));
  // FP32 / float-float: build in FP64 into the buffer the last pass does not read, then round
  double* tmp = run.at<double>(g.d == 3 ? run.L.t2 : run.L.t1);
  CKS(run.build_coefficient(side, tmp));
  if (precision == HOM_FF)
    KL(launch_convert_d2f_ff(tmp, nullptr, static_cast<ffloat*>(d_coef), (long long)g.ncomp * g.grid, run.st));
  else
    KL(launch_convert_d2f(tmp, static_cast<float*>(d_coef), (long long)g.ncomp * g.grid, run.st));
  return HOM_OK;
}

hom_status hom_rhs(hom_ctx* ctx, const hom_problem* prob, int32_t side, int32_t precision,
                   int32_t nrhs, void* d_b, void* d_ws, size_t ws_bytes, void* stream) {
  if (!ctx || !d_b) return fail(ctx, HOM_ERR_INVALID_ARG, "NULL argument");
  if (side != 0 && side != 1) return fail(ctx, HOM_ERR_INVALID_ARG, "side must be 0 or 1");
  if (precision != HOM_FP64 && precision != HOM_FP32) return fail(ctx, HOM_ERR_INVALID_ARG, "precision");
  CKS(set_device(ctx));
  Geometry g;
  CKS(build_geometry(ctx, prob, g));
  if (g.even && precision != HOM_FP64) return fail(ctx, HOM_ERR_INVALID_ARG, "even grids run in FP64");
  if (nrhs < 1 || nrhs > g.d) return fail(ctx, HOM_ERR_INVALID_ARG, "nrhs must be in [1, d]");
  if (!g.bitmap.empty())
    return fail(ctx, HOM_ERR_INVALID_ARG, "hom_rhs: a pixel image has no closed-form right-hand side "
                                          "(apply hom_matvec to the constant field)");
  Runner run{ctx, g, make_layout(g, nrhs, 16, 1), static_cast<unsigned char*>(d_ws),
             static_cast<cudaStream_t>(stream), nrhs};
  if (!d_ws || ws_bytes < run.L.total) return fail(ctx, HOM_ERR_WORKSPACE, "workspace too small");
  CKS(run.upload_tables());
  SpecArgs sa = run.spec_args(side);
  KL(launch_axis_tables(sa.nincl, g.d, g.M, run.L.Mmax, g.invY, sa.incl, run.at<double2>(run.L.phase),
                        run.at<double>(run.L.sinc), run.st));
  if (run.L.radlen > 0) KL(launch_radial_table(sa, run.at<double>(run.L.radtab), run.L.radgroups, run.st));
  const int N3[3] = {g.N[0], g.N[1], g.N[2]};
  if (precision == HOM_FP64)
    KL(launch_rhs<double>(sa, side, nrhs, g.Nh, N3, d_b, run.at<double>(run.L.partial), kVecBlocks, run.st));
  else
    KL(launch_rhs<float>(sa, side, nrhs, g.Nh, N3, d_b, run.at<double>(run.L.partial), kVecBlocks, run.st));
  return HOM_OK;
}

hom_status hom_matvec(hom_ctx* ctx, const hom_problem* prob, int32_t side, int32_t precision,
                      int32_t project, int32_t nrhs, const void* d_coef, const void* d_in, void* d_out,
                      void* d_ws, size_t ws_bytes, void* stream) {
  if (!ctx || !d_coef || !d_in || !d_out) return fail(ctx, HOM_ERR_INVALID_ARG, "NULL argument");
  if (d_in == d_out) return fail(ctx, HOM_ERR_INVALID_ARG, "d_in and d_out must not alias");
  if (side != 0 && side != 1) return fail(ctx, HOM_ERR_INVALID_ARG, "side must be 0 or 1");
  if (precision != HOM_FP64 && precision != HOM_FP32 && precision != HOM_FF)
    return fail(ctx, HOM_ERR_INVALID_ARG, "precision");
  CKS(set_device(ctx));
  Geometry g;
  CKS(build_geometry(ctx, prob, g));
  if (g.even && precision != HOM_FP64) return fail(ctx, HOM_ERR_INVALID_ARG, "even grids run in FP64");
  if (nrhs < 1 || nrhs > g.d) return fail(ctx, HOM_ERR_INVALID_ARG, "nrhs must be in [1, d]");
  Runner run{ctx, g, make_layout(g, nrhs, 16, 1), static_cast<unsigned char*>(d_ws),
             static_cast<cudaStream_t>(stream), nrhs};
  if (!d_ws || ws_bytes < run.L.total) return fail(ctx, HOM_ERR_WORKSPACE, "workspace too small");
  CKS(run.upload_tables());
  const int proj = project ? side + 1 : 0;
  if (precision == HOM_FP64)
    return run.matvec<double>(d_in, d_out, d_coef, proj, nullptr, nullptr, nullptr, 0);
  if (precision == HOM_FF)
    return run.matvec<ffloat>(d_in, d_out, d_coef, proj, nullptr, nullptr, nullptr, 0);
  return run.matvec<float>(d_in, d_out, d_coef, proj, nullptr, nullptr, nullptr, 0);
}

hom_status hom_energy(hom_ctx* ctx, const hom_problem* prob, int32_t nrhs, int32_t add_constant,
                      const void* d_coef, const void* d_x, double* W, void* d_ws, size_t ws_bytes,
                      void* stream) {
  if (!ctx || !d_coef || !d_x || !W) return fail(ctx, HOM_ERR_INVALID_ARG, "NULL argument");
  CKS(set_device(ctx));
  Geometry g;
  CKS(build_geometry(ctx, prob, g));
  if (nrhs < 1 || nrhs > g.d) return fail(ctx, HOM_ERR_INVALID_ARG, "nrhs must be in [1, d]");
  Runner run{ctx, g, make_layout(g, nrhs, 16, 1), static_cast<unsigned char*>(d_ws),
             static_cast<cudaStream_t>(stream), nrhs};
  if (!d_ws || ws_bytes < run.L.total) return fail(ctx, HOM_ERR_WORKSPACE, "workspace too small");
  CKS(run.upload_tables());
  CKS(run.energy(static_cast<const double*>(d_coef), static_cast<const double2*>(d_x), add_constant, 0));
  CK(d2h_copy(ctx, ctx->host_e, run.at<double>(run.L.eout), 9 * sizeof(double), run.st));
  CK(cudaStreamSynchronize(run.st));
  for (int i = 0; i < nrhs * nrhs; ++i) W[i] = ctx->host_e[i] / (double)g.grid;
  return HOM_OK;
}

hom_status hom_fft(hom_ctx* ctx, int32_t M, int32_t precision, int32_t dir, int32_t howmany,
                   const void* d_in, void* d_out, void* d_ws, size_t ws_bytes, void* stream) {
  if (!ctx || !d_in || !d_out || !d_ws) return fail(ctx, HOM_ERR_INVALID_ARG, "NULL argument");
  if (M < 1 || M > 4096) return fail(ctx, HOM_ERR_INVALID_ARG, "M must be in [1, 4096]");
  if (dir != 1 && dir != -1) return fail(ctx, HOM_ERR_INVALID_ARG, "dir must be +1 or -1");
  if (howmany < 0) return fail(ctx, HOM_ERR_INVALID_ARG, "howmany < 0");
  if (precision != HOM_FP64 && precision != HOM_FP32) return fail(ctx, HOM_ERR_INVALID_ARG, "precision");
  if (ws_bytes < (size_t)M * 16) return fail(ctx, HOM_ERR_WORKSPACE, "workspace too small");
  if (howmany == 0) return HOM_OK;
  CKS(set_device(ctx));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<double2> w64;
  std::vector<float2> w32;
  twiddles(M, w64, w32);
  FftPlan plan;
  make_plan(M, plan);
  if (precision == HOM_FP64) {
    CK(cudaMemcpyAsync(d_ws, w64.data(), M * sizeof(double2), cudaMemcpyHostToDevice, st));
    KL(launch_fft_batch<double>(d_in, d_out, M, howmany, dir, d_ws, plan, st));
  } else {
    CK(cudaMemcpyAsync(d_ws, w32.data(), M * sizeof(float2), cudaMemcpyHostToDevice, st));
    KL(launch_fft_batch<float>(d_in, d_out, M, howmany, dir, d_ws, plan, st));
  }
  return HOM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// hom_matvec_noalloc: the operator with library-owned scratch instead of a workspace
// ---------------------------------------------------------------------------------
namespace {
// Scratch of hom_matvec_noalloc, resident on every device that loads the library.
static __device__ __align__(256) unsigned char g_noalloc_scratch[HOM_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[256] = {};   // device address of the array, per device ordinal

// Device address of the scratch on `device` (which must be current). Host code cannot use
// the symbol's name as a device pointer; the runtime gives the address once per device.
hom_status noalloc_scratch(hom_ctx* ctx, int device, void** out) {
  if (device < 0 || device >= 256) return fail(ctx, HOM_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      return fail(ctx, HOM_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") +
                                         cudaGetErrorString(e));
    }
    g_noalloc_ptr[device] = p;
  }
  *out = g_noalloc_ptr[device];
  return HOM_OK;
}
}  // namespace

extern "C" {

hom_status hom_matvec_noalloc(hom_ctx* ctx, const hom_problem* prob, int32_t side, int32_t precision,
                              int32_t project, int32_t nrhs, const void* d_coef, const void* d_in,
                              void* d_out, void* stream) {
  if (!ctx || !d_coef || !d_in || !d_out) return fail(ctx, HOM_ERR_INVALID_ARG, "NULL argument");
  if (d_in == d_out) return fail(ctx, HOM_ERR_INVALID_ARG, "d_in and d_out must not alias");
  if (side != 0 && side != 1) return fail(ctx, HOM_ERR_INVALID_ARG, "side must be 0 or 1");
  if (precision != HOM_FP64 && precision != HOM_FP32) return fail(ctx, HOM_ERR_INVALID_ARG, "precision");
  CKS(set_device(ctx));
  Geometry g;
  CKS(build_geometry(ctx, prob, g));
  if (g.even && precision != HOM_FP64) return fail(ctx, HOM_ERR_INVALID_ARG, "even grids run in FP64");
  if (nrhs < 1 || nrhs > g.d) return fail(ctx, HOM_ERR_INVALID_ARG, "nrhs must be in [1, d]");
  const Layout L = make_layout(g, nrhs, 16, 1);
  if (L.total > (size_t)HOM_NOALLOC_SCRATCH_BYTES) {
    char b[200];
    snprintf(b, sizeof b, "hom_matvec_noalloc: problem needs %zu bytes of scratch, the static scratch holds %u",
             L.total, (unsigned)HOM_NOALLOC_SCRATCH_BYTES);
    return fail(ctx, HOM_ERR_WORKSPACE, b);
  }
  void* scratch = nullptr;
  CKS(noalloc_scratch(ctx, ctx->device, &scratch));
  Runner run{ctx, g, L, static_cast<unsigned char*>(scratch), static_cast<cudaStream_t>(stream), nrhs};
  ctx->tables_key.clear();   // the static scratch is shared by every context: always upload
  CKS(run.upload_tables());
  ctx->tables_key.clear();
  const int proj = project ? side + 1 : 0;
  if (precision == HOM_FP64)
    return run.matvec<double>(d_in, d_out, d_coef, proj, nullptr, nullptr, nullptr, 0);
  return run.matvec<float>(d_in, d_out, d_coef, proj, nullptr, nullptr, nullptr, 0);
}

hom_status hom_set_batch_threads(hom_ctx* ctx, int32_t threads) {
  if (!ctx) return HOM_ERR_INVALID_ARG;
  if (threads != 0 && threads != 256 && threads != 512 && threads != 1024)
    return fail(ctx, HOM_ERR_INVALID_ARG, "batched threads per CTA must be 0, 256, 512 or 1024");
  ctx->batch_threads = threads;
  return HOM_OK;
}

hom_status hom_set_batch_warp_passes(hom_ctx* ctx, int32_t enable) {
  if (!ctx) return HOM_ERR_INVALID_ARG;
  if (enable != 0 && enable != 1) return fail(ctx, HOM_ERR_INVALID_ARG, "warp passes: 0 (off) or 1 (on)");
  ctx->batch_wpass = enable;
  return HOM_OK;
}

hom_status hom_set_batch_cluster(hom_ctx* ctx, int32_t cluster, int32_t coop_min_M) {
  if (!ctx) return HOM_ERR_INVALID_ARG;
  if (cluster != 0 && cluster != 1 && cluster != 2 && cluster != 4 && cluster != 8)
    return fail(ctx, HOM_ERR_INVALID_ARG, "batched cluster size must be 0, 1, 2, 4 or 8");
  ctx->batch_cluster = cluster;
  ctx->batch_coopM = coop_min_M;
  return HOM_OK;
}

hom_status hom_set_slab_pass(hom_ctx* ctx, int32_t enable) {
  if (!ctx) return HOM_ERR_INVALID_ARG;
  if (enable < 0 || (enable > 1 && (enable < 4 || enable > 20 || enable % 4)))
    return fail(ctx, HOM_ERR_INVALID_ARG, "slab pass: 0 (off), 1 (automatic) or 4..20 warps in steps of 4");
  ctx->slab_on = enable != 0;
  ctx->slab_warps = enable > 1 ? enable : 0;
  return HOM_OK;
}

hom_status hom_set_inner_drift(hom_ctx* ctx, double c) {
  if (!ctx) return HOM_ERR_INVALID_ARG;
  if (!(c >= 0.0) || !std::isfinite(c)) return fail(ctx, HOM_ERR_INVALID_ARG, "drift coefficient must be >= 0");
  ctx->inner_drift = c;
  return HOM_OK;
}

hom_status hom_set_refine_arith(hom_ctx* ctx, int32_t mode) {
  if (!ctx) return HOM_ERR_INVALID_ARG;
  if (mode < 0 || mode > 2) return fail(ctx, HOM_ERR_INVALID_ARG, "refinement arithmetic: 0 default, 1 FP64, 2 float-float");
  ctx->refine_arith = mode;
  return HOM_OK;
}

hom_status hom_set_inner_floor(hom_ctx* ctx, double eta) {
  if (!ctx) return HOM_ERR_INVALID_ARG;
  if (!(eta >= 0.0 && eta < 1.0)) return fail(ctx, HOM_ERR_INVALID_ARG, "inner floor must be in [0, 1)");
  ctx->inner_floor = eta;
  return HOM_OK;
}

hom_status hom_set_pipe_passes(hom_ctx* ctx, int32_t enable) {
  if (!ctx) return HOM_ERR_INVALID_ARG;
  if (enable < 0 || enable > 7)
    return fail(ctx, HOM_ERR_INVALID_ARG, "pipelined passes: a mask of 1 (last pass), 2 (z inverse), 4 (wide chunks)");
  ctx->zpipe_mask = enable;
  return HOM_OK;
}

hom_status hom_set_pass_chunks(hom_ctx* ctx, int32_t ypass_pencils, int32_t xpass_planes) {
  if (!ctx) return HOM_ERR_INVALID_ARG;
  if (ypass_pencils < 0 || xpass_planes < 0) return fail(ctx, HOM_ERR_INVALID_ARG, "chunk sizes must be >= 0");
  ctx->ypass_xc = ypass_pencils;
  ctx->xpass_yb = xpass_planes;
  return HOM_OK;
}

hom_status hom_profile_kernel(hom_ctx* ctx, const char* name) {
  if (!ctx) return HOM_ERR_INVALID_ARG;
  ctx->prof_family = name ? name : "";
  ctx->ev_used = 0;
  ctx->graph_prof_ms = 0;
  ctx->graph_prof_n = 0;
  return HOM_OK;
}

hom_status hom_peak_probe(hom_ctx* ctx, int32_t precision, void* stream, double* tflops) {
  if (!ctx || !tflops || (precision != HOM_FP64 && precision != HOM_FP32))
    return fail(ctx, HOM_ERR_INVALID_ARG, "hom_peak_probe: precision HOM_FP64 or HOM_FP32, tflops not NULL");
  CKS(set_device(ctx));
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int fp64 = precision == HOM_FP64;
  // 4 CTAs of 512 threads per SM; FP64 issues about 1/64 of the FP32 rate, so fewer steps
  const int blocks = 4 * device_sms(ctx->device);
  const int iters = fp64 ? 2048 : 65536;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best = 1e30;
  hom_status s = HOM_OK;
  for (int rep = 0; rep < 6 && s == HOM_OK; ++rep) {
    cudaError_t e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = launch_fma_probe(fp64, blocks, iters, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      s = fail(ctx, HOM_ERR_CUDA, std::string("hom_peak_probe: ") + cudaGetErrorString(e));
    } else if (rep > 0) {   // the first launch warms up clocks and caches
      best = std::min(best, (double)ms);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != HOM_OK) return s;
  const double flops = 2.0 * 8.0 * (double)iters * (double)blocks * 512.0;
  *tflops = flops / (best * 1e-3) / 1e12;
  return HOM_OK;
}

hom_status hom_kernel_timing(hom_ctx* ctx, int64_t* launches, double* total_ms) {
  if (!ctx) return HOM_ERR_INVALID_ARG;
  double tot = 0;
  for (size_t i = 0; i + 1 < ctx->ev_used; i += 2) {
    CK(cudaEventSynchronize(ctx->ev[i + 1]));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]));
    tot += ms;
  }
  if (launches) *launches = (int64_t)(ctx->ev_used / 2) + ctx->graph_prof_n;
  if (total_ms) *total_ms = tot + ctx->graph_prof_ms;
  ctx->ev_used = 0;
  ctx->graph_prof_ms = 0;
  ctx->graph_prof_n = 0;
  return HOM_OK;
}


// ---- learned warm start ------------------------------------------------------------
static hom_status net_cfg(hom_ctx* ctx, const hom_net_config* c, NetConfig* out) {
  if (!c) return fail(ctx, HOM_ERR_INVALID_ARG, "NULL config");
  const int d = c->d == 0 ? 2 : c->d;
  if (c->N < 3 || c->N % 2 == 0 || c->N > 255 || c->cin < 1 || c->width < 1 || c->width > 256 || c->modes < 1 ||
      2 * c->modes > c->N || c->layers < 1 || c->layers > 8 || c->proj < 1 || c->cout < 1 || c->cout > c->proj ||
      (d != 2 && d != 3))
    return fail(ctx, HOM_ERR_INVALID_ARG, "invalid network configuration");
  *out = NetConfig{c->N, c->cin, c->width, c->modes, c->layers, c->proj, c->cout, d};
  return HOM_OK;
}

static size_t net_ws_bytes(const NetConfig& c, int batch) {
  return (size_t)(bases_floats(c) + 256 + net_workspace_floats(c, batch)) * sizeof(float) + 1024;
}

// bases at the front of the workspace (256-float aligned), the rest for activations
static hom_status net_prepare(hom_ctx* ctx, const NetConfig& c, int batch, void* d_ws, size_t ws_bytes,
                              cudaStream_t st, float** bases, float** rest) {
  if (!d_ws || ws_bytes < net_ws_bytes(c, batch)) return fail(ctx, HOM_ERR_WORKSPACE, "workspace too small");
  float* b = static_cast<float*>(d_ws);
  ctx->tables_key.clear();
  if (ctx->net_bases_ws != d_ws || ctx->net_bases_N != c.N || ctx->net_bases_modes != c.modes ||
      ctx->net_bases_d != c.d) {
    std::vector<float> hb((size_t)bases_floats(c));
    fill_bases(c, hb.data());
    CK(h2d_copy(ctx, b, hb.data(), hb.size() * sizeof(float), st));
    ctx->net_bases_ws = d_ws;
    ctx->net_bases_N = c.N;
    ctx->net_bases_modes = c.modes;
    ctx->net_bases_d = c.d;
  }
  *bases = b;
  *rest = b + ((bases_floats(c) + 255) / 256) * 256;
  return HOM_OK;
}

// Tensor-core GEMMs of one call: bind this context's timeout flag and clear it on the
// stream; at the end, read it back (stream synchronised) unless the stream is being captured.
static hom_status gemm_begin(hom_ctx* ctx, cudaStream_t st) {
  gemm_set_context(ctx->gemm_slot, ctx->gemm_spin);
  CK(gemm_timeout_clear(ctx->gemm_slot, st));
  return HOM_OK;
}

static hom_status gemm_end(hom_ctx* ctx, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) return HOM_OK;
  int* flag = reinterpret_cast<int*>(ctx->host_e + 63);
  *flag = 0;
  CK(gemm_timeout_read(ctx->gemm_slot, flag, st));
  CK(cudaStreamSynchronize(st));
  if (*flag) return fail(ctx, HOM_ERR_TIMEOUT, "tensor-core GEMM completion wait timed out");
  return HOM_OK;
}

hom_status hom_set_net_chunk(hom_ctx* ctx, int32_t cells) {
  if (!ctx || cells < 0) return fail(ctx, HOM_ERR_INVALID_ARG, "cells must be >= 0");
  ctx->net_chunk = cells;
  return HOM_OK;
}

hom_status hom_set_gemm_spin_limit(hom_ctx* ctx, int64_t polls) {
  if (!ctx || polls < 0) return fail(ctx, HOM_ERR_INVALID_ARG, "polls must be >= 0");
  ctx->gemm_spin = polls;
  return HOM_OK;
}

hom_status hom_net_sizes(hom_ctx* ctx, const hom_net_config* cfg, int32_t batch, int64_t* n_params,
                         size_t* workspace_bytes) {
  NetConfig c;
  CKS(net_cfg(ctx, cfg, &c));
  if (batch < 1) return fail(ctx, HOM_ERR_INVALID_ARG, "batch < 1");
  if (n_params) *n_params = net_offsets(c).total;
  if (workspace_bytes) *workspace_bytes = net_ws_bytes(c, batch);
  return HOM_OK;
}

hom_status hom_net_init(hom_ctx* ctx, const hom_net_config* cfg, uint64_t seed, float* d_params, void* stream) {
  NetConfig c;
  CKS(net_cfg(ctx, cfg, &c));
  CKS(set_device(ctx));
  KL(init_params(c, d_params, seed, static_cast<cudaStream_t>(stream)));
  return HOM_OK;
}

hom_status hom_net_forward(hom_ctx* ctx, const hom_net_config* cfg, const float* d_params, int32_t batch,
                           const float* d_in, float* d_out, void* d_ws, size_t ws_bytes, void* stream) {
  NetConfig c;
  CKS(net_cfg(ctx, cfg, &c));
  if (!d_params || !d_in || !d_out || batch < 1) return fail(ctx, HOM_ERR_INVALID_ARG, "bad argument");
  CKS(set_device(ctx));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float *bases, *rest;
  CKS(net_prepare(ctx, c, batch, d_ws, ws_bytes, st, &bases, &rest));
  CKS(gemm_begin(ctx, st));
  KL(net_forward(c, d_params, bases, batch, d_in, d_out, rest, 0, st));
  return gemm_end(ctx, st);
}

hom_status hom_net_gradient(hom_ctx* ctx, const hom_net_config* cfg, const float* d_params, int32_t batch,
                            const float* d_in, const float* d_target, float* d_grad, float* loss, void* d_ws,
                            size_t ws_bytes, void* stream) {
  NetConfig c;
  CKS(net_cfg(ctx, cfg, &c));
  if (!d_params || !d_in || !d_target || !d_grad || batch < 1) return fail(ctx, HOM_ERR_INVALID_ARG, "bad argument");
  CKS(set_device(ctx));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float *bases, *rest;
  CKS(net_prepare(ctx, c, batch, d_ws, ws_bytes, st, &bases, &rest));
  // the loss scalar lives in the last float of the workspace
  float* dloss = reinterpret_cast<float*>(static_cast<unsigned char*>(d_ws) + ws_bytes) - 1;
  CKS(gemm_begin(ctx, st));
  KL(net_backward(c, d_params, bases, batch, d_in, d_target, d_grad, dloss, rest, st));
  float h = 0.f;
  CK(d2h_copy(ctx, &h, dloss, sizeof(float), st));
  CKS(gemm_end(ctx, st));
  if (loss) *loss = h;
  return HOM_OK;
}

hom_status hom_net_train_step(hom_ctx* ctx, const hom_net_config* cfg, float* d_params, float* d_m, float* d_v,
                              float* d_grad, int32_t step, float lr, int32_t batch, const float* d_in,
                              const float* d_target, float* d_loss, void* d_ws, size_t ws_bytes, void* stream) {
  NetConfig c;
  CKS(net_cfg(ctx, cfg, &c));
  if (!d_params || !d_m || !d_v || !d_grad || !d_in || !d_target || batch < 1 || step < 1)
    return fail(ctx, HOM_ERR_INVALID_ARG, "bad argument");
  CKS(set_device(ctx));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float *bases, *rest;
  CKS(net_prepare(ctx, c, batch, d_ws, ws_bytes, st, &bases, &rest));
  float* dloss = d_loss ? d_loss : reinterpret_cast<float*>(static_cast<unsigned char*>(d_ws) + ws_bytes) - 1;
  CKS(gemm_begin(ctx, st));
  KL(net_backward(c, d_params, bases, batch, d_in, d_target, d_grad, dloss, rest, st));
  KL(adam_step(d_params, d_grad, d_m, d_v, net_offsets(c).total, lr, 0.9f, 0.999f, 1e-8f, step, st));
  return gemm_end(ctx, st);
}

namespace {
struct FeatIncl {
  int shape;
  float c[3], h[3], value;
};
// one thread per grid point x_j = Y j / N of one cell (2D or 3D); strict membership with
// periodic images, later inclusions overwrite earlier ones
__global__ void k_features(int n, int d, int N, const int* offs, const FeatIncl* incl, const float* base_val,
                           const float* Y, float* out) {
  const long long per = d == 3 ? (long long)N * N * N : (long long)N * N;
  const long long total = (long long)n * per;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(t / per);
    long long j = t - (long long)p * per;
    int jx = (int)(j % N);
    j /= N;
    const int jy = (int)(j % N);
    const int jz = (int)(j / N);
    float x[3] = {Y[3 * p] * jx / N, Y[3 * p + 1] * jy / N, d == 3 ? Y[3 * p + 2] * jz / N : 0.f};
    float v = base_val[p];
    for (int k = offs[p]; k < offs[p + 1]; ++k) {
      const FeatIncl& I = incl[k];
      bool in = true;
      float r2 = 0.f;
      for (int a = 0; a < d; ++a) {
        float dx = x[a] - I.c[a];
        dx -= Y[3 * p + a] * rintf(dx / Y[3 * p + a]);
        in = in && fabsf(dx) < 0.5f * I.h[a];
        r2 += dx * dx;
      }
      if (I.shape != 0) in = r2 < I.h[0] * I.h[0];
      if (in) v = I.value;
    }
    out[t] = v;
  }
}
}  // namespace

static size_t features_stage_bytes(int n, size_t n_incl) {
  return 256 + (size_t)(n + 1) * 4 + 256 + std::max<size_t>(n_incl, 1) * sizeof(FeatIncl) + 256 + (size_t)n * 4 +
         256 + (size_t)n * 12 + 256;
}

// log10 of the mean diagonal phase value at the N-grid points of each cell, divided by 3
// (phase values 1e-2 .. 1e3 map to [-2/3, 1]), [n][(N)][N][N]
static hom_status features_impl(hom_ctx* ctx, int32_t n, const hom_problem* probs, float* d_features, void* d_ws,
                                size_t ws_bytes, cudaStream_t st) {
  if (!ctx || n < 1 || !probs || !d_features) return fail(ctx, HOM_ERR_INVALID_ARG, "bad argument");
  std::vector<int> offs(n + 1, 0);
  std::vector<FeatIncl> inc;
  std::vector<float> basev(n), Y(3 * n);
  int N = -1, d = -1;
  for (int i = 0; i < n; ++i) {
    Geometry g;
    CKS(build_geometry(ctx, &probs[i], g));
    if (!g.bitmap.empty()) return fail(ctx, HOM_ERR_INVALID_ARG, "features take inclusion cells, not images");
    if (d >= 0 && g.d != d) return fail(ctx, HOM_ERR_INVALID_ARG, "features need cells of one dimension");
    d = g.d;
    bool cubic = g.N[0] == g.N[1] && (d == 2 || g.N[2] == g.N[0]);
    if (!cubic || (N >= 0 && g.N[0] != N)) return fail(ctx, HOM_ERR_INVALID_ARG, "features need one cubic grid");
    N = g.N[0];
    double tr = 0.0;
    for (int a = 0; a < d; ++a) tr += g.A0[a][a];
    basev[i] = (float)(std::log10(tr / d) / 3.0);
    for (int a = 0; a < 3; ++a) Y[3 * i + a] = a < d ? (float)g.Y[a] : 1.f;
    for (const hom_inclusion& I : g.incl) {
      FeatIncl f;
      f.shape = I.shape == HOM_BOX ? 0 : 1;
      double itr = 0.0;
      for (int a = 0; a < 3; ++a) {
        f.c[a] = a < d ? (float)I.center[a] : 0.f;
        f.h[a] = a < d ? (float)I.size[a] : 0.f;
      }
      for (int a = 0; a < d; ++a) itr += I.A[a * 3 + a];
      f.value = (float)(std::log10(itr / d) / 3.0);
      inc.push_back(f);
    }
    offs[i + 1] = (int)inc.size();
  }
  const size_t need = features_stage_bytes(n, inc.size());
  if (inc.empty()) inc.resize(1);
  if (!d_ws || ws_bytes < need) return fail(ctx, HOM_ERR_WORKSPACE, "workspace too small");
  unsigned char* b = static_cast<unsigned char*>(d_ws);
  size_t off = 0;
  auto put = [&](const void* src, size_t bytes) {
    void* dst = b + off;
    off = (off + bytes + 255) & ~(size_t)255;
    return std::make_pair(dst, bytes);
  };
  auto p_offs = put(offs.data(), offs.size() * 4);
  auto p_inc = put(inc.data(), inc.size() * sizeof(FeatIncl));
  auto p_base = put(basev.data(), basev.size() * 4);
  auto p_Y = put(Y.data(), Y.size() * 4);
  CK(h2d_copy(ctx, p_offs.first, offs.data(), p_offs.second, st));
  CK(h2d_copy(ctx, p_inc.first, inc.data(), p_inc.second, st));
  CK(h2d_copy(ctx, p_base.first, basev.data(), p_base.second, st));
  CK(h2d_copy(ctx, p_Y.first, Y.data(), p_Y.second, st));
  const long long total = (long long)n * N * N * (d == 3 ? N : 1);
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 16);
  k_features<<<blocks, 256, 0, st>>>(n, d, N, static_cast<const int*>(p_offs.first), static_cast<const FeatIncl*>(p_inc.first),
                                     static_cast<const float*>(p_base.first), static_cast<const float*>(p_Y.first),
                                     d_features);
  CK(cudaGetLastError());
  ++ctx->launches;
  // the host vectors must outlive the pageable copies: they are staged before return
  CK(cudaStreamSynchronize(st));
  return HOM_OK;
}

hom_status hom_net_features(hom_ctx* ctx, int32_t n, const hom_problem* probs, float* d_features, void* d_ws,
                            size_t ws_bytes, void* stream) {
  if (!ctx) return HOM_ERR_INVALID_ARG;
  CKS(set_device(ctx));
  return features_impl(ctx, n, probs, d_features, d_ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

static bool half_args_ok(int32_t d, int32_t N, int32_t batch, int32_t ch) {
  return (d == 2 || d == 3) && N >= 1 && N % 2 == 1 && N <= 169 && batch >= 1 && ch >= 1 &&
         (long long)batch * ch * (d == 3 ? N : 1) < 0x7fffffffLL;
}

hom_status hom_grid_to_half(hom_ctx* ctx, int32_t d, int32_t N, int32_t batch, int32_t ch, const float* d_grid,
                            void* d_half, int32_t precision, void* stream) {
  if (!ctx || !half_args_ok(d, N, batch, ch) || !d_grid || !d_half) return fail(ctx, HOM_ERR_INVALID_ARG, "bad argument");
  CKS(set_device(ctx));
  KL(grid_to_half(d, N, batch, ch, d_grid, d_half, precision == HOM_FP64 ? 1 : 0, static_cast<cudaStream_t>(stream)));
  return HOM_OK;
}

hom_status hom_half_to_grid_workspace_size(hom_ctx* ctx, int32_t d, int32_t N, int32_t batch, int32_t ch,
                                           size_t* bytes) {
  if (!ctx || !half_args_ok(d, N, batch, ch) || !bytes) return fail(ctx, HOM_ERR_INVALID_ARG, "bad argument");
  *bytes = d == 3 ? half3d_tmp_bytes(N, batch, ch) : 0;
  return HOM_OK;
}

hom_status hom_half_to_grid(hom_ctx* ctx, int32_t d, int32_t N, int32_t batch, int32_t ch, const void* d_half,
                            float* d_grid, int32_t precision, void* d_ws, size_t ws_bytes, void* stream) {
  if (!ctx || !half_args_ok(d, N, batch, ch) || !d_grid || !d_half) return fail(ctx, HOM_ERR_INVALID_ARG, "bad argument");
  if (d == 3 && (!d_ws || ws_bytes < half3d_tmp_bytes(N, batch, ch)))
    return fail(ctx, HOM_ERR_WORKSPACE, "workspace too small");
  CKS(set_device(ctx));
  KL(half_to_grid(d, N, batch, ch, d_half, d_grid, precision == HOM_FP64 ? 1 : 0, d_ws,
                  static_cast<cudaStream_t>(stream)));
  return HOM_OK;
}

hom_status hom_resample_fields(hom_ctx* ctx, int32_t d, const int32_t N_from[3], const int32_t N_to[3],
                               int64_t count, int32_t precision, const void* d_in, void* d_out, void* stream) {
  if (!ctx || !N_from || !N_to || !d_in || !d_out || count < 1 || (d != 2 && d != 3) ||
      (precision != HOM_FP64 && precision != HOM_FP32))
    return fail(ctx, HOM_ERR_INVALID_ARG, "bad argument");
  long long nf = count, nt = count;
  for (int a = 0; a < d; ++a) {
    if (N_from[a] < 1 || N_to[a] < 1 || N_from[a] > 4096 || N_to[a] > 4096)
      return fail(ctx, HOM_ERR_INVALID_ARG, "grid sizes must be in [1, 4096]");
    nf *= a == 0 ? (N_from[0] + 1) / 2 : N_from[a];
    nt *= a == 0 ? (N_to[0] + 1) / 2 : N_to[a];
  }
  const size_t el = precision == HOM_FP64 ? 16 : 8;
  const char* pi = static_cast<const char*>(d_in);
  const char* po = static_cast<const char*>(d_out);
  if (pi < po + nt * el && po < pi + nf * el) return fail(ctx, HOM_ERR_INVALID_ARG, "d_in and d_out overlap");
  CKS(set_device(ctx));
  const int f[3] = {N_from[0], N_from[1], d == 3 ? N_from[2] : 1};
  const int t[3] = {N_to[0], N_to[1], d == 3 ? N_to[2] : 1};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (precision == HOM_FP64) KL(launch_resample<double>(d_in, d_out, count, d, f, t, st));
  else KL(launch_resample<float>(d_in, d_out, count, d, f, t, st));
  return HOM_OK;
}

hom_status hom_net_normalise_targets(hom_ctx* ctx, int32_t d, int32_t N, int32_t n, float* d_grid,
                                     void* stream) {
  if (!ctx || (d != 2 && d != 3) || N < 1 || n < 1 || !d_grid) return fail(ctx, HOM_ERR_INVALID_ARG, "bad argument");
  CKS(set_device(ctx));
  const long long pts = d == 3 ? (long long)N * N * N : (long long)N * N;
  KL(normalise_groups(d_grid, n, pts, 2 * d * d, d, static_cast<cudaStream_t>(stream)));
  return HOM_OK;
}

static uint64_t fnv1a(const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

static const char kNetMagic[8] = {'H', 'O', 'M', 'B', 'N', 'E', 'T', 1};

hom_status hom_net_save(hom_ctx* ctx, const hom_net_config* cfg, const float* d_params, const char* path,
                        void* stream) {
  NetConfig c;
  CKS(net_cfg(ctx, cfg, &c));
  if (!d_params || !path) return fail(ctx, HOM_ERR_INVALID_ARG, "bad argument");
  CKS(set_device(ctx));
  const long long n = net_offsets(c).total;
  std::vector<float> host((size_t)n);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CK(d2h_copy(ctx, host.data(), d_params, (size_t)n * 4, st));
  CK(cudaStreamSynchronize(st));
  FILE* f = fopen(path, "wb");
  if (!f) return fail(ctx, HOM_ERR_INVALID_ARG, std::string("cannot write ") + path);
  const int32_t version = 1;
  int32_t conf[8] = {cfg->N, cfg->cin, cfg->width, cfg->modes, cfg->layers, cfg->proj, cfg->cout, c.d};
  const int64_t count = n;
  const uint64_t sum = fnv1a(host.data(), host.size() * 4);
  bool ok = fwrite(kNetMagic, 1, 8, f) == 8 && fwrite(&version, 4, 1, f) == 1 && fwrite(conf, 4, 8, f) == 8 &&
            fwrite(&count, 8, 1, f) == 1 && fwrite(host.data(), 4, host.size(), f) == host.size() &&
            fwrite(&sum, 8, 1, f) == 1;
  ok = (fclose(f) == 0) && ok;
  if (!ok) return fail(ctx, HOM_ERR_INVALID_ARG, std::string("write failed: ") + path);
  return HOM_OK;
}

hom_status hom_net_load(hom_ctx* ctx, const char* path, hom_net** out) {
  if (!ctx || !path || !out) return fail(ctx, HOM_ERR_INVALID_ARG, "bad argument");
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return fail(ctx, HOM_ERR_INVALID_ARG, std::string("cannot read ") + path);
  char magic[8];
  int32_t version = 0, conf[8];
  int64_t count = 0;
  uint64_t sum = 0;
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kNetMagic, 8) == 0 && fread(&version, 4, 1, f) == 1 &&
            version == 1 && fread(conf, 4, 8, f) == 8 && fread(&count, 8, 1, f) == 1;
  hom_net_config hc{conf[0], conf[1], conf[2], conf[3], conf[4], conf[5], conf[6], conf[7]};
  NetConfig c{};
  if (ok) {
    if (net_cfg(ctx, &hc, &c) != HOM_OK || count != net_offsets(c).total) ok = false;
  }
  std::vector<float> params;
  if (ok) {
    params.resize((size_t)count);
    ok = fread(params.data(), 4, params.size(), f) == params.size() && fread(&sum, 8, 1, f) == 1 &&
         sum == fnv1a(params.data(), params.size() * 4);
  }
  fclose(f);
  if (!ok) return fail(ctx, HOM_ERR_INVALID_ARG, std::string("not a valid network file: ") + path);
  static std::atomic<unsigned long long> ids{0};
  hom_net* net = new hom_net();
  net->cfg = hc;
  net->params = std::move(params);
  net->id = ++ids;
  *out = net;
  return HOM_OK;
}

hom_status hom_net_free(hom_net* net) {
  delete net;
  return HOM_OK;
}

hom_status hom_net_info(const hom_net* net, hom_net_config* cfg, int64_t* n_params) {
  if (!net) return HOM_ERR_INVALID_ARG;
  if (cfg) *cfg = net->cfg;
  if (n_params) *n_params = (int64_t)net->params.size();
  return HOM_OK;
}

hom_status hom_gemm_bf16(hom_ctx* ctx, int32_t M, int32_t N, int32_t K, const float* d_A, int32_t lda,
                         int32_t transA, const float* d_B, int32_t ldb, int32_t transB, float* d_C, int32_t ldc,
                         float alpha, float beta, void* stream) {
  if (!ctx || M < 0 || N < 0 || K < 0 || !d_A || !d_B || !d_C) return fail(ctx, HOM_ERR_INVALID_ARG, "bad argument");
  CKS(set_device(ctx));
  GemmArgs g;
  g.A = d_A; g.B = d_B; g.C = d_C; g.M = M; g.N = N; g.K = K; g.lda = lda; g.ldb = ldb; g.ldc = ldc;
  g.ta = transA; g.tb = transB; g.sA = g.sB = g.sC = 0; g.batch = 1; g.alpha = alpha; g.beta = beta;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  CKS(gemm_begin(ctx, st));
  KL(gemm_bf16(g, st));
  return gemm_end(ctx, st);
}

}  // extern "C"
