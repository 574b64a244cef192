/*
 * homb.h - C ABI of the GB300 library for guaranteed upper-lower bounds on the
 * homogenized conductivity matrix A_H of a periodic matrix-inclusion composite,
 * computed by the FFT-based Galerkin method with exact (double-grid) integration
 * (J. Vondrejc, J. Zeman, I. Marek, "Guaranteed upper-lower bounds on homogenized
 * properties by FFT-based Galerkin method").
 *
 * The problem statement follows the paper:
 *   cell Y = prod_a (-Y_a/2, Y_a/2), grid N (odd, Eq. N_odd, or general: see
 *   hom_problem.N), coefficient
 *   A(x) = A0 + sum_j f_j(x - x_j) (A_j - A0)            (Eq. A_with_inclusions)
 *   with f_j the indicator of a box (Remark "inclusion") or a ball/disk;
 *   upper bound  A_up[a][b] = a(e_b + e^(b), e_a + e^(a)), e^(a) in E_N minimising
 *   the energy; lower bound inv(B_up) from the dual fields in J_N
 *   (Def. upper_lower_bounds, Eqs. GaNi_bounds / approx_homog_with_error);
 *   the Galerkin fields are found by conjugate gradients (Sec. 6.1) whose matvec
 *   zero-pads to the 2N-1 grid, transforms, multiplies by the double-grid
 *   coefficient A_{2N-1} (Lemma double-grid, Eq. MBA_GA; Lemma
 *   bounds_for_matrix-inclusion) and projects with Gamma^E or Gamma^J (Def. projection).
 *
 * Conventions shared by every entry point
 *   - Every function returns hom_status; no exception crosses the ABI.
 *   - Host inputs are read during the call only; the library keeps no caller pointer.
 *   - Device memory: the library never allocates device memory. Every device buffer
 *     (workspace, fields, coefficients) is owned by the caller (e.g. a torch tensor)
 *     and must stay valid until the work queued on `stream` has finished. Pointers
 *     given as `void* d_...` are device pointers, 256-byte aligned.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     hom_bounds / hom_bounds_batched synchronise `stream` before returning; the
 *     step-level calls (hom_coefficient ... hom_energy) only enqueue work.
 *   - A hom_ctx is bound to one device and is not thread-safe; use one per thread.
 *   - Small constant tables (twiddles, inclusion tables, DFT bases) stay at the front of a
 *     workspace between calls on the same context and are not uploaded again while the
 *     workspace pointer and the problem are unchanged: do not write into a workspace
 *     between library calls (hand the library a workspace it owns for its lifetime).
 *
 * Axis convention: coordinate x_1 (index 0) is the fastest-varying memory axis.
 *
 * Device field layout ("half spectrum"): a set of R vector fields with C = d
 * components each, stored as interleaved complex numbers (double2 for FP64,
 * float2 for FP32), index [r][c][k3][k2][k1] (2D: [r][c][k2][k1]) with
 *   k1 in [0, (N1+1)/2)          (non-negative frequencies only, Hermitian symmetry
 *                                 u(-k) = conj u(k) gives the rest),
 *   k2 in [0, N2), k3 in [0, N3) (FFT order: index i is frequency i for
 *                                 i <= (N-1)/2, else i - N).
 * Coefficient layout: real, [q][j3][j2][j1] on the double grid M = 2N-1, j in [0, M)
 * (grid point x = Y j / M, periodic), q over `ncomp` components: 1 for isotropic
 * phases (a scalar field), else the symmetric tensor packed (11,22,12) in 2D and
 * (11,22,33,23,13,12) in 3D.
 */
#ifndef HOMB_H
#define HOMB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HOM_OK = 0,
  HOM_WARN_NOT_CONVERGED = 1,  /* max_iter reached: the returned bounds are still
                                  guaranteed (any conforming field gives a bound,
                                  Lemma bounds), only looser                      */
  HOM_ERR_INVALID_ARG = -1,    /* N < 1, even N where only odd grids run, a grid
                                  too large for the shared-memory passes, d not
                                  2/3, non-SPD phase, overlapping or oversized
                                  inclusion, NULL pointer, bad sizes              */
  HOM_ERR_BREAKDOWN = -2,      /* CG breakdown: NaN/Inf or p.Cp <= 0              */
  HOM_ERR_CUDA = -3,           /* a CUDA runtime call failed (see hom_last_error) */
  HOM_ERR_WORKSPACE = -4,      /* workspace smaller than hom_workspace_size      */
  HOM_ERR_TIMEOUT = -5,        /* a bounded device wait gave up (the tensor-core
                                  GEMM's completion barrier); the context stays
                                  usable                                          */
  HOM_ERR_NOT_SPD_RESULT = -6  /* dual energy matrix not invertible              */
} hom_status;

typedef enum { HOM_BOX = 0, HOM_BALL = 1 /* disk when d == 2 */ } hom_shape;
typedef enum { HOM_FP64 = 0, HOM_MIXED = 1 /* FP32 inner CG, FP64 scalars/bounds */,
               HOM_FP32 = 2 /* step-level calls only */,
               HOM_FF = 3   /* hom_coefficient and hom_matvec only: float-float arithmetic
                               (pairs of FP32, about 48 significant bits) on FP64 fields */
} hom_precision;
typedef enum { HOM_PRIMAL = 0 /* A, Gamma^E: upper bound */,
               HOM_DUAL = 1   /* A^{-1}, Gamma^J: lower bound */ } hom_side;

typedef struct {
  int32_t shape;       /* hom_shape                                              */
  int32_t reserved;
  double center[3];    /* x_j                                                    */
  double size[3];      /* HOM_BOX: side lengths h (0 < h_a <= Y_a);
                          HOM_BALL: size[0] = radius (2R <= min Y_a)            */
  double A[9];         /* absolute SPD phase tensor, row-major, leading dim 3   */
} hom_inclusion;

typedef struct {
  int32_t d;                   /* 2 or 3                                         */
  int32_t N[3];                /* grid sizes N_a >= 1, a < d. Odd grids (Eq. N_odd)
                                  everywhere; even sizes (general grids, Sec. "Fully
                                  discrete spaces --- general grids") in hom_bounds
                                  (FP64 and mixed) and the FP64 step-level calls: the
                                  conforming spaces E_N, J_N exclude the Nyquist
                                  frequency k_a = -N_a/2 (Def. FD_proj_E), which every
                                  field keeps at zero; the stored x frequencies are
                                  0..(N_1+1)/2-1 in both cases. Ga on an even axis
                                  then equals Ga on N_a - 1; GaNi samples the N_a
                                  points and gives B_{H,N}^-1 <= A_{H,N} (Prop.
                                  FD_even_problem). Sizes: N_a <= 2049. Each FP64
                                  pass keeps one pencil or plane of rows of the
                                  double-grid length M_a in 220 KB of shared memory.
                                  hom_bounds' energy pass holds the d^2 rows of a
                                  plane: N_a <= 1348 in 2D (M = 2695) and 613 in 3D
                                  (M = 1225), checked by hom_workspace_size and
                                  hom_bounds before any work. The step-level operator
                                  (M = 2N - 1, 2 d + 1 pencils in its last pass) takes
                                  N <= 1405 in 2D and 1003 in 3D in FP64. Larger
                                  grids return HOM_ERR_INVALID_ARG.                */
  double Y[3];                 /* cell side lengths Y_a > 0                      */
  double A0[9];                /* matrix phase, SPD, row-major, leading dim 3    */
  int32_t n_incl;              /* number of inclusions (may be 0)                */
  int32_t reserved;
  const hom_inclusion* incl;   /* host array [n_incl]; inclusions must not
                                  overlap (touching is allowed)                 */
  const double* bitmap;        /* optional pixel image of an isotropic scalar
                                  conductivity (A = a I), host array
                                  [P_d]...[P_1] with the x index fastest; pixel
                                  (i_1..i_d) covers prod_a (-Y_a/2 + i_a h_a,
                                  -Y_a/2 + (i_a + 1) h_a), h_a = Y_a / P_a; values
                                  finite and > 0. NULL: the inclusion model above.
                                  With an image, n_incl must be 0 and A0 is unused;
                                  its Fourier coefficients are those of a sum of
                                  pixel boxes (Remark "inclusion"). Read during the
                                  call only.                                     */
  int32_t bitmap_n[3];         /* P_a, a < d (1 for unused axes)                 */
  int32_t closed;               /* GaNi sampling of a grid point exactly on an
                                  inclusion boundary: 0 matrix (strict membership,
                                  the paper's Eq. S, S1), 1 inclusion (Eq. S2). The
                                  Galerkin discretization does not depend on it.  */
  int32_t smooth;              /* pixel images only (else 0): 1 replaces the image by
                                  the paper's local average (Sec. 7.3) before the
                                  coefficient is formed: weight 4/16 for the pixel,
                                  2/16 for each edge neighbour, 1/16 for each corner
                                  neighbour, periodic; a 3D image takes weights
                                  1/2, 1/4, 1/4 along every axis, multiplied. The
                                  primal coefficient is smoothed; the dual side
                                  inverts the smoothed values. Done on the device
                                  when the image is uploaded.                    */
} hom_problem;

/* A trained warm-start network held on the host (config and FP32 parameters); see
 * hom_net_load. */
typedef struct hom_net hom_net;

typedef struct {
  int32_t precision;    /* hom_precision: HOM_FP64 or HOM_MIXED                  */
  int32_t max_iter;     /* per solve; <= 0 selects 10000 (hom_bounds_batched with
                           starting fields takes 0 literally: no CG iteration)   */
  double tol;           /* stop when ||r_i|| <= tol ||E|| (Remark "Convergence
                           criteria", Parseval L2 norm); <= 0 selects 1e-8       */
  int32_t check_every;  /* host polls convergence every k iterations; 0 -> 8     */
  int32_t sides;        /* bit 0: primal (upper), bit 1: dual (lower); 0 -> both */
  int32_t graph;        /* hom_bounds: 0 or 1 replays blocks of check_every CG
                           iterations from captured CUDA graphs, -1 launches every
                           kernel directly; hom_bounds_batched: 1 replays the batch
                           launch as a graph captured on `stream` (non-NULL)     */
  int32_t autotune;     /* hom_bounds_batched: time the shared-memory chunk sizes
                           on this batch once and keep the fastest in the ctx    */
  int32_t dual_start;   /* hom_bounds with both sides: 0 starts the dual CG from
                           zero; 1 starts it from the primal minimisers (Remark
                           "Avoiding the solution of dual formulation", Eq.
                           FD_superposition_odd_A): j0 = Gamma^J[A sum_a E_a
                           (e_a + e^(a))], E = inv(upper) e_b, through the
                           double-grid operator of the primal coefficient. Any
                           start in J_N keeps the lower bound guaranteed.        */
  int32_t discretization; /* hom_bounds: 0 Ga (CG with the exact double-grid operator);
                           1 GaNi, the paper's algorithm (Sec. 6.2): CG on the N grid
                           with the coefficient sampled at the grid points (Def.
                           GaNi; a point on an inclusion boundary belongs to the
                           matrix unless hom_problem.closed), then the double-grid
                           energies of those minimisers give the bounds (Eq.
                           GaNi_bounds). When an N_a has a prime factor above 13 the
                           GaNi matrix is applied on the double grid instead (the
                           same operator, fast FFT lengths). FP64 or mixed; no
                           starting / output fields.                             */
  int32_t warm_start;   /* hom_bounds and hom_bounds_batched, Ga only: 0 starts CG from
                           zero; 1 from the learned start of `net` (no counterpart in the
                           paper's algorithm; any start projected onto E_N / J_N keeps
                           the bounds guaranteed, Lemma bounds): the library samples the
                           cell on its N grid (log10 of the phase value / 3), runs the
                           network (tensor-core GEMMs) on that grid, takes the half
                           spectra of its 2 d^2 output channels (side, rhs, component)
                           and starts each CG from their projection (hom_bounds: block
                           Rayleigh-Ritz; batched: one Rayleigh-Ritz scale per
                           right-hand side). The grid must be cubic (one N on every
                           axis) with 2 modes <= N; in a batch every cell has the same
                           N, and the network runs on chunks of cells (activations of
                           at most 512 MiB a chunk). Not with starting fields.      */
  int32_t reserved;
  const struct hom_net* net; /* warm_start = 1: a network from hom_net_load            */
} hom_opts;

typedef struct {
  int32_t iters[2][3];  /* [side][rhs] CG iterations                             */
  double resid[2][3];   /* [side][rhs] final recursive residual / ||E||          */
  int32_t matvecs;      /* operator applications issued (all rhs together)       */
  int32_t status[2][3]; /* per solve: 0 converged, 1 max_iter or stalled         */
  double ms_total;      /* host wall time of the call                            */
  int64_t launches;     /* CUDA kernels launched by the call                     */
  int64_t h2d_bytes;    /* host->device bytes copied by the call                 */
  int64_t d2h_bytes;    /* device->host bytes copied by the call                 */
  double gani[2][9];    /* hom_bounds with GaNi: the GaNi homogenized matrices
                           A_{H,N} and B_{H,N} (Cor. FD_GaNi), d x d row-major    */
  int32_t batch_config[6]; /* hom_bounds_batched launch: threads per CTA, chunk
                           capacity, radix schedule (1: 5/3, 2: composite), cluster
                           size, smallest cooperative 2N-1, CTAs launched          */
  double elem_lo[9];    /* hom_bounds with both sides: intervals [elem_lo, elem_hi]
                           for each entry of A_H, d x d row-major (Lemma bounds):
                           diagonal [lower_aa, upper_aa] (Eq. estimate_diagonal),
                           off-diagonal mean_ab -+ (D_aa + D_bb) (Eq.
                           estimate_nondiagonal)                                 */
  double elem_hi[9];
} hom_report;

typedef struct hom_ctx hom_ctx;

/* Context bound to `device` (cudaSetDevice is called inside each entry point).
 * Allocates only host memory (a small pinned staging buffer). */
hom_status hom_create(hom_ctx** ctx, int device);
hom_status hom_destroy(hom_ctx* ctx);
/* Last error message of this context (static storage of the context; "" if none). */
const char* hom_last_error(const hom_ctx* ctx);
/* Library version string, e.g. "homb 0.1". */
const char* hom_version(void);

/* Sizes for a problem: ncomp (coefficient components), M[3] (double grid, 1 for
 * unused axes), field_elems = complex elements of ONE component of ONE field in
 * the half-spectrum layout, grid_elems = prod M. Validates the problem. */
hom_status hom_problem_info(hom_ctx* ctx, const hom_problem* prob, int32_t* ncomp,
                            int32_t M[3], int64_t* field_elems, int64_t* grid_elems);

/* Bytes of device workspace hom_bounds needs for this problem and options. */
hom_status hom_workspace_size(hom_ctx* ctx, const hom_problem* prob, const hom_opts* opts,
                              size_t* bytes);

/* Starting fields in / converged fields out for hom_bounds_io (device memory, complex
 * FP64, layout [side 2][rhs d][comp d][Nz][Ny][(N1+1)/2], the half-spectrum layout of
 * the fields with side 0 primal and 1 dual). A start is projected with Gamma (so any
 * array gives a conforming field, Def. FD_projections); each right-hand side of a side then
 * starts from its Galerkin solution in the span of the side's d projected starts (block
 * Rayleigh-Ritz; the per-right-hand-side scaling when they are dependent), which never gives a
 * larger energy error than x = 0; CG then runs from it and the bounds stay guaranteed (Lemma
 * bounds). The batched launch scales each start by its own Rayleigh-Ritz factor. The fields
 * out are the FP64 re-projected CG fields the bounds were evaluated with. Either pointer
 * may be NULL; not with GaNi. */
typedef struct {
  const void* d_x0;
  void* d_fields;
} hom_field_io;

/* Whole pipeline (Algorithm of Sec. 6.2 with the exact double-grid operator in CG):
 * build both double-grid coefficients once, run d primal and d dual CG solves from
 * x0 = 0, re-project the fields in FP64 and evaluate the bound energies exactly on
 * the double grid. Outputs are host arrays, d x d row-major with leading dim d;
 * any of upper/lower/mean/D/rep may be NULL. lower = inv(B_up); mean = (upper +
 * lower)/2; D = (upper - lower)/2 (Eq. approx_homog_with_error). With `sides` not
 * both, the missing outputs are left untouched. */
hom_status hom_bounds(hom_ctx* ctx, const hom_problem* prob, const hom_opts* opts,
                      void* d_workspace, size_t workspace_bytes, void* stream,
                      double* upper, double* lower, double* mean, double* D,
                      hom_report* rep);
/* The energy bounds of one macroscopic field E (Def. upper_lower_bounds: the bound
 * matrices are symmetric bilinear forms): *upper = E . A_up E >= E . A_H E >= E . inv(B_up) E
 * = *lower, with A_up and inv(B_up) those hom_bounds computes for the same problem and
 * options (one full hom_bounds run; E has d entries, host memory). rep may be NULL. */
hom_status hom_energy_bounds(hom_ctx* ctx, const hom_problem* prob, const hom_opts* opts,
                             void* d_workspace, size_t workspace_bytes, void* stream,
                             const double* E, double* upper, double* lower, hom_report* rep);
/* hom_bounds with starting and / or converged fields (hom_field_io; NULL: hom_bounds). */
hom_status hom_bounds_io(hom_ctx* ctx, const hom_problem* prob, const hom_opts* opts,
                         void* d_workspace, size_t workspace_bytes, void* stream,
                         double* upper, double* lower, double* mean, double* D, hom_report* rep,
                         const hom_field_io* io);

/* Batched bounds for n two-dimensional cells of possibly different N, geometry and
 * phases, in ONE persistent kernel launch: each CTA takes (problem, side) tasks from an
 * atomic work queue (largest grids first) and runs the whole pipeline of hom_bounds for
 * its task (coefficient, CG on both right-hand sides with block reductions, FP64
 * re-projection and exact energies). precision HOM_MIXED: FP32 CG vectors and matvecs,
 * FP64 scalars, coefficients, re-projection and energies; HOM_FP64: everything FP64.
 * There is no outer refinement: a mixed solve stops at tol or when FP32 accuracy runs
 * out (status 2), and the bounds stay guaranteed. Outputs (host): upper, lower [n][2][2]
 * row-major, status [n] (worst of the four solves: 0 ok, 1 max_iter/FP32 floor, -2
 * breakdown), iters [n][2][2] (side, rhs; may be NULL), rep aggregated (may be NULL).
 * Returns HOM_WARN_NOT_CONVERGED when any status is not 0. Synchronises `stream`. */
/* Optional device pools of hom_bounds_batched for batches whose cells share one grid N:
 * d_x0 (starting fields) and d_fields (final CG fields), both [n][side][rhs][comp][N][Nh]
 * half spectra in the inner precision (float2 for HOM_MIXED, double2 for HOM_FP64). A
 * starting field is projected with Gamma^E / Gamma^J before use, so any input gives
 * guaranteed bounds (Lemma bounds); CG then runs from it (Remark after Eq.
 * linear_system_dual: iterates stay in E_N / J_N). */
typedef struct {
  const void* d_x0;
  void* d_fields;
} hom_batch_io;

hom_status hom_batched_workspace_size(hom_ctx* ctx, int32_t n, const hom_problem* probs,
                                      const hom_opts* opts, size_t* bytes);
hom_status hom_bounds_batched(hom_ctx* ctx, int32_t n, const hom_problem* probs,
                              const hom_opts* opts, void* d_workspace, size_t workspace_bytes,
                              void* stream, double* upper, double* lower, int32_t* status,
                              int32_t* iters, hom_report* rep, const hom_batch_io* io);

/* ---- learned warm start: a 2D or 3D Fourier-layer network (no counterpart in the paper's
 * algorithm; the paper's guarantee makes any starting field admissible after projection,
 * Lemma bounds and the remark after Eq. linear_system_dual).
 * Layers: lift (cin -> width), `layers` spectral layers keeping kx in [0, modes) and
 * ky (and kz in 3D) in [-modes, modes) with per-mode complex channel mixing plus a 1x1
 * path and GELU, projection width -> proj (GELU) -> cout (cout <= proj). Every product is a
 * BF16 tensor-core GEMM with FP32 accumulation; parameters are FP32 (a flat array, layout
 * fixed by the config; spectral weights [re/im][kz][ky][kx][width][width]). Activations are
 * channels-last [batch][(N)][N][N][ch] FP32. The spectral layers use 1/N^d-normalised
 * inverse transforms, so one set of parameters runs on any grid with 2 modes <= N. The
 * network calls keep the DFT bases at the front of their workspace between calls with the
 * same workspace pointer and grid: do not write into a network workspace between network
 * calls. d = 0 is read as 2.
 * Every call that runs tensor-core GEMMs (hom_net_forward, hom_net_gradient,
 * hom_net_train_step, hom_gemm_bf16) synchronises `stream` before it returns and returns
 * HOM_ERR_TIMEOUT when a GEMM's bounded wait on its completion barrier gave up during the
 * call (the GEMM then skips its result; the context stays usable). The flag is per context
 * (256 slots: a context shares its flag with the one created 256 contexts earlier). Inside
 * a stream capture the flag is not read. */
typedef struct {
  int32_t N, cin, width, modes, layers, proj, cout, d;
} hom_net_config;

/* number of parameters and workspace bytes for `batch` samples */
hom_status hom_net_sizes(hom_ctx* ctx, const hom_net_config* cfg, int32_t batch, int64_t* n_params,
                         size_t* workspace_bytes);
hom_status hom_net_init(hom_ctx* ctx, const hom_net_config* cfg, uint64_t seed, float* d_params,
                        void* stream);
/* the network's output for `batch` inputs; synchronises `stream` (see above). */
hom_status hom_net_forward(hom_ctx* ctx, const hom_net_config* cfg, const float* d_params,
                           int32_t batch, const float* d_in, float* d_out, void* d_workspace,
                           size_t workspace_bytes, void* stream);
/* mean squared error against d_target and its gradient w.r.t. the parameters (d_grad
 * overwritten); *loss (host) receives the loss; synchronises `stream`. */
hom_status hom_net_gradient(hom_ctx* ctx, const hom_net_config* cfg, const float* d_params,
                            int32_t batch, const float* d_in, const float* d_target, float* d_grad,
                            float* loss, void* d_workspace, size_t workspace_bytes, void* stream);
/* one Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected with `step` >= 1) on the
 * gradient of one batch; loss written to *d_loss (device float, may be NULL); synchronises
 * `stream` (see above). */
hom_status hom_net_train_step(hom_ctx* ctx, const hom_net_config* cfg, float* d_params, float* d_m,
                              float* d_v, float* d_grad, int32_t step, float lr, int32_t batch,
                              const float* d_in, const float* d_target, float* d_loss,
                              void* d_workspace, size_t workspace_bytes, void* stream);
/* Training targets on the N grid, [n][(N)][N][N][2 d^2] FP32 (channels (side, rhs,
 * component)): each (side, rhs) group of d channels of each cell scaled in place to unit
 * RMS over its grid points and components (the network learns the shape of each corrector;
 * the solver's Rayleigh-Ritz scaling of the start finds its size). Enqueue only. */
hom_status hom_net_normalise_targets(hom_ctx* ctx, int32_t d, int32_t N, int32_t n, float* d_grid,
                                     void* stream);
/* Network files (no counterpart in the paper): hom_net_save writes the config and the
 * `n_params` FP32 parameters at d_params (device, as hom_net_sizes counts them) to `path`:
 * 8-byte magic "HOMBNET" + version byte 1, int32 version 1, the hom_net_config as 8 int32,
 * int64 parameter count, the parameters (little-endian FP32), a 64-bit FNV-1a checksum of
 * the parameter bytes. Synchronises `stream`. hom_net_load reads such a file into a host
 * object (config + parameters; no device memory), checking the magic, version, config,
 * count and checksum (HOM_ERR_INVALID_ARG otherwise); hom_net_free releases it;
 * hom_net_info returns its config and parameter count. The object is read-only and may be
 * shared by contexts; hom_bounds uploads its parameters into the workspace (once per
 * workspace and network). */
hom_status hom_net_save(hom_ctx* ctx, const hom_net_config* cfg, const float* d_params, const char* path,
                        void* stream);
hom_status hom_net_load(hom_ctx* ctx, const char* path, hom_net** net);
hom_status hom_net_free(hom_net* net);
hom_status hom_net_info(const hom_net* net, hom_net_config* cfg, int64_t* n_params);
/* input features of n inclusion cells (all 2D or all 3D, one cubic grid N) on their N
 * grid: log10 of the mean diagonal phase value at the grid points x_j = Y j / N, divided
 * by 3 (phase values 1e-2 .. 1e3 map to [-2/3, 1]), [n][(N)][N][N][1]; synchronises
 * `stream` (tables staged from host). */
hom_status hom_net_features(hom_ctx* ctx, int32_t n, const hom_problem* probs, float* d_features,
                            void* d_workspace, size_t workspace_bytes, void* stream);
/* real N-grid fields [B][(N)][N][N][ch] <-> half spectra [B][ch][(N)][N][(N+1)/2] (the
 * solver's field layout) with the 1/N^d of Eq. DFT on the forward side; d = 2 or 3, odd
 * N <= 169; precision HOM_FP64 (double2) or HOM_FP32 (float2); sums in FP32 (the fields
 * are network inputs and outputs). The 3D inverse needs a device scratch of
 * hom_half_to_grid_workspace_size bytes (ignored in 2D, may be NULL there); enqueue only. */
hom_status hom_grid_to_half(hom_ctx* ctx, int32_t d, int32_t N, int32_t batch, int32_t ch,
                            const float* d_grid, void* d_half, int32_t precision, void* stream);
hom_status hom_half_to_grid_workspace_size(hom_ctx* ctx, int32_t d, int32_t N, int32_t batch,
                                           int32_t ch, size_t* bytes);
hom_status hom_half_to_grid(hom_ctx* ctx, int32_t d, int32_t N, int32_t batch, int32_t ch,
                            const void* d_half, float* d_grid, int32_t precision,
                            void* d_workspace, size_t workspace_bytes, void* stream);
/* Half-spectrum fields of one grid on another grid of the same dimension: `count` field
 * components [Nz][Ny][(N1+1)/2] (e.g. count = 2 d d for a hom_field_io block) from grid
 * N_from to grid N_to, out(k) = in(k) where N_from holds frequency k (Nyquist rows of even
 * grids excluded) and 0 elsewhere. The coefficients do not depend on the grid (Eq. DFT), so
 * this is the exact prolongation of a coarse trigonometric polynomial (the odd-grid spaces
 * are nested) and the truncation P_N of a fine one. precision HOM_FP64 (double2) or HOM_FP32
 * (float2); d_in and d_out must not overlap; enqueue only. */
hom_status hom_resample_fields(hom_ctx* ctx, int32_t d, const int32_t N_from[3], const int32_t N_to[3],
                               int64_t count, int32_t precision, const void* d_in, void* d_out,
                               void* stream);
/* the tensor-core GEMM: C = alpha op(A) op(B) + beta C (row-major FP32 in memory, BF16
 * products on tcgen05.mma, FP32 accumulation in tensor memory); synchronises `stream` and
 * returns HOM_ERR_TIMEOUT if a completion wait gave up (see above). */
hom_status hom_gemm_bf16(hom_ctx* ctx, int32_t M, int32_t N, int32_t K, const float* d_A, int32_t lda,
                         int32_t transA, const float* d_B, int32_t ldb, int32_t transB, float* d_C,
                         int32_t ldc, float alpha, float beta, void* stream);

/* Step-level entry points (device buffers; enqueue only). Workspace for these is
 * hom_step_workspace_size. */
hom_status hom_step_workspace_size(hom_ctx* ctx, const hom_problem* prob, int32_t nrhs,
                                   size_t* bytes);

/* Double-grid coefficient A_{2N-1}(x_j) = sum_{n in Z_{2N-1}} w^{jn} A_hat(n) (Eq. MBA_GA)
 * of the primal (A) or dual (A^{-1}) side from the closed-form inclusion
 * coefficients (Lemma bounds_for_matrix-inclusion). d_coef: real, coefficient
 * layout above, FP64 (precision HOM_FP64), FP32 (HOM_FP32: computed in FP64,
 * rounded) or float-float (HOM_FF: computed in FP64, each value as two floats hi, lo
 * with hi = fl32(a), lo = fl32(a - hi); 8 bytes a value). */
hom_status hom_coefficient(hom_ctx* ctx, const hom_problem* prob, int32_t side,
                           int32_t precision, void* d_coef, void* d_workspace,
                           size_t workspace_bytes, void* stream);

/* Right-hand sides b_r = -Gamma(k) A_hat(k) e_r, r < nrhs <= d (Eq. linear_system_primal /
 * _dual with E = e_r), in the half-spectrum layout, precision HOM_FP64 or HOM_FP32. */
hom_status hom_rhs(hom_ctx* ctx, const hom_problem* prob, int32_t side, int32_t precision,
                   int32_t nrhs, void* d_b, void* d_workspace, size_t workspace_bytes,
                   void* stream);

/* Galerkin operator on nrhs fields: d_out = Gamma P_N F_M (A_M/|M|) F_M^{-1} Pad(d_in)
 * (project = 1) or without Gamma (project = 0). d_coef from hom_coefficient in the
 * same precision; d_in / d_out half-spectrum fields [nrhs][d]... (must not alias), double2
 * for HOM_FP64 and HOM_FF, float2 for HOM_FP32. HOM_FF (odd grids, not the even-grid
 * path) computes every transform, the coefficient product and Gamma in float-float
 * arithmetic between FP64 input and output: the residual arithmetic of HOM_MIXED's
 * refinement steps (hom_set_refine_arith). */
hom_status hom_matvec(hom_ctx* ctx, const hom_problem* prob, int32_t side, int32_t precision,
                      int32_t project, int32_t nrhs, const void* d_coef, const void* d_in,
                      void* d_out, void* d_workspace, size_t workspace_bytes, void* stream);

/* Energy matrix W[r][s] = a(u_s, u_r) with u_r = e_r + x_r (add_constant = 1) or
 * u_r = x_r (add_constant = 0), evaluated exactly on the double grid
 * (Lemma double-grid): (1/|M|) sum_j u_r(x_j) . A_M(x_j) u_s(x_j). FP64 only;
 * d_x: [nrhs][d] half-spectrum FP64; W: host, nrhs x nrhs row-major. Synchronises
 * `stream`. */
hom_status hom_energy(hom_ctx* ctx, const hom_problem* prob, int32_t nrhs,
                      int32_t add_constant, const void* d_coef, const void* d_x, double* W,
                      void* d_workspace, size_t workspace_bytes, void* stream);

/* Batched 1D FFT of `howmany` contiguous complex sequences of length M <= 4096
 * (any factorisation; radix-3/5/7/11/13 butterflies, generic radix 2 and primes
 * above 13 one output per thread; the double grid only needs odd lengths, images
 * may be even):
 * out[j] = sum_k in[k] exp(dir * 2 pi i j k / M), dir = -1 (forward) or +1
 * (inverse), no normalisation. FP64 (double2) or FP32 (float2). */
hom_status hom_fft(hom_ctx* ctx, int32_t M, int32_t precision, int32_t dir, int32_t howmany,
                   const void* d_in, void* d_out, void* d_workspace, size_t workspace_bytes,
                   void* stream);  /* workspace >= 16*M bytes (twiddle table) */

/* hom_matvec without a caller workspace. The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc (or cannot hand the library a scratch
 * buffer): code whose device memory is owned and capped by another allocator, such as a
 * framework's caching allocator or an application that reserves all device memory up
 * front, and loops that must not allocate because an allocation could block or fail at
 * an unpredictable moment. Instead of a workspace it uses one scratch array that lives
 * in the library itself (HOM_NOALLOC_SCRATCH_BYTES = 32 MiB of device memory, held on
 * every GPU that loads the library until the process exits).
 * Arguments and results are those of hom_matvec without d_workspace/workspace_bytes, for
 * precision HOM_FP64 or HOM_FP32 (HOM_FF is refused with HOM_ERR_INVALID_ARG).
 * - Problems whose scratch (twiddle and inclusion tables plus the two intermediate
 *   double-grid buffers) exceeds the array are rejected with HOM_ERR_WORKSPACE and a
 *   message giving the bytes needed; e.g. the 3D N = 41 cube with 3 fields in FP64 fits.
 * - The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 *   device made current); make that first call before any stream capture.
 * - Every call on a device shares the same array and it keeps the last call's contents;
 *   nothing in it needs to start at zero (every pass writes all it later reads). Calls
 *   whose work can overlap on the GPU (different streams or threads without ordering)
 *   race on the array: serialise them.
 * - Allocates nothing: no cudaMalloc, cudaFree or allocating library routine. */
#define HOM_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
hom_status hom_matvec_noalloc(hom_ctx* ctx, const hom_problem* prob, int32_t side,
                              int32_t precision, int32_t project, int32_t nrhs,
                              const void* d_coef, const void* d_in, void* d_out, void* stream);

/* Tuning: pencils per CTA of the operator's y passes and planes per CTA of its row pass
 * (0: automatic, the shared-memory budget's maximum; larger requests are capped to it). */
hom_status hom_set_pass_chunks(hom_ctx* ctx, int32_t ypass_pencils, int32_t xpass_planes);
/* The 3D operator with an isotropic coefficient and equal x and y transform lengths
 * M = R * R (R in 3, 5, 9, 15) fuses the inverse y transforms, the x row pass and the
 * forward y transforms into one pass over (rhs, component, z) slabs held in shared memory,
 * by persistent CTAs that stage each slab's input with a bulk asynchronous copy issued
 * while the previous slab is still being transformed (enable = 1, the default: warps per
 * CTA chosen from the slab's shared memory; 4..20 in steps of 4 asks for that many warps
 * where they fit). enable = 0 runs them as three separate passes; the results agree to
 * rounding. A staged copy that does not complete within a bounded wait makes hom_bounds
 * return HOM_ERR_TIMEOUT. Applies to later calls on this context. */
hom_status hom_set_slab_pass(hom_ctx* ctx, int32_t enable);
/* The first and last passes of the FP32 3D operator at double-grid length 225 along z
 * (the zero-padded inverse z transform with the CG prologue, and the truncating forward z
 * transform with Gamma and the CG partial sums) can run as persistent CTAs, two per SM, that
 * stage the input of their next chunk of pencils with asynchronous copies while they
 * transform the current one. enable is a mask: 1 the last pass (the default: measured
 * faster), 2 the z inverse (measured slower than the chunked pass: its CG prologue goes
 * through shared memory), 4 with 1: the last pass on chunks of 16 positions (one CTA per SM;
 * measured 5 % slower than 8), 0 neither. The results agree to rounding. Applies to later
 * calls. */
hom_status hom_set_pipe_passes(hom_ctx* ctx, int32_t enable);
/* Target of the FP32 inner solves of HOM_MIXED (no counterpart in the paper: a precision
 * scheme of this library). An inner solve that starts from the FP64 residual r0 stops when its
 * recursive residual is below max(tol/2, tol - c eps_32 |r0|) (and below 1e-5 |r0|, its FP32
 * limit), eps_32 = 2^-24: c bounds how far the recursive residual may drift from the true one,
 * which the FP64 check after the inner solve measures. A larger c costs inner iterations, a
 * smaller one risks another FP64 refinement step; the bounds stay guaranteed either way.
 * c >= 0; c = 0 restores the default, 100. Applies to later calls on this context. */
hom_status hom_set_inner_drift(hom_ctx* ctx, double c);
/* Relative floor eta of the FP32 inner target of HOM_MIXED (a precision scheme of this
 * library): an inner solve that starts from the FP64 residual r0 stops no lower than
 * eta |r0|, the depth to which its FP32 recursive residual is trusted to follow the true
 * one; below that a restart from a fresh FP64 residual takes over. 0 <= eta < 1; 0 restores
 * the default, 1e-5. The bounds stay guaranteed for any eta; it only moves work between inner
 * iterations and FP64 refinement steps. Applies to later calls on this context. */
hom_status hom_set_inner_floor(hom_ctx* ctx, double eta);
/* Arithmetic of the residual b - C x64 that every refinement step of HOM_MIXED evaluates
 * (a precision scheme of this library): mode 1 FP64; mode 2 float-float, i.e. every
 * transform pass in pairs of FP32 numbers (about 48 significant bits, error-free
 * TwoSum / FMA product steps) between the FP64 iterate and the FP64 residual, on the FP32
 * pipes (this GPU issues FP64 at under a sixtieth of the FP32 rate); mode 0, the default:
 * float-float when the solve starts cold (x = 0) and its tolerance is at least 2e-12 |b|
 * (then float-float rounding, about 1e-14 of |C x| ~ |b|, stays below a hundredth of the
 * tolerance), FP64 otherwise. The iterate, the residual, the re-projection and the bound
 * energies stay FP64 in memory either way, so the bounds stay guaranteed; mode 2 at a
 * tolerance near 1e-14 |b| may stop on a stalled refinement (status 1). Applies to later
 * calls on this context. */
hom_status hom_set_refine_arith(hom_ctx* ctx, int32_t mode);

/* Threads per CTA of the persistent batched kernel: 256 (two CTAs per SM), 512 or 1024
 * (one CTA per SM: more threads per cell, fewer cells at a time), or 0 (default: the
 * autotuned choice when hom_opts.autotune is set, else 256). Applies to later
 * hom_bounds_batched calls on this context. */
hom_status hom_set_batch_threads(hom_ctx* ctx, int32_t threads);

/* Thread-block clusters for the largest cells of a batch: the cells whose larger
 * double-grid extent 2N-1 is at least coop_min_M are each worked on by all `cluster` CTAs
 * of a cluster together (splitting every transform pass and reduction over them, with
 * cluster barriers between passes); the other cells take one CTA each. cluster 1 turns
 * this off; 0 (default) uses the autotuned choice when hom_opts.autotune is set, else 1.
 * Results equal the single-CTA ones to rounding (reduction order). Applies to later
 * hom_bounds_batched calls on this context. */
hom_status hom_set_batch_cluster(hom_ctx* ctx, int32_t cluster, int32_t coop_min_M);
/* The CG iterations of HOM_MIXED batches run their transform passes as warp-owned pencils
 * where every double-grid length of the batch's cells is 45, 125, 225 or 405 (N = 23, 63,
 * 113, 203): each warp takes whole columns or row pairs from load to store with no CTA
 * barrier inside a pass (enable = 1, the default); enable = 0 runs the chunked block-level
 * passes. Results agree to rounding. Applies to later hom_bounds_batched calls. */
hom_status hom_set_batch_warp_passes(hom_ctx* ctx, int32_t enable);

/* Kernel timing (CUDA events around each launch of one kernel family on the
 * launching stream). name: "zpass", "ypass", "xpass", "slab", "final", "cg", "coef", or ""
 * to disable. hom_kernel_timing returns launches and total milliseconds since the
 * last hom_profile_kernel call (synchronises the events). Inside the CG iteration
 * graphs of hom_bounds the events are event-record nodes of the graph; each replay
 * of a graph holding them is waited for and its pairs summed before the call goes on. */
/* Test aid for the failure path of the tensor-core GEMM (no counterpart in the paper): the
 * GEMMs of this context's later calls poll their completion barrier at most `polls` times
 * with a non-blocking test before giving up (0 restores the default, about 4 M blocking
 * polls). A small value makes the wait give up at once: the GEMM then records the timeout,
 * drains its committed MMAs with the default bound, frees its tensor memory and returns, and
 * the call returns HOM_ERR_TIMEOUT. */
hom_status hom_set_gemm_spin_limit(hom_ctx* ctx, int64_t polls);
/* The learned start of hom_bounds_batched runs the network on chunks of at most `cells`
 * cells (0 restores the default: as many as fit 512 MiB of activations). Changes the
 * workspace hom_batched_workspace_size reports; results do not depend on it. */
hom_status hom_set_net_chunk(hom_ctx* ctx, int32_t cells);
/* Measured FMA rate of this GPU (no counterpart in the paper; a measurement aid):
 * precision HOM_FP32 or HOM_FP64; runs 8 independent FMA chains per thread on 4 CTAs
 * of 512 threads per SM on `stream`, best of 5 timed launches after one warm-up, and
 * returns the rate in TFLOP/s (one FMA = 2 flops) in *tflops. The denominator of the
 * ALU-bound rooflines of the FFT passes. Uses no memory beyond a static 8-byte sink. */
hom_status hom_peak_probe(hom_ctx* ctx, int32_t precision, void* stream, double* tflops);
hom_status hom_profile_kernel(hom_ctx* ctx, const char* name);
hom_status hom_kernel_timing(hom_ctx* ctx, int64_t* launches, double* total_ms);

#ifdef __cplusplus
}
#endif
#endif /* HOMB_H */
