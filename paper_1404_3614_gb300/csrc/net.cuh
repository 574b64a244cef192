// Learned CG warm start: a 2D or 3D Fourier-layer network on the N-grid of one cell.
// Declarations shared by net.cu (kernels, orchestration) and api.cu (C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace homb {

struct NetConfig {
  int N;       // grid points per axis (odd)
  int cin;     // input channels
  int width;   // hidden channels W
  int modes;   // kept modes K: kx in [0, K), ky in [-K, K)
  int layers;  // Fourier layers L
  int proj;    // projection hidden channels P
  int cout;    // output channels
  int d;       // dimension: 2 (kx in [0, K), ky in [-K, K)) or 3 (also kz in [-K, K))
};

// offsets (floats) of the parameter tensors in the flat parameter array
struct NetOffsets {
  long long lift_w, lift_b;
  long long R[8], W[8], b[8];   // per layer: spectral weights [re/im][kz][ky][kx][W][W], 1x1 weight, bias
  long long p1_w, p1_b, p2_w, p2_b;
  long long total;
};

NetOffsets net_offsets(const NetConfig& c);
long long net_workspace_floats(const NetConfig& c, int batch);

// GEMM on the tensor cores (tcgen05.mma, accumulators in tensor memory): C[b] = alpha *
// op(A[b]) op(B[b]) + beta * C[b]; A, B, C FP32 in memory, rounded to BF16 when staged,
// FP32 accumulation. op = transpose when ta/tb.
// A is M x K (row-major with lda) or K x M when ta; B is K x N (ldb) or N x K when tb.
struct GemmArgs {
  const float* A;
  const float* B;
  float* C;
  int M, N, K;
  int lda, ldb, ldc;
  int ta, tb;
  long long sA, sB, sC;   // batch strides
  int batch;
  float alpha, beta;
  int vecA, vecC;         // set by gemm_bf16: 16-byte vector loads of A rows / stores of C rows
  long long spin;         // set by gemm_bf16: polls of the completion barrier before giving up
  int slot;               // set by gemm_bf16: the calling context's timeout flag
};
cudaError_t gemm_bf16(const GemmArgs& g, cudaStream_t s);
// Number of per-context GEMM timeout flags; context k uses flag k mod kGemmFlagSlots.
constexpr int kGemmFlagSlots = 256;
// The GEMMs launched by this host thread from now on report a timeout in flag `slot` and
// poll their completion barrier at most `spin` times (0: the default limit, ~4 M polls;
// a small value, a test aid, makes the wait give up at once without blocking).
void gemm_set_context(int slot, long long spin);
// Clear (async, on `s`) or read into *flag (async copy to pinned host memory) the timeout
// flag of `slot`: 1 if a GEMM's bounded wait on its tensor-core completion barrier gave up.
cudaError_t gemm_timeout_clear(int slot, cudaStream_t s);
cudaError_t gemm_timeout_read(int slot, int* host_flag, cudaStream_t s);

// forward (keeps activations in ws for a backward when train != 0); out [B*N^d, cout]
cudaError_t net_forward(const NetConfig& c, const float* params, const float* bases, int B, const float* in,
                        float* out, float* ws, int train, cudaStream_t s);
// loss = mean (out - target)^2 ; gradient of the parameters into grad (overwritten)
cudaError_t net_backward(const NetConfig& c, const float* params, const float* bases, int B, const float* in,
                         const float* target, float* grad, float* loss_dev, float* ws, cudaStream_t s);
// scale each group of `group` consecutive channels of each of n samples ([n][pts][ch]) to
// unit RMS over its points and channels
cudaError_t normalise_groups(float* grid, int n, long long pts, int ch, int group, cudaStream_t s);
cudaError_t adam_step(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                      float eps, int step, cudaStream_t s);
// DFT bases for the spectral layers, [bases_floats(c)] floats, computed on the host in FP64
long long bases_floats(const NetConfig& c);
void fill_bases(const NetConfig& c, float* host);
cudaError_t init_params(const NetConfig& c, float* params, unsigned long long seed, cudaStream_t s);

// real N-grid fields [B][(N)][N][N][ch] <-> half spectra [B][ch][(N)][N][Nh] (complex FP64/FP32),
// forward with the 1/N^d factor of Eq. DFT. In 3D the forward runs in place along z; the
// inverse needs `tmp` of half3d_tmp_bytes (unused in 2D).
cudaError_t grid_to_half(int d, int N, int B, int ch, const float* grid, void* half, int fp64, cudaStream_t s);
size_t half3d_tmp_bytes(int N, int B, int ch);
cudaError_t half_to_grid(int d, int N, int B, int ch, const void* half, float* grid, int fp64, void* tmp,
                         cudaStream_t s);

}  // namespace homb
