// Arithmetic peak probe: the FP32 and FP64 FMA rates this GPU sustains, the denominators
// of the ALU-bound rooflines of the FFT passes. Each thread runs 8 independent FMA chains
// x <- x a + b (a just below 1, so the values stay bounded) for `iters` steps; the result
// goes to a device-side sink only when an impossible value appears, so the compiler
// keeps every FMA and memory traffic is nil.
#include "kernels.cuh"

namespace homb {

__device__ double g_probe_sink;

template <typename T>
__global__ void __launch_bounds__(512) k_fma_probe(int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = T(threadIdx.x) * T(1e-3) + T(i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == T(-1234.5)) g_probe_sink = (double)s;
}

cudaError_t launch_fma_probe(int precision_fp64, int blocks, int iters, cudaStream_t s) {
  if (precision_fp64)
    k_fma_probe<double><<<blocks, 512, 0, s>>>(iters, 0.999999, 1e-7);
  else
    k_fma_probe<float><<<blocks, 512, 0, s>>>(iters, 0.999999f, 1e-7f);
  return cudaGetLastError();
}

}  // namespace homb
