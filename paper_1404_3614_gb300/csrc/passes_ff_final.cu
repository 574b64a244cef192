// Operator pass kernels, float-float instantiations of the final pass (the FP64-accurate
// residual of the mixed-precision refinement on the FP32 pipes; one pass per translation
// unit, so that the three compile in parallel).
#include "passes.cuh"
namespace homb {
template cudaError_t launch_final<ffloat>(const FinalArgs&, cudaStream_t);
}  // namespace homb
