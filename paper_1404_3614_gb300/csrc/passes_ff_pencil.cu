// Operator pass kernels, float-float instantiations of the pencil pass (the FP64-accurate
// residual of the mixed-precision refinement on the FP32 pipes; one pass per translation
// unit, so that the three compile in parallel).
#include "passes.cuh"
namespace homb {
static_assert(sizeof(cpx<ffloat>) == sizeof(double2), "float-float complex values take FP64's storage");
template cudaError_t launch_pencil<ffloat>(const PencilArgs&, cudaStream_t);
template int pencil_xc<ffloat>(int, int, int);
}  // namespace homb
