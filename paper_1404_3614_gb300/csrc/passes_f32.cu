// Operator pass kernels, FP32 instantiations.
#include "passes.cuh"
namespace homb {
HOMB_INST_PASSES(float)
}  // namespace homb
