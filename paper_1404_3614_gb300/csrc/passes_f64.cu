// Operator pass kernels, FP64 instantiations.
#include "passes.cuh"
namespace homb {
HOMB_INST_PASSES(double)
}  // namespace homb
