// Operator pass kernels, FP32 instantiations.
#include "passes.cuh"
namespace homb {
HOMB_INST_PASSES(float)

int zpipe_pad_grid(int M, int Pin, int Pout, int Nlog, int dir, int X, int nslab, int sms) {
  if (M != 225 || dir <= 0 || Pin != Nlog || Pout != M || !zero_band_free(M, Nlog) || X < 1 || nslab < 1) return 0;
  return zp_pad_grid(X, nslab, sms);
}

int zpipe_final_grid(int M, int Nlog, int d, int C, int X, int nrhs, int sms, int xc) {
  if (M != 225 || d != 3 || C != 3 || Nlog > 3 * 48 || !zero_band_free(M, Nlog) || X < 1 || nrhs < 1 ||
      nrhs > 3 || (xc != 8 && xc != 16))
    return 0;
  return zp_final_grid(X, nrhs, sms, xc);
}
}  // namespace homb
