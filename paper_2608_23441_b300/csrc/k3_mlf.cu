// K3 with the ML preconditioner gain, fused with the CG residual update r -= alpha q.
#include "k3_ml.cuh"

namespace ipfb {
cudaError_t k3_ml_fused(int C, int S, float2* z2, const float* window, int N, const MlGainParams& gp,
                        cudaStream_t st) {
  return gp.ntap == 4 ? k3_ml_cs<4, true>(C, S, z2, window, N, gp, st)
                      : k3_ml_cs<0, true>(C, S, z2, window, N, gp, st);
}
}  // namespace ipfb
