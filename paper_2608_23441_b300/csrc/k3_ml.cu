// K3 with the ML preconditioner gain: the plain form (z = M_W z) and the dispatcher.
#include "k3_ml.cuh"

namespace ipfb {
cudaError_t launch_k3_ml(int C, int S, float2* z2, const float* window, int N, const MlGainParams& gp,
                         cudaStream_t st) {
  if (gp.r_io) return k3_ml_fused(C, S, z2, window, N, gp, st);
  return gp.ntap == 4 ? k3_ml_cs<4, false>(C, S, z2, window, N, gp, st)
                      : k3_ml_cs<0, false>(C, S, z2, window, N, gp, st);
}
}  // namespace ipfb
