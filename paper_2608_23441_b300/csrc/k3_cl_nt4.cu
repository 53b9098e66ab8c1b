// K3 instantiations: column clusters, 4 taps.
#include "k3_launch.cuh"

namespace ipfb {
cudaError_t k3_cl_nt4(int C, int S, float2* d2, const float* window, int N, GainParams gp, cudaStream_t st) {
  return k3_dispatch_cl<4>(C, S, d2, window, N, gp, st);
}
}  // namespace ipfb
