// K3 instantiations: column clusters, any tap count up to 16.
#include "k3_launch.cuh"

namespace ipfb {
cudaError_t k3_cl_gen(int C, int S, float2* d2, const float* window, int N, GainParams gp, cudaStream_t st) {
  return k3_dispatch_cl<0>(C, S, d2, window, N, gp, st);
}
}  // namespace ipfb
