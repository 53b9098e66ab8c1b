// K3 instantiations: one CTA per column pair, any tap count up to 16.
#include "k3_launch.cuh"

namespace ipfb {
cudaError_t k3_c1_gen(int S, float2* d2, const float* window, int N, GainParams gp, cudaStream_t st) {
  return k3_dispatch_c1<0>(S, d2, window, N, gp, st);
}
}  // namespace ipfb
