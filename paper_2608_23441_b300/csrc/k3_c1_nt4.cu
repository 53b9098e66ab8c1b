// K3 instantiations: one CTA per column pair, 4 taps; and the K3 dispatcher.
#include "k3_launch.cuh"

namespace ipfb {
cudaError_t k3_c1_nt4(int S, float2* d2, const float* window, int N, GainParams gp, cudaStream_t st) {
  return k3_dispatch_c1<4>(S, d2, window, N, gp, st);
}

cudaError_t launch_k3(int C, int S, float2* d2, const float* window, int N, GainParams gp, cudaStream_t st) {
  // the Wiener filter with 4 taps has compile-time-tap kernels; other filters and tap
  // counts take the generic ones
  if (gp.ntap == 4 && gp.mode == 0)
    return C > 1 ? k3_cl_nt4(C, S, d2, window, N, gp, st) : k3_c1_nt4(S, d2, window, N, gp, st);
  return C > 1 ? k3_cl_gen(C, S, d2, window, N, gp, st) : k3_c1_gen(S, d2, window, N, gp, st);
}
}  // namespace ipfb
