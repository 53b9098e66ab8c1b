// Batched column kernel, variant 5: cluster of 2, S / 16 threads (S = 512 .. 2048),
// radix <= 32; one kernel per M class.
#include "batched_kernels.cuh"

namespace ipfb {
cudaError_t kb3_launch_v5(int M, const BStream* s, const BItem* it, int n, int* ctr, cudaStream_t stream,
                          int* nclusters) {
  return Kb3LaunchAutoT<2, 32>::launch(M, s, it, n, ctr, stream, nclusters);
}
}  // namespace ipfb
