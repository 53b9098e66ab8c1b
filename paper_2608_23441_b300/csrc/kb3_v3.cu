// Batched column kernel, variant 3: cluster of 8, 256 threads, radix <= 32; one kernel per M class.
#include "batched_kernels.cuh"

namespace ipfb {
cudaError_t kb3_launch_v3(int M, const BStream* s, const BItem* it, int n, int* ctr, cudaStream_t stream,
                          int* nclusters) {
  return Kb3Launch<8, 256, 32>::launch(M, s, it, n, ctr, stream, nclusters);
}
}  // namespace ipfb
