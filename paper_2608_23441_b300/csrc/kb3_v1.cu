// Batched column kernel, variant 1: cluster of 4, 256 threads, radix <= 16; one kernel per M class.
#include "batched_kernels.cuh"

namespace ipfb {
cudaError_t kb3_launch_v1(int M, const BStream* s, const BItem* it, int n, int* ctr, cudaStream_t stream,
                          int* nclusters) {
  return Kb3Launch<4, 256, 16>::launch(M, s, it, n, ctr, stream, nclusters);
}
}  // namespace ipfb
