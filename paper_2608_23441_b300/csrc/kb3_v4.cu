// Batched column kernel, variant 4: one CTA per column pair (no cluster), 512 threads,
// radix <= 32, up to M = 16384 in one shared-memory buffer; one kernel per M class.
#include "batched_kernels.cuh"

namespace ipfb {
cudaError_t kb3_launch_v4(int M, const BStream* s, const BItem* it, int n, int* ctr, cudaStream_t stream,
                          int* nclusters) {
  return Kb3Launch<1, 512, 32>::launch(M, s, it, n, ctr, stream, nclusters);
}
}  // namespace ipfb
