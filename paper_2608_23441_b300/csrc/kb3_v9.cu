// Batched column kernel, variant 9: one CTA per column pair (no cluster), 256 threads
// (32 elements each), radix <= 32, two CTAs per SM, for M = 8192.
#include "batched_kernels.cuh"

namespace ipfb {
cudaError_t kb3_launch_v9(int M, const BStream* s, const BItem* it, int n, int* ctr, cudaStream_t stream,
                          int* nclusters) {
  if (M == 8192) return Kb3Launch<1, 256, 32>::template go<8192>(s, it, n, ctr, stream, nclusters);
  return cudaErrorNotSupported;
}
}  // namespace ipfb
