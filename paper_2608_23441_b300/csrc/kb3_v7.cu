// Batched column kernel, variant 7: cluster of 2, 512 threads, radix <= 32, 16384
// elements per CTA (one shared buffer, one CTA per SM) for M = 32768.
#include "batched_kernels.cuh"

namespace ipfb {
cudaError_t kb3_launch_v7(int M, const BStream* s, const BItem* it, int n, int* ctr, cudaStream_t stream,
                          int* nclusters) {
  if (M == 32768) return Kb3Launch<2, 512, 32>::template go<16384>(s, it, n, ctr, stream, nclusters);
  return cudaErrorNotSupported;
}
}  // namespace ipfb
