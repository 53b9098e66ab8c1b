// Batched column kernels, variants 10 and 11: 1024 threads (16 elements each) on runs
// of 16384 elements, one CTA per SM: a single CTA per column pair for M = 16384
// (variant 10), a 2-CTA cluster for M = 32768 (variant 11); radix <= 32.
#include "batched_kernels.cuh"

namespace ipfb {
cudaError_t kb3_launch_v10(int M, const BStream* s, const BItem* it, int n, int* ctr, cudaStream_t stream,
                           int* nclusters) {
  if (M == 16384) return Kb3Launch<1, 1024, 32>::template go<16384>(s, it, n, ctr, stream, nclusters);
  return cudaErrorNotSupported;
}
cudaError_t kb3_launch_v11(int M, const BStream* s, const BItem* it, int n, int* ctr, cudaStream_t stream,
                           int* nclusters) {
  if (M == 32768) return Kb3Launch<2, 1024, 32>::template go<16384>(s, it, n, ctr, stream, nclusters);
  return cudaErrorNotSupported;
}
}  // namespace ipfb
