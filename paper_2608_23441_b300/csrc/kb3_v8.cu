// Batched column kernel, variant 8: one CTA per column pair (no cluster), S / 16
// threads (128 for M = 2048, 256 for M = 4096), radix <= 32, two CTAs per SM.
#include "batched_kernels.cuh"

namespace ipfb {
cudaError_t kb3_launch_v8(int M, const BStream* s, const BItem* it, int n, int* ctr, cudaStream_t stream,
                          int* nclusters) {
  switch (M) {
    case 2048: return Kb3Launch<1, 128, 32>::template go<2048>(s, it, n, ctr, stream, nclusters);
    case 4096: return Kb3Launch<1, 256, 32>::template go<4096>(s, it, n, ctr, stream, nclusters);
  }
  return cudaErrorNotSupported;
}
}  // namespace ipfb
