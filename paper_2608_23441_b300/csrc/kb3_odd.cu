// Batched column kernels for the Bluestein lengths M = C * 4096 with C = 5, 6
// (20480, 24576): streams with 8192 < J <= 12288 need M >= 2J - 1 > 16384, and these
// lengths serve them with 25-38 % fewer points than 32768.  Cluster of C CTAs (the
// C-point cross stage is a direct DFT), 256 threads, radix <= 32.  Also the matching
// FFT_M(b) tables.
#include "batched_kernels.cuh"

namespace ipfb {
namespace {
template <int C>
cudaError_t bhat_odd(const int* Js, const int* Ms, const float2* const* chirps, float2* const* bhats, int nJ,
                     cudaStream_t stream) {
  constexpr int S = 4096;
  auto kern = kb_bhat_s<C, S, 256, 32>;
  const size_t smem = (size_t)padded_len(S) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nJ * C);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, Js, Ms, chirps, bhats, nJ);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}
}  // namespace

// M = 20480 or 24576; anything else is not supported here
cudaError_t kb3_launch_odd(int M, const BStream* s, const BItem* it, int n, int* ctr, cudaStream_t stream,
                           int* nclusters) {
  switch (M) {
    case 5 * 4096: return Kb3Launch<5, 256, 32>::template go<4096>(s, it, n, ctr, stream, nclusters);
    case 6 * 4096: return Kb3Launch<6, 256, 32>::template go<4096>(s, it, n, ctr, stream, nclusters);
  }
  return cudaErrorNotSupported;
}

// FFT_M(b) of every distinct J whose M is one of the two lengths above (the others
// are skipped by these kernels and filled by kb_bhat)
cudaError_t kb_bhat_odd_launch(const int* Js, const int* Ms, const float2* const* chirps, float2* const* bhats,
                               int nJ, cudaStream_t stream) {
  cudaError_t e = bhat_odd<5>(Js, Ms, chirps, bhats, nJ, stream);
  if (e == cudaSuccess) e = bhat_odd<6>(Js, Ms, chirps, bhats, nJ, stream);
  return e;
}
}  // namespace ipfb
