// Batched column kernel, variant 2: cluster of 2, 256 threads, radix <= 32.
#include "batched_kernels.cuh"

namespace ipfb {
cudaError_t kb3_launch_v2(const BStream* s, const BItem* it, int n, int* ctr, cudaStream_t stream, int* nclusters) {
  auto kern = kb3_columns<2, 256, 32>;
  const size_t smem = 2 * (size_t)padded_len(8192) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(2);
  int nc = 0;
  e = cudaOccupancyMaxActiveClusters(&nc, kern, &cfg);
  if (e != cudaSuccess) return e;
  if (nc < 1) nc = 1;
  if (nc > n) nc = n;
  *nclusters = nc;
  cfg.gridDim = dim3(nc * 2);
  e = cudaLaunchKernelEx(&cfg, kern, s, it, n, ctr);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}
}  // namespace ipfb
