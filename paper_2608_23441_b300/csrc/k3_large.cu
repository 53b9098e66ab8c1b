// K3 column Wiener instantiations (large).
#include "ipfb_kernels.cuh"
#include "launch.h"

namespace ipfb {
template <int C, int S>
cudaError_t k3_launch(float2* d2, const float* window, int N, GainParams gp, cudaStream_t st) {
  constexpr int T = t_for(S);
  const size_t smem = (size_t)padded_len(S) * sizeof(float2);
  auto kern = k3_column_wiener<C, S, T>;
  cudaError_t e;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int npairs = N / 2;
  if constexpr (C == 1) {
    kern<<<npairs, T, smem, st>>>(d2, window, N, gp);
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(npairs * C);
    cfg.blockDim = dim3(T);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, d2, window, N, gp);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}
cudaError_t launch_k3_small(int S, float2* d2, const float* window, int N, GainParams gp, cudaStream_t st);
cudaError_t launch_k3_cluster(int C, int S, float2* d2, const float* window, int N, GainParams gp,
                              cudaStream_t st);

cudaError_t launch_k3(int C, int S, float2* d2, const float* window, int N, GainParams gp, cudaStream_t st) {
  if (C > 1) return launch_k3_cluster(C, S, d2, window, N, gp, st);
  switch (S) {
    case 2048: return k3_launch<1, 2048>(d2, window, N, gp, st);
    case 4096: return k3_launch<1, 4096>(d2, window, N, gp, st);
    case 8192: return k3_launch<1, 8192>(d2, window, N, gp, st);
  }
  return launch_k3_small(S, d2, window, N, gp, st);
}
}  // namespace ipfb
