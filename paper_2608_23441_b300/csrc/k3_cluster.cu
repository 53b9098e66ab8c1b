// K3 column Wiener instantiations (cluster).
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
// Clusters only arise for J > 8192, where the split gives S = 8192; S = 512 is kept
// so that the cluster path can be exercised at small sizes.
cudaError_t launch_k3_cluster(int C, int S, float2* d2, const float* window, int N, GainParams gp,
                              cudaStream_t st) {
  if (S == 8192) {
    switch (C) {
      case 2: return k3_launch<2, 8192>(d2, window, N, gp, st);
      case 4: return k3_launch<4, 8192>(d2, window, N, gp, st);
      case 8: return k3_launch<8, 8192>(d2, window, N, gp, st);
    }
  } else if (S == 512) {
    switch (C) {
      case 2: return k3_launch<2, 512>(d2, window, N, gp, st);
      case 4: return k3_launch<4, 512>(d2, window, N, gp, st);
      case 8: return k3_launch<8, 512>(d2, window, N, gp, st);
    }
  }
  return cudaErrorNotSupported;
}
}  // namespace ipfb
