// K3 column Wiener instantiations (small).
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
cudaError_t launch_k3_small(int S, float2* d2, const float* window, int N, GainParams gp, cudaStream_t st) {
  switch (S) {
    case 16: return k3_launch<1, 16>(d2, window, N, gp, st);
    case 32: return k3_launch<1, 32>(d2, window, N, gp, st);
    case 64: return k3_launch<1, 64>(d2, window, N, gp, st);
    case 128: return k3_launch<1, 128>(d2, window, N, gp, st);
    case 256: return k3_launch<1, 256>(d2, window, N, gp, st);
    case 512: return k3_launch<1, 512>(d2, window, N, gp, st);
    case 1024: return k3_launch<1, 1024>(d2, window, N, gp, st);
  }
  return cudaErrorNotSupported;
}
}  // namespace ipfb
