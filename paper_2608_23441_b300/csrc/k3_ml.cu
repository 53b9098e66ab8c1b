// K3 with the ML solve's Wiener preconditioner gain (k3_column_ml): column clusters of
// the residue splits the HBM-resident ML solve uses (C = 2, 4, 8; S = 512 or 8192).
#include "ipfb_kernels.cuh"
#include "launch.h"

namespace ipfb {
namespace {
template <int C, int S, int NT>
cudaError_t k3_ml(float2* z2, const float* window, int N, const MlGainParams& gp, cudaStream_t st) {
  constexpr int T = t_for(S);
  const size_t smem = (size_t)padded_len(S) * sizeof(float2);
  auto kern = k3_column_ml<C, S, T, NT>;
  cudaError_t e;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int npairs = N / 2;
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
  e = cudaLaunchKernelEx(&cfg, kern, z2, window, N, gp);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int NT>
cudaError_t k3_ml_cs(int C, int S, float2* z2, const float* window, int N, const MlGainParams& gp,
                     cudaStream_t st) {
  if (S == 8192) {
    switch (C) {
      case 2: return k3_ml<2, 8192, NT>(z2, window, N, gp, st);
      case 4: return k3_ml<4, 8192, NT>(z2, window, N, gp, st);
      case 8: return k3_ml<8, 8192, NT>(z2, window, N, gp, st);
    }
  } else if (S == 512) {
    switch (C) {
      case 2: return k3_ml<2, 512, NT>(z2, window, N, gp, st);
      case 4: return k3_ml<4, 512, NT>(z2, window, N, gp, st);
      case 8: return k3_ml<8, 512, NT>(z2, window, N, gp, st);
    }
  }
  return cudaErrorNotSupported;
}
}  // namespace

cudaError_t launch_k3_ml(int C, int S, float2* z2, const float* window, int N, const MlGainParams& gp,
                         cudaStream_t st) {
  return gp.ntap == 4 ? k3_ml_cs<4>(C, S, z2, window, N, gp, st) : k3_ml_cs<0>(C, S, z2, window, N, gp, st);
}
}  // namespace ipfb
