// Launch helper for K3 with the ML solve's preconditioner gain (k3_column_ml) on the
// residue splits of the HBM-resident ML solve (C = 2, 4, 8; S = 512 or 8192).
#pragma once

#include "ipfb_kernels.cuh"
#include "launch.h"

namespace ipfb {
template <int C, int S, int NT, bool FUSED>
cudaError_t k3_ml(float2* z2, const float* window, int N, const MlGainParams& gp, cudaStream_t st) {
  constexpr int T = t_for(S);
  const size_t smem = (size_t)padded_len(S) * sizeof(float2);
  auto kern = k3_column_ml<C, S, T, NT, FUSED>;
  cudaError_t e;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((N / 2) * C);
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

template <int NT, bool FUSED>
cudaError_t k3_ml_cs(int C, int S, float2* z2, const float* window, int N, const MlGainParams& gp,
                     cudaStream_t st) {
  if (S == 8192) {
    switch (C) {
      case 2: return k3_ml<2, 8192, NT, FUSED>(z2, window, N, gp, st);
      case 4: return k3_ml<4, 8192, NT, FUSED>(z2, window, N, gp, st);
      case 8: return k3_ml<8, 8192, NT, FUSED>(z2, window, N, gp, st);
    }
  } else if (S == 512) {
    switch (C) {
      case 2: return k3_ml<2, 512, NT, FUSED>(z2, window, N, gp, st);
      case 4: return k3_ml<4, 512, NT, FUSED>(z2, window, N, gp, st);
      case 8: return k3_ml<8, 512, NT, FUSED>(z2, window, N, gp, st);
    }
  }
  return cudaErrorNotSupported;
}

cudaError_t k3_ml_fused(int C, int S, float2* z2, const float* window, int N, const MlGainParams& gp,
                        cudaStream_t st);
}  // namespace ipfb
