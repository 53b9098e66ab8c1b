// Launch helper for the K3 instantiations (one translation unit per family).
#pragma once

#include "ipfb_kernels.cuh"
#include "launch.h"

namespace ipfb {
template <int C, int S, int NT>
cudaError_t k3_launch(float2* d2, const float* window, int N, GainParams gp, cudaStream_t st) {
  constexpr int T = t_for(S);
  const size_t smem = (size_t)padded_len(S) * sizeof(float2);
  auto kern = k3_column_wiener<C, S, T, NT>;
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

template <int NT>
cudaError_t k3_dispatch_c1(int S, float2* d2, const float* window, int N, GainParams gp, cudaStream_t st) {
  switch (S) {
    case 16: return k3_launch<1, 16, NT>(d2, window, N, gp, st);
    case 32: return k3_launch<1, 32, NT>(d2, window, N, gp, st);
    case 64: return k3_launch<1, 64, NT>(d2, window, N, gp, st);
    case 128: return k3_launch<1, 128, NT>(d2, window, N, gp, st);
    case 256: return k3_launch<1, 256, NT>(d2, window, N, gp, st);
    case 512: return k3_launch<1, 512, NT>(d2, window, N, gp, st);
    case 1024: return k3_launch<1, 1024, NT>(d2, window, N, gp, st);
    case 2048: return k3_launch<1, 2048, NT>(d2, window, N, gp, st);
    case 4096: return k3_launch<1, 4096, NT>(d2, window, N, gp, st);
    case 8192: return k3_launch<1, 8192, NT>(d2, window, N, gp, st);
  }
  return cudaErrorNotSupported;
}

// Clusters arise for J > 8192, where the split gives S = 8192; S = 512 is kept so
// the cluster path can be exercised at small sizes.
template <int NT>
cudaError_t k3_dispatch_cl(int C, int S, float2* d2, const float* window, int N, GainParams gp,
                           cudaStream_t st) {
  if (S == 8192) {
    switch (C) {
      case 2: return k3_launch<2, 8192, NT>(d2, window, N, gp, st);
      case 4: return k3_launch<4, 8192, NT>(d2, window, N, gp, st);
      case 8: return k3_launch<8, 8192, NT>(d2, window, N, gp, st);
    }
  } else if (S == 512) {
    switch (C) {
      case 2: return k3_launch<2, 512, NT>(d2, window, N, gp, st);
      case 4: return k3_launch<4, 512, NT>(d2, window, N, gp, st);
      case 8: return k3_launch<8, 512, NT>(d2, window, N, gp, st);
    }
  }
  return cudaErrorNotSupported;
}

cudaError_t k3_c1_nt4(int S, float2* d2, const float* window, int N, GainParams gp, cudaStream_t st);
cudaError_t k3_c1_gen(int S, float2* d2, const float* window, int N, GainParams gp, cudaStream_t st);
cudaError_t k3_cl_nt4(int C, int S, float2* d2, const float* window, int N, GainParams gp, cudaStream_t st);
cudaError_t k3_cl_gen(int C, int S, float2* d2, const float* window, int N, GainParams gp, cudaStream_t st);
}  // namespace ipfb
