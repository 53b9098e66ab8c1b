// Up-channelizer launches.
#include "launch.h"
#include "upchan_kernels.cuh"

namespace ipfb {
namespace {
template <int CU, int U, int PP>
cudaError_t k4(const UpchanSrc& src, long long nblocks, float2* out, float* x_out, cudaStream_t st) {
  constexpr int T = 256;
  auto kern = k4_upchan<CU, U, PP, T>;
  const size_t smem = (size_t)(padded_len(U * PP) + 1024) * sizeof(float2);
  cudaError_t e;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if constexpr (CU == 1) {
    kern<<<(unsigned)nblocks, T, smem, st>>>(src, out, x_out);
    return cudaGetLastError();
  } else {
    if (CU > 8) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nblocks * CU));
    cfg.blockDim = dim3(T);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CU;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, src, out, x_out);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
}
}  // namespace

// L = block length.  Time-order source: U = 64 (32 for L = 1024), P = L/(2U).
// Column-pair source: U = L/N (the up-channelization factor), P = N/2.
cudaError_t launch_upchan(const UpchanSrc& src, int L, long long nblocks, float2* out, float* x_out,
                          cudaStream_t st) {
  const int Q = L / 2;
  int U, P;
  if (src.x) {
    U = (Q >= 1024) ? 64 : 32;
    P = Q / U;
  } else {
    P = src.N / 2;
    U = Q / P;
    if (U % src.C) return cudaErrorNotSupported;
  }
  int CU = 1;
  while (Q / CU > 8192) CU *= 2;
  const int PP = P / CU;
#define IPFB_K4(cu, u, pp) \
  if (CU == cu && U == u && PP == pp) return k4<cu, u, pp>(src, nblocks, out, x_out, st)
  IPFB_K4(16, 64, 128);
  IPFB_K4(8, 64, 128);
  IPFB_K4(4, 64, 128);
  IPFB_K4(2, 64, 128);
  IPFB_K4(1, 64, 128);
  IPFB_K4(1, 64, 64);
  IPFB_K4(1, 64, 32);
  IPFB_K4(1, 64, 16);
  IPFB_K4(1, 32, 16);
#undef IPFB_K4
  return cudaErrorNotSupported;
}
}  // namespace ipfb
