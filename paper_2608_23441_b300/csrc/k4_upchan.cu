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

// Polyphase sum over blocks for the windowed re-channelizer: xs[b L + t] =
// sum_{r<p} w[r L + t] x[((b + r) mod nb) L + t], four consecutive t per thread.
__global__ void __launch_bounds__(256)
k_block_polyphase(const float4* __restrict__ x, const float4* __restrict__ w, int L4, int ntap, long long nb,
                  float4* __restrict__ xs) {
  const long long total = nb * L4;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / L4;
    const int t = (int)(i % L4);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    long long bb = b;
    for (int r = 0; r < ntap; ++r) {
      const float4 wv = __ldg(w + (size_t)r * L4 + t);
      const float4 xv = __ldg(x + bb * L4 + t);
      acc.x = fmaf(wv.x, xv.x, acc.x);
      acc.y = fmaf(wv.y, xv.y, acc.y);
      acc.z = fmaf(wv.z, xv.z, acc.z);
      acc.w = fmaf(wv.w, xv.w, acc.w);
      bb = (bb + 1 == nb) ? 0 : bb + 1;
    }
    xs[i] = acc;
  }
}

cudaError_t launch_block_polyphase(const float* x, const float* w, int L, int ntap, long long nb, float* xs,
                                   cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long total = nb * (L / 4);
  const long long want = (total + 255) / 256;
  const int grid = (int)(want < (long long)sms * 8 ? want : (long long)sms * 8);
  k_block_polyphase<<<grid > 0 ? grid : 1, 256, 0, st>>>(reinterpret_cast<const float4*>(x),
                                                         reinterpret_cast<const float4*>(w), L / 4, ntap, nb,
                                                         reinterpret_cast<float4*>(xs));
  return cudaGetLastError();
}

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
