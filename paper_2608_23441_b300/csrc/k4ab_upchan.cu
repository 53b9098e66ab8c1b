// Launches of the two-pass up-channelizer of the column-pair scratch (k4a, k4b).
#include "launch.h"
#include "upchan2_kernels.cuh"

namespace ipfb {
namespace {
template <int P>
cudaError_t k4a(const float2* d2, int J, long long nblocks, float2* W, float* x_out, cudaStream_t st) {
  constexpr int Q = K4Shape<P>::Q;
  const size_t smem = (size_t)(64 * 128 + 128 * 66 + (Q >> 9) + 512) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k4a_frames<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k4a_frames<P>, kK4aThreads, smem)) != cudaSuccess)
    return e;
  const long long tiles = nblocks * (K4Shape<P>::PB / K4Shape<P>::NPB);
  const long long res = (long long)sms * (per > 0 ? per : 1);
  k4a_frames<P><<<(unsigned)(tiles < res ? tiles : res), kK4aThreads, smem, st>>>(
      d2, J, nblocks, W, reinterpret_cast<float2*>(x_out));
  return cudaGetLastError();
}

template <int P>
cudaError_t k4b(const float2* W, long long nblocks, float2* out, cudaStream_t st) {
  const size_t smem = k4b_smem_bytes<P>();
  cudaError_t e = cudaFuncSetAttribute(k4b_pairs<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k4b_pairs<P><<<(unsigned)(nblocks * (K4Shape<P>::PA / 2)), kK4bThreads, smem, st>>>(W, out);
  return cudaGetLastError();
}
}  // namespace

bool upchan2_supported(int N, int C, int U) {
  return U == 64 && (N == 1024 || N == 2048 || N == 4096) && C >= 1 && C <= 64 && (C & (C - 1)) == 0;
}

cudaError_t launch_k4a(const float2* d2, int N, int J, long long nblocks, float2* W, float* x_out,
                       cudaStream_t st) {
  switch (N / 2) {
    case 512: return k4a<512>(d2, J, nblocks, W, x_out, st);
    case 1024: return k4a<1024>(d2, J, nblocks, W, x_out, st);
    case 2048: return k4a<2048>(d2, J, nblocks, W, x_out, st);
  }
  return cudaErrorNotSupported;
}

cudaError_t launch_k4b(const float2* W, int N, long long nblocks, float2* out, cudaStream_t st) {
  switch (N / 2) {
    case 512: return k4b<512>(W, nblocks, out, st);
    case 1024: return k4b<1024>(W, nblocks, out, st);
    case 2048: return k4b<2048>(W, nblocks, out, st);
  }
  return cudaErrorNotSupported;
}
}  // namespace ipfb
