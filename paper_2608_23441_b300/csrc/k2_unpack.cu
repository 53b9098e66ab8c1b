// Inverse-PFB first stage (unpack + per-frame inverse real FFT) and the
// column-pair -> time-order transpose.
#include "ipfb_kernels.cuh"
#include "launch.h"

namespace ipfb {
namespace {
template <int H>
cudaError_t k2(const uint8_t* codes, const float* scale, float2* d2, int C, int S, cudaStream_t st) {
  constexpr int TPF = tpf_for(H), F = fpc_for(H);
  const size_t smem = ((size_t)F * k2_frame_stride(H) + 256) * sizeof(float2) + (size_t)F * H + (size_t)(H + 4) * sizeof(float);
  auto kern = k2_unpack_irfft<H, TPF, F>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (S % F) return cudaErrorNotSupported;
  kern<<<(C * S) / F, TPF * F, smem, st>>>(codes, scale, d2, C, S);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_k2(int H, const uint8_t* codes, const float* scale, float2* d2, int C, int S,
                      cudaStream_t st) {
  switch (H) {
    case 32: return k2<32>(codes, scale, d2, C, S, st);
    case 64: return k2<64>(codes, scale, d2, C, S, st);
    case 128: return k2<128>(codes, scale, d2, C, S, st);
    case 256: return k2<256>(codes, scale, d2, C, S, st);
    case 512: return k2<512>(codes, scale, d2, C, S, st);
    case 1024: return k2<1024>(codes, scale, d2, C, S, st);
    case 2048: return k2<2048>(codes, scale, d2, C, S, st);
    case 4096: return k2<4096>(codes, scale, d2, C, S, st);
    case 8192: return k2<8192>(codes, scale, d2, C, S, st);
  }
  return cudaErrorNotSupported;
}

cudaError_t launch_pairs_to_time(const float2* d2, float* x, int N, int C, int S, cudaStream_t st) {
  const int J = C * S;
  const int H = N / 2;
  if (J >= 64) {
    dim3 grid((H + 31) / 32, J / 64);
    k_pairs_to_time<64><<<grid, 256, 0, st>>>(d2, x, N, C, S);
  } else {
    dim3 grid((H + 31) / 32, J / 16);
    k_pairs_to_time<16><<<grid, 256, 0, st>>>(d2, x, N, C, S);
  }
  return cudaGetLastError();
}
}  // namespace ipfb
