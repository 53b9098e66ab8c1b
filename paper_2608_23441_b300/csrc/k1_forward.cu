// Forward PFB launches (polyphase sum + real FFT, RMS, quantize + pack).
#include "launch.h"
#include "pfb_kernels.cuh"

namespace ipfb {
namespace {
template <class K>
cudaError_t smem_attr(K kern, size_t bytes) {
  if (bytes > 48 * 1024) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}
template <int H>
size_t k1_smem() {
  constexpr int F = fpc_for(H);
  const size_t a = ((size_t)F * padded_len(H) + 256) * sizeof(float2);
  const size_t b = (size_t)F * 4 * (H / 2 + 1) * sizeof(float);
  return a > b ? a : b;
}
template <int H, int NT>
cudaError_t power_nt(const float* x, const float* w, int ntap, int J, double* sums, cudaStream_t st) {
  constexpr int TPF = tpf_for(H), F = fpc_for(H);
  auto kern = k1_pfb_power<H, TPF, F, NT>;
  const size_t smem = k1_smem<H>();
  cudaError_t e = smem_attr(kern, smem);
  if (e != cudaSuccess) return e;
  const int nblk = (J + F - 1) / F;
  const int grid = nblk < 148 * 4 ? nblk : 148 * 4;
  kern<<<grid, TPF * F, smem, st>>>(x, w, ntap, J, sums);
  return cudaGetLastError();
}
template <int H, int NT>
cudaError_t quant_nt(const float* x, const float* w, int ntap, int J, const float* scale, uint8_t* codes,
                     float2* spectra, cudaStream_t st) {
  constexpr int TPF = tpf_for(H), F = fpc_for(H);
  auto kern = k1_pfb_quant<H, TPF, F, NT>;
  // frames + twiddles, then the H + 1 reciprocal steps
  const size_t smem = ((size_t)F * padded_len(H) + 256) * sizeof(float2) + (size_t)(H + 4) * sizeof(float);
  cudaError_t e = smem_attr(kern, smem);
  if (e != cudaSuccess) return e;
  const int nblk = (J + F - 1) / F;
  const int grid = nblk < 148 * 4 ? nblk : 148 * 4;  // persistent: the twiddle table is built once per CTA
  kern<<<grid, TPF * F, smem, st>>>(x, w, ntap, J, scale, codes, spectra);
  return cudaGetLastError();
}
// 4 taps (the paper's and every benchmark's) get the unrolled loader
template <int H>
cudaError_t power(const float* x, const float* w, int ntap, int J, double* sums, cudaStream_t st) {
  return (ntap == 4 && J >= 4) ? power_nt<H, 4>(x, w, ntap, J, sums, st) : power_nt<H, 0>(x, w, ntap, J, sums, st);
}
template <int H>
cudaError_t quant(const float* x, const float* w, int ntap, int J, const float* scale, uint8_t* codes,
                  float2* spectra, cudaStream_t st) {
  return (ntap == 4 && J >= 4) ? quant_nt<H, 4>(x, w, ntap, J, scale, codes, spectra, st)
                               : quant_nt<H, 0>(x, w, ntap, J, scale, codes, spectra, st);
}
}  // namespace

#define IPFB_H_SWITCH(H, CALL)                      \
  switch (H) {                                      \
    case 32: return CALL(32);                       \
    case 64: return CALL(64);                       \
    case 128: return CALL(128);                     \
    case 256: return CALL(256);                     \
    case 512: return CALL(512);                     \
    case 1024: return CALL(1024);                   \
    case 2048: return CALL(2048);                   \
    case 4096: return CALL(4096);                   \
    case 8192: return CALL(8192);                   \
  }                                                 \
  return cudaErrorNotSupported

cudaError_t launch_k1_power(int H, const float* x, const float* window, int ntap, int J, double* sums,
                            cudaStream_t st) {
#define CALL(h) power<h>(x, window, ntap, J, sums, st)
  IPFB_H_SWITCH(H, CALL);
#undef CALL
}

cudaError_t launch_k1_scale(int H, int J, const double* sums, float* scale, cudaStream_t st) {
  k1_scale_from_sums<<<(H + 1 + 255) / 256, 256, 0, st>>>(sums, H, J, scale);
  return cudaGetLastError();
}

cudaError_t launch_k1_quant(int H, const float* x, const float* window, int ntap, int J, const float* scale,
                            uint8_t* codes, float2* spectra, cudaStream_t st) {
#define CALL(h) quant<h>(x, window, ntap, J, scale, codes, spectra, st)
  IPFB_H_SWITCH(H, CALL);
#undef CALL
}

cudaError_t launch_quantize(int H, long long nspec, const float2* spec, const float* scale, uint8_t* codes,
                            cudaStream_t st) {
  const long long total = nspec * H;
  long long blocks = (total + 255) / 256;
  if (blocks > 148LL * 32) blocks = 148LL * 32;
  if (blocks < 1) blocks = 1;
  k_quantize<<<(unsigned)blocks, 256, 0, st>>>(spec, scale, H, nspec, codes);
  return cudaGetLastError();
}
}  // namespace ipfb
