// Flexible-CG launches (learned preconditioner) and the net's training-pair builder.
#include "fcg_kernels.cuh"
#include "launch.h"

namespace ipfb {
namespace {

template <int J>
cudaError_t fcg_step(int phase, const float2* d2, const FcgBufs& b, const uint8_t* mask, const float* prior,
                     const float* window, int N, const MLParams& mp, int* counter, cudaStream_t st) {
  constexpr int T = fcg_threads(J);
  auto kern = k5_fcg_step<J, T, 3, 4>;
  const size_t smem = fcg_smem_bytes<J, T>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<N / 2, T, smem, st>>>(phase, d2, b.X, b.R, b.P, b.Z, b.U, mask, prior, window, N, mp, b.cs, b.Y, b.netin,
                               b.mb, counter);
  return cudaGetLastError();
}

template <int J>
cudaError_t fcg_finish(const float2* d2, const FcgBufs& b, const uint8_t* mask, const float* prior,
                       const float* window, int N, const MLParams& mp, int* iters, float* resid, cudaStream_t st) {
  constexpr int T = fcg_threads(J);
  auto kern = k5_fcg_finish<J, T, 3, 4>;
  const size_t smem = fcg_smem_bytes<J, T>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<N / 2, T, smem, st>>>(d2, b.X, mask, prior, window, N, mp, b.cs, iters, resid);
  return cudaGetLastError();
}

template <int J>
cudaError_t net_pairs(const float2* xs, const float2* xk, const int* pl, int npairs, const uint8_t* mask,
                      const float* window, int N, const MLParams& mp, float* xin, float* target, cudaStream_t st) {
  constexpr int T = fcg_threads(J);
  auto kern = k5_net_pairs<J, T, 3, 4>;
  const size_t smem = fcg_smem_bytes<J, T>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<npairs, T, smem, st>>>(xs, xk, pl, mask, window, N, mp, xin, target);
  return cudaGetLastError();
}
}  // namespace

#define IPFB_FCG_J(F, ...)                 \
  switch (J) {                             \
    case 128: return F<128>(__VA_ARGS__);  \
    case 256: return F<256>(__VA_ARGS__);  \
    case 512: return F<512>(__VA_ARGS__);  \
    case 1024: return F<1024>(__VA_ARGS__); \
    case 2048: return F<2048>(__VA_ARGS__); \
    case 4096: return F<4096>(__VA_ARGS__); \
    case 8192: return F<8192>(__VA_ARGS__); \
  }                                        \
  return cudaErrorNotSupported

cudaError_t launch_fcg_step(int J, int phase, const float2* d2, const FcgBufs& b, const uint8_t* mask,
                            const float* prior, const float* window, int N, const MLParams& mp, int* counter,
                            cudaStream_t st) {
  if (mp.ntap != 4) return cudaErrorNotSupported;
  IPFB_FCG_J(fcg_step, phase, d2, b, mask, prior, window, N, mp, counter, st);
}

cudaError_t launch_fcg_finish(int J, const float2* d2, const FcgBufs& b, const uint8_t* mask, const float* prior,
                              const float* window, int N, const MLParams& mp, int* iters, float* resid,
                              cudaStream_t st) {
  if (mp.ntap != 4) return cudaErrorNotSupported;
  IPFB_FCG_J(fcg_finish, d2, b, mask, prior, window, N, mp, iters, resid, st);
}

cudaError_t launch_net_pairs(int J, const float2* xs, const float2* xk, const int* pl, int npairs,
                             const uint8_t* mask, const float* window, int N, const MLParams& mp, float* xin,
                             float* target, cudaStream_t st) {
  if (mp.ntap != 4) return cudaErrorNotSupported;
  if (npairs < 1) return cudaSuccess;
  IPFB_FCG_J(net_pairs, xs, xk, pl, npairs, mask, window, N, mp, xin, target, st);
}
#undef IPFB_FCG_J

size_t fcg_col_bytes() { return sizeof(FcgCol); }
}  // namespace ipfb
