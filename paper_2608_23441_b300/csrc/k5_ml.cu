// ML conjugate-gradient launches and the time-order -> column-pair transpose.
#define IPFB_ML_HOST_KERNELS
#include "launch.h"
#include "ml_kernels.cuh"

namespace ipfb {
namespace {
template <int J, int RMAX, int PRE, int NT>
cudaError_t k5(const float2* d2, float2* x2, const uint8_t* mask, const float* prior, const float* window, int N,
               const MLParams& mp, int* iters, float* resid, const FcgBufs& ex, int ex_max_iter, cudaStream_t st) {
  constexpr int T = (J / 16 < 32) ? 32 : (J / 16 > 512 ? 512 : J / 16);
  auto kern = k5_ml_cg<J, T, RMAX, PRE, NT>;
  size_t smem = 2 * (size_t)padded_len(J) * sizeof(float2) + 24 * sizeof(double) + (size_t)(T / 32) * 4 * sizeof(float);
  if (PRE == 1) smem += (size_t)padded_len(J) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<N / 2, T, smem, st>>>(d2, x2, mask, prior, window, N, mp, iters, resid, ex, ex_max_iter);
  return cudaGetLastError();
}

template <int RMAX, int PRE, int NT>
cudaError_t k5_j(int J, const float2* d2, float2* x2, const uint8_t* mask, const float* prior, const float* window,
                 int N, const MLParams& mp, int* iters, float* resid, const FcgBufs& ex, int ex_max_iter,
                 cudaStream_t st) {
  switch (J) {
    case 128: return k5<128, RMAX, PRE, NT>(d2, x2, mask, prior, window, N, mp, iters, resid, ex, ex_max_iter, st);
    case 256: return k5<256, RMAX, PRE, NT>(d2, x2, mask, prior, window, N, mp, iters, resid, ex, ex_max_iter, st);
    case 512: return k5<512, RMAX, PRE, NT>(d2, x2, mask, prior, window, N, mp, iters, resid, ex, ex_max_iter, st);
    case 1024: return k5<1024, RMAX, PRE, NT>(d2, x2, mask, prior, window, N, mp, iters, resid, ex, ex_max_iter, st);
    case 2048: return k5<2048, RMAX, PRE, NT>(d2, x2, mask, prior, window, N, mp, iters, resid, ex, ex_max_iter, st);
    case 4096: return k5<4096, RMAX, PRE, NT>(d2, x2, mask, prior, window, N, mp, iters, resid, ex, ex_max_iter, st);
    case 8192: return k5<8192, RMAX, PRE, NT>(d2, x2, mask, prior, window, N, mp, iters, resid, ex, ex_max_iter, st);
  }
  return cudaErrorNotSupported;
}
}  // namespace

cudaError_t launch_k5(int J, const float2* d2, float2* x2, const uint8_t* mask, const float* prior,
                      const float* window, int N, const MLParams& mp, int* iters, float* resid, cudaStream_t st) {
  const FcgBufs none = {};
  if (mp.ntap == 4) {
    if (mp.precond == 1) return k5_j<3, 1, 4>(J, d2, x2, mask, prior, window, N, mp, iters, resid, none, 0, st);
    return k5_j<3, 0, 4>(J, d2, x2, mask, prior, window, N, mp, iters, resid, none, 0, st);
  }
  if (mp.precond == 1) return k5_j<15, 1, 0>(J, d2, x2, mask, prior, window, N, mp, iters, resid, none, 0, st);
  return k5_j<15, 0, 0>(J, d2, x2, mask, prior, window, N, mp, iters, resid, none, 0, st);
}

cudaError_t launch_k5_handover(int J, const float2* d2, const uint8_t* mask, const float* prior,
                               const float* window, int N, const MLParams& mp, const FcgBufs& b, int fcg_max_iter,
                               int* iters, float* resid, cudaStream_t st) {
  if (mp.ntap != 4 || !b.X) return cudaErrorNotSupported;
  return k5_j<3, 1, 4>(J, d2, b.X, mask, prior, window, N, mp, iters, resid, b, fcg_max_iter, st);
}

namespace {
// per-column maxima over the chunks of an overlap-save solve (a NaN residual is kept)
__global__ void k_max_merge(int* __restrict__ it, const int* __restrict__ itc, float* __restrict__ res,
                            const float* __restrict__ resc, int N) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) it[i] = max(it[i], itc[i]);
  if (i < 2 * N) {
    const float a = res[i], b = resc[i];
    res[i] = (b > a || isnan(b)) ? b : a;
  }
}
}  // namespace

cudaError_t launch_max_merge(int* iters, const int* iters_c, float* resid, const float* resid_c, int N,
                             cudaStream_t st) {
  k_max_merge<<<(2 * N + 255) / 256, 256, 0, st>>>(iters, iters_c, resid, resid_c, N);
  return cudaGetLastError();
}

cudaError_t launch_time_to_pairs(const float* x, float2* x2, int N, int J, cudaStream_t st) {
  dim3 grid((N / 2 + 31) / 32, (J + 31) / 32);
  k_time_to_pairs<<<grid, 256, 0, st>>>(x, x2, N, J);
  return cudaGetLastError();
}
}  // namespace ipfb
