// Flexible-CG launches (learned preconditioner) and the net's training-pair builder.
#include <algorithm>

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
  // one CTA per SM (the kernel's shared memory allows no more) walks the pairs
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int grid = std::max(1, std::min(N / 2, sms));
  kern<<<grid, T, smem, st>>>(phase, d2, b.X, b.R, b.P, b.Z, b.U, mask, prior, window, N, mp, b.cs, b.Y, b.netin,
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

namespace {
// One trip of the learned solve's graph loop is done (or about to start): count it and
// keep the loop running while any column is still active and trips remain.  (Open net
// requests are not the test: before net_from a column is active without asking the net.)
__global__ void __launch_bounds__(256)
k_fcg_loop_ctrl(const FcgCol* __restrict__ cs, int ncols, int* __restrict__ trips, int max_trips,
                cudaGraphConditionalHandle h) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  int mine = 0;
  for (int i = threadIdx.x; i < ncols; i += blockDim.x) mine |= cs[i].active;
  if (mine) atomicOr(&any, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int t = *trips + 1;
    *trips = t;
    cudaGraphSetConditional(h, (any && t <= max_trips) ? 1u : 0u);
  }
}

// The plain-CG fallback runs when any per-column residual is not finite (a net that
// returned NaN or Inf) or when the net gave up waiting for its accumulators.
__global__ void __launch_bounds__(256)
k_fcg_fallback_check(const float* __restrict__ resid, int n2, const int* __restrict__ net_status,
                     int* __restrict__ flag, cudaGraphConditionalHandle h) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = *net_status != 0;
  __syncthreads();
  int mine = 0;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) mine |= !isfinite(resid[i]);
  if (mine) atomicOr(&bad, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    *flag = bad;
    cudaGraphSetConditional(h, bad ? 1u : 0u);
  }
}
}  // namespace

cudaError_t launch_fcg_loop_ctrl(const FcgBufs& b, int ncols, int* trips, int max_trips,
                                 cudaGraphConditionalHandle h, cudaStream_t st) {
  k_fcg_loop_ctrl<<<1, 256, 0, st>>>(b.cs, ncols, trips, max_trips, h);
  return cudaGetLastError();
}

cudaError_t launch_fcg_fallback_check(const float* resid, int n2, const int* net_status, int* flag,
                                      cudaGraphConditionalHandle h, cudaStream_t st) {
  k_fcg_fallback_check<<<1, 256, 0, st>>>(resid, n2, net_status, flag, h);
  return cudaGetLastError();
}
}  // namespace ipfb
