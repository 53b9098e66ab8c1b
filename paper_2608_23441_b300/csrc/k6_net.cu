// Learned-preconditioner net launches: weight packing, forward, backward, gradient
// reduction and Adam.
#include "launch.h"
#include "net_kernels.cuh"

namespace ipfb {
using namespace netk;

namespace {
// resident CTAs of a kernel over the whole GPU (persistent grids)
int resident_ctas(const void* kern, int threads, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem) != cudaSuccess) return 0;
  return sms * per;
}
// resident CTAs over the GPU of a kernel that holds `tmem_cols` TMEM columns per CTA
int resident_ctas_tmem(const void* kern, int threads, size_t smem, uint32_t tmem_cols) {
  int dev = 0, sms = 0, regs_sm = 0, smem_sm = 0, rsv = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess)
    return 0;
  const int by_regs = regs_sm / (((fa.numRegs + 7) / 8 * 8) * threads);
  const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + (size_t)rsv);
  const int by_tmem = 512 / (int)tmem_cols;
  const int by_threads = 2048 / threads;
  int per = by_regs < by_smem ? by_regs : by_smem;
  per = per < by_tmem ? per : by_tmem;
  per = per < by_threads ? per : by_threads;
  return sms * (per > 0 ? per : 1);
}
}  // namespace

size_t net_pack_bytes() { return PACK_BYTES; }
int net_nparams() { return NPARAM; }
long long net_bwd_items(int nslots, int J) { return (long long)nslots * ((J + BT - 1) / BT); }
long long net_fwd_items(int nslots, int J) { return (long long)nslots * ((J + FT - 1) / FT); }

cudaError_t launch_net_pack(const float* theta, uint8_t* packed, cudaStream_t st) {
  k6_net_pack<<<(NPACK_BF + 68 + 255) / 256, 256, 0, st>>>(theta, packed);
  return cudaGetLastError();
}

cudaError_t launch_net_forward(const uint8_t* packed, const float* in, float* y, int J, int nslots_host,
                               const int* count, int* zero_other, int max_slots, long long wait_limit, int* status,
                               cudaStream_t st) {
  const size_t smem = fwd_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k6_net_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long items = net_fwd_items(count ? max_slots : nslots_host, J);
  // The occupancy query answers one CTA per SM for this kernel (it allocates tensor
  // memory), but three fit: count them from its registers, shared memory and TMEM.
  const int res = resident_ctas_tmem((const void*)k6_net_forward, 256, smem, kNetTmemCols);
  if (res <= 0) return cudaErrorInvalidConfiguration;
  const long long grid = items < res ? (items < 1 ? 1 : items) : res;
  k6_net_forward<<<(unsigned)grid, 256, smem, st>>>(packed, in, y, J, nslots_host, count, zero_other,
                                                    wait_limit < 0 ? kNetMmaWait : wait_limit, status);
  return cudaGetLastError();
}

cudaError_t launch_net_backward(const uint8_t* packed, const float* in, const float* target, int J, int nslots,
                                float inv_n, float* part, cudaStream_t st) {
  const size_t smem = BwdSmem::total;
  cudaError_t e = cudaFuncSetAttribute(k6_net_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long items = net_bwd_items(nslots, J);
  const int res = resident_ctas((const void*)k6_net_backward, 256, smem);
  if (res <= 0) return cudaErrorInvalidConfiguration;
  const long long grid = items < res ? items : res;
  if (grid < 1) return cudaSuccess;
  k6_net_backward<<<(unsigned)grid, 256, smem, st>>>(packed, in, target, J, nslots, inv_n, part);
  return cudaGetLastError();
}

cudaError_t launch_net_reduce(const float* part, long long nitems, float* grad, float* loss, cudaStream_t st) {
  k6_net_reduce<<<(NPARAM + 1 + 255) / 256, 256, 0, st>>>(part, nitems, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* theta, float* m, float* v, const float* g, int n, float lr, float beta1, float beta2,
                        float eps, float c1, float c2, cudaStream_t st) {
  k6_adam<<<(n + 255) / 256, 256, 0, st>>>(theta, m, v, g, n, lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError();
}
}  // namespace ipfb
