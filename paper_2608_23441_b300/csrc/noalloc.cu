// pfb_forward_noalloc: the forward PFB + 4-bit quantization of pfb_forward, for
// callers that cannot hand the library a workspace.
//
// Who needs it: streaming ingest code (e.g. a telescope back end that channelizes
// continuously) typically reserves all of its device memory once at start-up and
// must not allocate afterwards -- cudaMalloc can synchronize the device and stall
// the data stream -- and some host frameworks only pass a library the input and
// output buffers they own.  pfb_forward needs a small scratch buffer (the FP64
// per-channel power sums) that such callers cannot provide.  This entry point keeps
// that scratch in a fixed array compiled into the library instead.
//
// The scratch: a file-scope __device__ array of kNoallocSums doubles, enough for
// lblock <= 16384.  Every GPU that loads the library holds it (131 KB) until the
// process exits.  Host code cannot use the array's name as a device address, so the
// address is obtained with cudaGetSymbolAddress once per device, with that device
// current, the first time the entry point runs there.  That first call therefore
// does one extra runtime query; make it before any stream capture.
//
// All calls share the one array and it keeps the previous call's contents: each
// call clears the sums on its stream before use, and calls whose work overlaps on
// the GPU (different streams, or different host threads, on the same device) race
// on the array and give wrong scales.  Serialize them.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/ipfb.h"
#include "launch.h"

namespace {

constexpr int kNoallocMaxLblock = 16384;
constexpr int kNoallocSums = 2 * (kNoallocMaxLblock / 2 + 1);

__device__ __align__(256) double g_noalloc_sums[kNoallocSums];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {};

int noalloc_scratch(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return IPFB_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return IPFB_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_sums);
    if (e != cudaSuccess || !p) return IPFB_ERR_CUDA;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return IPFB_OK;
}

}  // namespace

extern "C" int pfb_forward_noalloc(const ipfb_geom* g, const float* x, const float* window, uint8_t* codes,
                                   float* scale_out, float* spectra_out, void* stream) {
  if (!g || !x || !window || !codes || !scale_out) return IPFB_ERR_INVALID;
  if (g->lblock < 2 || g->ntap < 1 || g->nframes < 1) return IPFB_ERR_INVALID;
  // sizes beyond the built-in scratch are refused before anything is enqueued
  if (g->lblock > kNoallocMaxLblock) return IPFB_ERR_UNSUPPORTED;
  if ((g->lblock & (g->lblock - 1)) != 0 || g->lblock < 64 || g->ntap > 16 || g->periodic != 1)
    return IPFB_ERR_UNSUPPORTED;
  double* sums = nullptr;
  int rc = noalloc_scratch(&sums);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int H = g->lblock / 2, J = g->nframes;
  cudaError_t e = cudaMemsetAsync(sums, 0, 2 * (size_t)(H + 1) * sizeof(double), st);
  if (e == cudaSuccess) e = ipfb::launch_k1_power(H, x, window, g->ntap, J, sums, st);
  if (e == cudaSuccess) e = ipfb::launch_k1_scale(H, J, sums, scale_out, st);
  if (e == cudaSuccess)
    e = ipfb::launch_k1_quant(H, x, window, g->ntap, J, scale_out, codes, reinterpret_cast<float2*>(spectra_out), st);
  if (e != cudaSuccess) return e == cudaErrorNotSupported ? IPFB_ERR_UNSUPPORTED : IPFB_ERR_CUDA;
  return IPFB_OK;
}
