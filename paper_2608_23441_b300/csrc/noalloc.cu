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
// process exits.  Host code cannot use the array's name as a device address, so
// every call asks the runtime for the array's address on the current device
// (cudaGetSymbolAddress, a host-side lookup that allocates nothing), with that
// device current.  Asking on every call, rather than caching the answer per
// device, keeps the address right after a device reset, when the library's device
// code is loaded again and the array may move.  The first call on a device also
// loads that device code there; make it before any stream capture.
//
// All calls share the one array and it keeps the previous call's contents: each
// call clears the sums on its stream before use, and calls whose work overlaps on
// the GPU (different streams, or different host threads, on the same device) race
// on the array and give wrong scales.  Serialize them.
#include <cuda_runtime.h>

#include "../../include/ipfb.h"
#include "abi.h"
#include "launch.h"

namespace {

constexpr int kNoallocMaxLblock = 16384;
constexpr int kNoallocSums = 2 * (kNoallocMaxLblock / 2 + 1);
// the array holds exactly what pfb_forward asks of its workspace at the largest lblock
static_assert(kNoallocSums * sizeof(double) >= ipfb::forward_ws_bytes(kNoallocMaxLblock),
              "built-in scratch smaller than the forward PFB's workspace");

__device__ __align__(256) double g_noalloc_sums[kNoallocSums];

}  // namespace

extern "C" int pfb_forward_noalloc(const ipfb_geom* g, const float* x, const float* window, uint8_t* codes,
                                   float* scale_out, float* spectra_out, void* stream) {
  int rc = ipfb::check_geom(g, false);
  if (rc) return rc;
  if (!x || !window || !codes || !scale_out) return IPFB_ERR_INVALID;
  // sizes beyond the built-in scratch are refused before anything is enqueued
  if (g->lblock > kNoallocMaxLblock) return IPFB_ERR_UNSUPPORTED;
  void* addr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_sums);
  if (e != cudaSuccess) return ipfb::cuda_fail(e, "cudaGetSymbolAddress");
  if (!addr) return ipfb::cuda_fail(cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
  double* sums = static_cast<double*>(addr);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int H = g->lblock / 2, J = g->nframes;
  if ((e = cudaMemsetAsync(sums, 0, ipfb::forward_ws_bytes(g->lblock), st)) != cudaSuccess)
    return ipfb::cuda_fail(e, "cudaMemsetAsync");
  if ((e = ipfb::launch_k1_power(H, x, window, g->ntap, J, sums, st)) != cudaSuccess)
    return ipfb::cuda_fail(e, "k1_pfb_power");
  if ((e = ipfb::launch_k1_scale(H, J, sums, scale_out, st)) != cudaSuccess)
    return ipfb::cuda_fail(e, "k1_scale_from_sums");
  if ((e = ipfb::launch_k1_quant(H, x, window, g->ntap, J, scale_out, codes, reinterpret_cast<float2*>(spectra_out),
                                 st)) != cudaSuccess)
    return ipfb::cuda_fail(e, "k1_pfb_quant");
  return IPFB_OK;
}
