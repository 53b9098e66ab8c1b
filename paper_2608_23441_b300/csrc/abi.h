// Host-side helpers shared by the C-ABI translation units (api.cu, noalloc.cu):
// the geometry check, the forward PFB's scratch size and the CUDA error record
// behind ipfb_last_cuda_error().
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/ipfb.h"

namespace ipfb {

// FP64 per-channel power sums of the forward PFB (Re^2 and Im^2 for N/2 + 1 channels)
constexpr size_t forward_ws_bytes(int lblock) { return 2 * (size_t)(lblock / 2 + 1) * sizeof(double); }

// IPFB_OK, or the IPFB_ERR_* code for a geometry outside the built kernels
// (need_inverse: the frame-count limits of the inverse transforms apply too)
int check_geom(const ipfb_geom* g, bool need_inverse);

// Record "<where>: <CUDA error string>" for ipfb_last_cuda_error() and return the
// status for e (IPFB_ERR_UNSUPPORTED for cudaErrorNotSupported, else IPFB_ERR_CUDA).
int cuda_fail(cudaError_t e, const char* where);

}  // namespace ipfb
