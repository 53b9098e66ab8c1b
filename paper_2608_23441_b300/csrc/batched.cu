// Batched inverse PFB of many uneven streams: host plan, workspace layout, the
// autotuner and the launches of the persistent kernels (batched_kernels.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/ipfb.h"
#define IPFB_BATCHED_HOST_KERNELS
#include "batched_kernels.cuh"

using namespace ipfb;

namespace {

// kb3 variants the autotuner chooses between: cluster size, threads (0: S / 16), max
// radix, and the run lengths S = M / C each serves
struct Variant {
  int C, T, MAXR, smin, smax;
  const char* name;
};
constexpr Variant kVariants[] = {{4, 256, 32, 512, 8192, "c4_t256_r32"},  {4, 256, 16, 512, 8192, "c4_t256_r16"},
                                 {2, 256, 32, 512, 8192, "c2_t256_r32"},  {8, 256, 32, 512, 8192, "c8_t256_r32"},
                                 {1, 512, 32, 512, 16384, "c1_t512_r32"}, {2, 0, 32, 512, 2048, "c2_ts16_r32"},
                                 {4, 0, 32, 512, 2048, "c4_ts16_r32"},    {2, 512, 32, 16384, 16384, "c2_t512_r32"},
                                 {1, 0, 32, 2048, 4096, "c1_ts16_r32"},   {1, 256, 32, 8192, 8192, "c1_t256_r32"},
                                 {1, 1024, 32, 16384, 16384, "c1_t1024_r32"},
                                 {2, 1024, 32, 16384, 16384, "c2_t1024_r32"}};
constexpr int kNumVariants = 12;
constexpr int kNumMClass = 5;   // power-of-two M = 2048 .. 32768, tuned among the variants
constexpr int kNumOddClass = 2; // M = 5, 6 x 4096, one kernel each (kb3_odd.cu)
constexpr int kNumClass = kNumMClass + kNumOddClass;

bool odd_len(int M) { return M == 5 * 4096 || M == 6 * 4096; }
int class_len(int c) { return c < kNumMClass ? (2048 << c) : (c - kNumMClass + 5) * 4096; }
int mclass(int M) {
  if (odd_len(M)) return kNumMClass + M / 4096 - 5;
  int c = 0;
  while ((2048 << c) < M) ++c;
  return c;
}
// a CTA of a cluster holds up to 8192 elements (two buffers); a single CTA up to 16384 (one)
bool variant_ok(int v, int M) {
  const int S = M / kVariants[v].C;
  return S >= kVariants[v].smin && S <= kVariants[v].smax;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Plan {
  std::vector<ipfb_stream_desc> in;
  std::vector<BStream> st;
  std::vector<BItem> items2[6], items4;  // items2: full items by lblock 1024, 2048, 4096, then the short ones
  std::vector<BItem> items3[kNumClass];
  std::vector<int> Js, Ms;
  std::vector<int> jidx;  // stream -> distinct J index
  size_t off_streams = 0, off_items2[6] = {}, off_items4 = 0, off_items3[kNumClass] = {}, off_counters = 0;
  size_t off_Js = 0, off_Ms = 0, off_chirp_ptr = 0, off_bhat_ptr = 0;
  std::vector<size_t> off_chirp, off_bhat, off_d2;
  std::vector<float2*> chirp_ptr, bhat_ptr;  // device addresses of the tables, uploaded by prepare
  size_t total = 0;
  // defaults = the autotuner's choice on the 256-stream batch (M = 2048 .. 32768)
  int variant[kNumMClass] = {8, 8, 9, 10, 11};
  const void* prepared_ws = nullptr;
  int normalize = 1;
};

thread_local char g_berr[256] = "";

int fail(cudaError_t e, const char* where) {
  std::snprintf(g_berr, sizeof(g_berr), "%s: %s", where, cudaGetErrorString(e));
  return IPFB_ERR_CUDA;
}
#define BCK(call, where)                          \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return fail(e_, where); \
  } while (0)

int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Bluestein convolution length of a J-point DFT: the smallest supported M >= 2J - 1,
// a power of two or, above 16384, 5 or 6 x 4096 (a 7-CTA cluster for 28672 measured
// twice the time per point of the 8-CTA one at 32768, so J > 12288 keeps 32768)
int bluestein_len(int J) {
  const int need = 2 * J - 1, p = next_pow2(need);
  if (p > 16384)
    for (int c = 5; c <= 6; ++c)
      if (c * 4096 >= need && c * 4096 < p) return c * 4096;
  return p;
}

void layout(Plan& P) {
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  P.off_streams = take(P.st.size() * sizeof(BStream));
  for (int q = 0; q < 6; ++q) P.off_items2[q] = take(std::max<size_t>(1, P.items2[q].size()) * sizeof(BItem));
  P.off_items4 = take(P.items4.size() * sizeof(BItem));
  for (int c = 0; c < kNumClass; ++c) P.off_items3[c] = take(std::max<size_t>(1, P.items3[c].size()) * sizeof(BItem));
  P.off_counters = take(16 * sizeof(int));
  P.off_Js = take(P.Js.size() * sizeof(int));
  P.off_Ms = take(P.Ms.size() * sizeof(int));
  P.off_chirp_ptr = take(P.Js.size() * sizeof(float2*));
  P.off_bhat_ptr = take(P.Js.size() * sizeof(float2*));
  P.off_chirp.resize(P.Js.size());
  P.off_bhat.resize(P.Js.size());
  for (size_t t = 0; t < P.Js.size(); ++t) {
    P.off_chirp[t] = take((size_t)P.Js[t] * sizeof(float2));
    P.off_bhat[t] = take((size_t)P.Ms[t] * sizeof(float2));
  }
  P.off_d2.resize(P.st.size());
  for (size_t s = 0; s < P.st.size(); ++s) P.off_d2[s] = take((size_t)P.st[s].J * (P.st[s].N / 2) * sizeof(float2));
  P.total = o;
}

}  // namespace

namespace ipfb {
cudaError_t kb3_launch_v0(int, const BStream*, const BItem*, int, int*, cudaStream_t, int*);
cudaError_t kb3_launch_v1(int, const BStream*, const BItem*, int, int*, cudaStream_t, int*);
cudaError_t kb3_launch_v2(int, const BStream*, const BItem*, int, int*, cudaStream_t, int*);
cudaError_t kb3_launch_v3(int, const BStream*, const BItem*, int, int*, cudaStream_t, int*);
cudaError_t kb3_launch_v4(int, const BStream*, const BItem*, int, int*, cudaStream_t, int*);
cudaError_t kb3_launch_v5(int, const BStream*, const BItem*, int, int*, cudaStream_t, int*);
cudaError_t kb3_launch_v6(int, const BStream*, const BItem*, int, int*, cudaStream_t, int*);
cudaError_t kb3_launch_v7(int, const BStream*, const BItem*, int, int*, cudaStream_t, int*);
cudaError_t kb3_launch_v8(int, const BStream*, const BItem*, int, int*, cudaStream_t, int*);
cudaError_t kb3_launch_v9(int, const BStream*, const BItem*, int, int*, cudaStream_t, int*);
cudaError_t kb3_launch_v10(int, const BStream*, const BItem*, int, int*, cudaStream_t, int*);
cudaError_t kb3_launch_v11(int, const BStream*, const BItem*, int, int*, cudaStream_t, int*);
cudaError_t kb3_launch_odd(int, const BStream*, const BItem*, int, int*, cudaStream_t, int*);
cudaError_t kb_bhat_odd_launch(const int*, const int*, const float2* const*, float2* const*, int, cudaStream_t);
}  // namespace ipfb

namespace {

int launch_kb3(const Plan& P, char* ws, int cls, int v, cudaStream_t stream) {
  const size_t n = P.items3[cls].size();
  if (n == 0) return IPFB_OK;
  const BStream* s = reinterpret_cast<const BStream*>(ws + P.off_streams);
  const BItem* it = reinterpret_cast<const BItem*>(ws + P.off_items3[cls]);
  int* ctr = reinterpret_cast<int*>(ws + P.off_counters) + 2 + cls;
  int nclusters = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if (cls >= kNumMClass) {
    e = kb3_launch_odd(class_len(cls), s, it, (int)n, ctr, stream, &nclusters);
    if (e != cudaSuccess) return fail(e, "kb3_columns");
    return IPFB_OK;
  }
  switch (v) {
    case 0: e = kb3_launch_v0(2048 << cls, s, it, (int)n, ctr, stream, &nclusters); break;
    case 1: e = kb3_launch_v1(2048 << cls, s, it, (int)n, ctr, stream, &nclusters); break;
    case 2: e = kb3_launch_v2(2048 << cls, s, it, (int)n, ctr, stream, &nclusters); break;
    case 3: e = kb3_launch_v3(2048 << cls, s, it, (int)n, ctr, stream, &nclusters); break;
    case 4: e = kb3_launch_v4(2048 << cls, s, it, (int)n, ctr, stream, &nclusters); break;
    case 5: e = kb3_launch_v5(2048 << cls, s, it, (int)n, ctr, stream, &nclusters); break;
    case 6: e = kb3_launch_v6(2048 << cls, s, it, (int)n, ctr, stream, &nclusters); break;
    case 7: e = kb3_launch_v7(2048 << cls, s, it, (int)n, ctr, stream, &nclusters); break;
    case 8: e = kb3_launch_v8(2048 << cls, s, it, (int)n, ctr, stream, &nclusters); break;
    case 9: e = kb3_launch_v9(2048 << cls, s, it, (int)n, ctr, stream, &nclusters); break;
    case 10: e = kb3_launch_v10(2048 << cls, s, it, (int)n, ctr, stream, &nclusters); break;
    case 11: e = kb3_launch_v11(2048 << cls, s, it, (int)n, ctr, stream, &nclusters); break;
  }
  if (e != cudaSuccess) return fail(e, "kb3_columns");
  return IPFB_OK;
}

int prepare(Plan& P, char* ws, cudaStream_t stream) {
  // device pointers inside the workspace
  for (size_t s = 0; s < P.st.size(); ++s) {
    P.st[s].d2 = reinterpret_cast<float2*>(ws + P.off_d2[s]);
    P.st[s].chirp = reinterpret_cast<const float2*>(ws + P.off_chirp[P.jidx[s]]);
    P.st[s].bhat = reinterpret_cast<const float2*>(ws + P.off_bhat[P.jidx[s]]);
  }
  // the pointer tables live in the plan, like every other uploaded array, so that the
  // host side of every copy outlives it without a synchronisation here
  std::vector<float2*>& cp = P.chirp_ptr;
  std::vector<float2*>& bp = P.bhat_ptr;
  cp.assign(P.Js.size(), nullptr);
  bp.assign(P.Js.size(), nullptr);
  for (size_t t = 0; t < P.Js.size(); ++t) {
    cp[t] = reinterpret_cast<float2*>(ws + P.off_chirp[t]);
    bp[t] = reinterpret_cast<float2*>(ws + P.off_bhat[t]);
  }
  auto up = [&](size_t off, const void* src, size_t bytes) -> cudaError_t {
    if (bytes == 0) return cudaSuccess;
    return cudaMemcpyAsync(ws + off, src, bytes, cudaMemcpyHostToDevice, stream);
  };
  BCK(up(P.off_streams, P.st.data(), P.st.size() * sizeof(BStream)), "upload streams");
  for (int q = 0; q < 6; ++q)
    BCK(up(P.off_items2[q], P.items2[q].data(), P.items2[q].size() * sizeof(BItem)), "upload items");
  BCK(up(P.off_items4, P.items4.data(), P.items4.size() * sizeof(BItem)), "upload items");
  for (int c = 0; c < kNumClass; ++c)
    BCK(up(P.off_items3[c], P.items3[c].data(), P.items3[c].size() * sizeof(BItem)), "upload items");
  BCK(up(P.off_Js, P.Js.data(), P.Js.size() * sizeof(int)), "upload J");
  BCK(up(P.off_Ms, P.Ms.data(), P.Ms.size() * sizeof(int)), "upload M");
  BCK(up(P.off_chirp_ptr, cp.data(), cp.size() * sizeof(float2*)), "upload ptr");
  BCK(up(P.off_bhat_ptr, bp.data(), bp.size() * sizeof(float2*)), "upload ptr");
  const int nJ = (int)P.Js.size();
  const int* dJ = reinterpret_cast<const int*>(ws + P.off_Js);
  const int* dM = reinterpret_cast<const int*>(ws + P.off_Ms);
  kb_chirp<<<dim3(16, nJ), 256, 0, stream>>>(dJ, reinterpret_cast<float2* const*>(ws + P.off_chirp_ptr), nJ);
  BCK(cudaGetLastError(), "kb_chirp");
  {
    auto kern = kb_bhat<4, 256, 32>;
    const size_t smem = (size_t)padded_len(8192) * sizeof(float2);
    BCK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "kb_bhat smem");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nJ * 4);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 4;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    BCK(cudaLaunchKernelEx(&cfg, kern, dJ, dM, reinterpret_cast<const float2* const*>(ws + P.off_chirp_ptr),
                           reinterpret_cast<float2* const*>(ws + P.off_bhat_ptr), nJ),
        "kb_bhat");
  }
  if (std::any_of(P.Ms.begin(), P.Ms.end(), odd_len))
    BCK(kb_bhat_odd_launch(dJ, dM, reinterpret_cast<const float2* const*>(ws + P.off_chirp_ptr),
                           reinterpret_cast<float2* const*>(ws + P.off_bhat_ptr), nJ, stream),
        "kb_bhat_s");
  P.prepared_ws = ws;
  return IPFB_OK;
}

// kb2 for the streams of lblock 2H: F spectra of TPF threads per CTA, items list q,
// counter ctr
template <int H, int TPF, int F, bool FULL>
int launch_kb2(const Plan& P, char* ws, int q, int* ctr, cudaStream_t stream) {
  const size_t n = P.items2[q].size();
  if (n == 0) return IPFB_OK;
  auto kern = kb2_unpack<H, TPF, F, FULL>;
  const size_t smem = ((size_t)F * k2_frame_stride(H) + 256) * sizeof(float2) + (size_t)F * H + (H + 4) * sizeof(float);
  BCK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "kb2 smem");
  int per_sm = 0, dev = 0, nsm = 0;
  BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TPF * F, smem), "kb2 occ");
  BCK(cudaGetDevice(&dev), "device");
  BCK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "sm count");
  const int grid = (int)std::min<size_t>(n, (size_t)std::max(1, per_sm) * nsm);
  kern<<<grid, TPF * F, smem, stream>>>(reinterpret_cast<const BStream*>(ws + P.off_streams),
                                        reinterpret_cast<const BItem*>(ws + P.off_items2[q]), (int)n, ctr);
  BCK(cudaGetLastError(), "kb2_unpack");
  return IPFB_OK;
}

int run_all(Plan& P, char* ws, cudaStream_t stream, bool columns_only = false, int only_cls = -1, int only_v = -1) {
  int* ctr = reinterpret_cast<int*>(ws + P.off_counters);
  BCK(cudaMemsetAsync(ctr, 0, 16 * sizeof(int), stream), "counters");
  const BStream* s = reinterpret_cast<const BStream*>(ws + P.off_streams);
  if (!columns_only) {
    // counters: 1 kb4, 2 + class kb3, 10 .. 15 kb2 (full items by lblock, then short)
    int rc = launch_kb2<512, 32, 16, true>(P, ws, 0, ctr + 10, stream);
    if (!rc) rc = launch_kb2<1024, 64, 8, true>(P, ws, 1, ctr + 11, stream);
    if (!rc) rc = launch_kb2<2048, 128, 4, true>(P, ws, 2, ctr + 12, stream);
    if (!rc) rc = launch_kb2<512, 32, 16, false>(P, ws, 3, ctr + 13, stream);
    if (!rc) rc = launch_kb2<1024, 64, 8, false>(P, ws, 4, ctr + 14, stream);
    if (!rc) rc = launch_kb2<2048, 128, 4, false>(P, ws, 5, ctr + 15, stream);
    if (rc) return rc;
  }
  for (int c = 0; c < kNumClass; ++c) {
    if (only_cls >= 0 && c != only_cls) continue;
    const int v = c >= kNumMClass ? 0 : (only_v >= 0 ? only_v : P.variant[c]);
    int rc = launch_kb3(P, ws, c, v, stream);
    if (rc) return rc;
  }
  if (!columns_only && !P.items4.empty()) {
    int dev = 0, nsm = 0;
    BCK(cudaGetDevice(&dev), "device");
    BCK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "sm count");
    const int grid = (int)std::min<size_t>(P.items4.size(), (size_t)nsm * 8);
    kb4_to_time<<<grid, 256, 0, stream>>>(s, reinterpret_cast<const BItem*>(ws + P.off_items4),
                                          (int)P.items4.size(), ctr + 1);
    BCK(cudaGetLastError(), "kb4_to_time");
  }
  return IPFB_OK;
}

void load_cache(Plan& P, const char* path) {
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[256];
  while (std::fgets(line, sizeof(line), f)) {
    int M = 0;
    char name[64] = "";
    if (std::sscanf(line, "%d %63s", &M, name) == 2) {
      for (int v = 0; v < kNumVariants; ++v)
        if (!std::strcmp(name, kVariants[v].name) && variant_ok(v, M) && M >= 2048 && M <= 32768)
          P.variant[mclass(M)] = v;
    }
  }
  std::fclose(f);
}

}  // namespace

extern "C" int ipfb_batched_plan(const ipfb_stream_desc* streams, int nstreams, int normalize,
                                 const char* tune_cache, void** plan_out, size_t* ws_bytes) {
  if (!streams || nstreams < 1 || !plan_out || !ws_bytes) return IPFB_ERR_INVALID;
  *plan_out = nullptr;
  Plan* P = new (std::nothrow) Plan();
  if (!P) return IPFB_ERR_INVALID;
  P->normalize = normalize ? 1 : 0;
  std::map<int, int> jmap;
  struct Cost {
    double c;
    BItem it;
  };
  std::vector<Cost> c2[6], c3[kNumClass], c4;
  for (int s = 0; s < nstreams; ++s) {
    const ipfb_stream_desc& d = streams[s];
    if (!d.codes || !d.scale || !d.window || !d.x_out || (reinterpret_cast<uintptr_t>(d.codes) & 15)) {
      delete P;
      return IPFB_ERR_INVALID;
    }
    if (!(d.lblock == 1024 || d.lblock == 2048 || d.lblock == 4096) || d.ntap != 4 ||
        d.nframes < 1024 || d.nframes > 16384 || !(d.noise_level >= 0.0) || !std::isfinite(d.noise_level)) {
      delete P;
      return IPFB_ERR_UNSUPPORTED;
    }
    P->in.push_back(d);
    BStream b = {};
    b.N = d.lblock;
    b.J = d.nframes;
    b.M = bluestein_len(d.nframes);
    b.ntap = d.ntap;
    b.phi2 = (float)d.noise_level;
    b.gnorm = (d.noise_level > 0.0 && normalize) ? (float)(1.0 + d.noise_level) : 1.0f;
    b.invJ = 1.0f / (float)d.nframes;
    b.codes = d.codes;
    b.scale = d.scale;
    b.window = d.window;
    b.x_out = d.x_out;
    auto f = jmap.find(b.J);
    int ji;
    if (f == jmap.end()) {
      ji = (int)P->Js.size();
      jmap[b.J] = ji;
      P->Js.push_back(b.J);
      P->Ms.push_back(b.M);
    } else {
      ji = f->second;
    }
    P->jidx.push_back(ji);
    P->st.push_back(b);
    const int F = 8192 / (b.N / 2) >= 16 ? 16 : 8192 / (b.N / 2);
    const int q = b.N == 1024 ? 0 : (b.N == 2048 ? 1 : 2);
    for (int j0 = 0; j0 < b.J; j0 += F) c2[j0 + F <= b.J ? q : q + 3].push_back({(double)b.N, {s, j0}});
    const int cls = mclass(b.M);
    for (int p = 0; p < b.N / 2; ++p) c3[cls].push_back({(double)b.M, {s, p}});
    const int ntp = (b.N / 2 + 31) / 32, ntj = (b.J + 63) / 64;
    for (int t = 0; t < ntp * ntj; ++t) c4.push_back({1.0, {s, t}});
  }
  auto sorted = [](std::vector<Cost>& v) {
    std::stable_sort(v.begin(), v.end(), [](const Cost& a, const Cost& b) { return a.c > b.c; });
    std::vector<BItem> out;
    out.reserve(v.size());
    for (auto& c : v) out.push_back(c.it);
    return out;
  };
  for (int q = 0; q < 6; ++q) P->items2[q] = sorted(c2[q]);
  for (int c = 0; c < kNumClass; ++c) P->items3[c] = sorted(c3[c]);
  P->items4 = sorted(c4);
  for (int c = 0; c < kNumMClass; ++c)
    if (!variant_ok(P->variant[c], 2048 << c)) P->variant[c] = 0;
  load_cache(*P, tune_cache);
  layout(*P);
  *plan_out = P;
  *ws_bytes = P->total;
  return IPFB_OK;
}

extern "C" int ipfb_batched_prepare(void* plan, void* ws, size_t ws_bytes, void* stream) {
  Plan* P = static_cast<Plan*>(plan);
  if (!P || !ws) return IPFB_ERR_INVALID;
  if (ws_bytes < P->total) return IPFB_ERR_WORKSPACE;
  return prepare(*P, static_cast<char*>(ws), reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int ipfb_batched_run(void* plan, void* ws, size_t ws_bytes, void* stream) {
  Plan* P = static_cast<Plan*>(plan);
  if (!P || !ws) return IPFB_ERR_INVALID;
  if (ws_bytes < P->total) return IPFB_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (P->prepared_ws != ws) {
    int rc = prepare(*P, static_cast<char*>(ws), st);
    if (rc) return rc;
  }
  return run_all(*P, static_cast<char*>(ws), st);
}

extern "C" int ipfb_batched_autotune(void* plan, void* ws, size_t ws_bytes, void* stream, const char* cache_path) {
  Plan* P = static_cast<Plan*>(plan);
  if (!P || !ws) return IPFB_ERR_INVALID;
  if (ws_bytes < P->total) return IPFB_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  if (P->prepared_ws != ws) {
    int rc = prepare(*P, w, st);
    if (rc) return rc;
  }
  {
    int rc = run_all(*P, w, st);  // fill the column scratch with real data first
    if (rc) return rc;
  }
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0), "event");
  BCK(cudaEventCreate(&e1), "event");
  for (int c = 0; c < kNumMClass; ++c) {
    if (P->items3[c].empty()) continue;
    float best = 1e30f;
    int bestv = P->variant[c];
    for (int v = 0; v < kNumVariants; ++v) {
      if (!variant_ok(v, 2048 << c)) continue;
      int rc = run_all(*P, w, st, true, c, v);  // warm-up (also loads the kernel)
      if (rc) return rc;
      BCK(cudaEventRecord(e0, st), "record");
      rc = run_all(*P, w, st, true, c, v);
      if (rc) return rc;
      BCK(cudaEventRecord(e1, st), "record");
      BCK(cudaEventSynchronize(e1), "sync");
      float ms = 0.0f;
      BCK(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
      if (ms < best) {
        best = ms;
        bestv = v;
      }
    }
    P->variant[c] = bestv;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cache_path) {
    FILE* f = std::fopen(cache_path, "w");
    if (f) {
      for (int c = 0; c < kNumMClass; ++c) std::fprintf(f, "%d %s\n", 2048 << c, kVariants[P->variant[c]].name);
      std::fclose(f);
    }
  }
  return IPFB_OK;
}

extern "C" int ipfb_batched_variant(void* plan, int M, char* name, size_t cap) {
  Plan* P = static_cast<Plan*>(plan);
  if (!P || !name || cap < 16 || M < 2048 || M > 32768) return IPFB_ERR_INVALID;
  if (odd_len(M)) {
    std::snprintf(name, cap, "c%d_t256_r32", M / 4096);
    return IPFB_OK;
  }
  if (M & (M - 1)) return IPFB_ERR_INVALID;
  std::snprintf(name, cap, "%s", kVariants[P->variant[mclass(M)]].name);
  return IPFB_OK;
}

extern "C" int ipfb_batched_free(void* plan) {
  delete static_cast<Plan*>(plan);
  return IPFB_OK;
}
