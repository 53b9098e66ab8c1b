// libipfb C ABI: argument checks, workspace sizing, kernel dispatch.
// Declarations and the meaning of every argument: include/ipfb.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ipfb.h"
#include "abi.h"
#include "launch.h"

using namespace ipfb;

namespace {

thread_local char g_cuda_err[256] = "";

bool misaligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) != 0; }

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

// request counters and status words of the learned solve
constexpr int kFcgCounters = 8;

// Workspace of the learned-preconditioner solve: the pair-packed data d, the
// flexible-CG vectors, the net requests and outputs, per-column state, two request
// counters and the packed BF16 weights.
struct FcgLayout {
  size_t d2, X, R, P, Z, U, Y, netin, cs, mb, cnt, pack, total;
};
FcgLayout fcg_layout(int N, int J) {
  const size_t vec = (size_t)J * (size_t)N * sizeof(float);
  FcgLayout L;
  size_t o = 0;
  for (size_t* f : {&L.d2, &L.X, &L.R, &L.P, &L.Z, &L.U, &L.Y}) {
    *f = o;
    o = al256(o + vec);
  }
  L.netin = o;
  o = al256(o + 2 * vec);
  L.cs = o;
  o = al256(o + (size_t)N * fcg_col_bytes());
  L.mb = o;
  o = al256(o + (size_t)(N / 2) * (size_t)fcg_threads(J) * sizeof(uint32_t));
  L.cnt = o;
  o = al256(o + kFcgCounters * sizeof(int));
  L.pack = o;
  o = al256(o + net_pack_bytes());
  L.total = o;
  return L;
}
std::atomic<int> g_max_column_run{8192};
// bound on the net forward's accumulator wait in SM clocks (< 0: the built-in ~1 s)
std::atomic<long long> g_net_wait_limit{-1};

// ---------------------------------------------------------------- stage timing
// When enabled, every kernel launch of a compute call is bracketed by two CUDA
// events recorded on the call's stream; ipfb_stage_times sums their elapsed times.
struct StageRec {
  const char* name;
  cudaEvent_t a, b;
};
std::mutex g_tmu;
bool g_timing = false;
std::vector<StageRec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t pool_get() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

struct Stage {
  const char* name;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  Stage(const char* n, cudaStream_t s) : name(n), st(s) {
    std::lock_guard<std::mutex> lk(g_tmu);
    if (g_timing) {
      a = pool_get();
      if (a) cudaEventRecord(a, st);
    }
  }
  void done() {
    if (!a) return;
    std::lock_guard<std::mutex> lk(g_tmu);
    cudaEvent_t b = pool_get();
    if (!b) return;
    cudaEventRecord(b, st);
    g_recs.push_back({name, a, b});
    a = nullptr;
  }
};

#define CK(call, where)                                 \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// column cluster split of J frames: C CTAs of S = J/C frames each (S <= max run)
void column_split(int J, int* C, int* S) {
  int c = 1;
  const int lim = g_max_column_run.load();
  while (J / c > lim && c < 8) c *= 2;
  *C = c;
  *S = J / c;
}

int run_inverse_core(const ipfb_geom* g, const uint8_t* codes, const float* scale, const float* window,
                     double noise_level, int normalize, float2* d2, int C, int S, cudaStream_t st,
                     int out_block_major = 0, int filter_mode = 0, double threshold = 0.0,
                     const float2* gains = nullptr) {
  const int N = g->lblock, J = g->nframes, H = N / 2;
  {
    Stage t("k2_unpack_irfft", st);
    CK(launch_k2(H, codes, scale, d2, C, S, st), "k2_unpack_irfft");
    t.done();
  }
  GainParams gp;
  gp.phi2 = (float)noise_level;
  gp.gnorm = (noise_level > 0.0 && normalize) ? (float)(1.0 + noise_level) : 1.0f;
  gp.invJ = 1.0f / (float)J;
  gp.J = J;
  gp.ntap = g->ntap;
  gp.out_block_major = out_block_major;
  gp.mode = filter_mode;
  gp.thresh2 = (float)(threshold * threshold);
  gp.gains = gains;
  Stage t("k3_column_wiener", st);
  CK(launch_k3(C, S, d2, window, N, gp, st), "k3_column_wiener");
  t.done();
  return IPFB_OK;
}

int check_noise(double noise_level) {
  if (!(noise_level >= 0.0) || !std::isfinite(noise_level)) return IPFB_ERR_INVALID;
  return IPFB_OK;
}

}  // namespace

namespace ipfb {

constexpr int kMaxTapsAbi = 16;

int check_geom(const ipfb_geom* g, bool need_inverse) {
  if (!g) return IPFB_ERR_INVALID;
  if (g->lblock < 2 || g->ntap < 1 || g->nframes < 1) return IPFB_ERR_INVALID;
  if (!is_pow2(g->lblock) || g->lblock < 64 || g->lblock > 16384) return IPFB_ERR_UNSUPPORTED;
  if (g->ntap > kMaxTapsAbi) return IPFB_ERR_UNSUPPORTED;
  if (g->periodic != 1) return IPFB_ERR_UNSUPPORTED;
  if (need_inverse) {
    if (!is_pow2(g->nframes) || g->nframes < 16 || g->nframes > 65536) return IPFB_ERR_UNSUPPORTED;
  }
  return IPFB_OK;
}

int cuda_fail(cudaError_t e, const char* where) {
  if (e == cudaErrorNotSupported) return IPFB_ERR_UNSUPPORTED;
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", where, cudaGetErrorString(e));
  return IPFB_ERR_CUDA;
}

}  // namespace ipfb

extern "C" {

const char* ipfb_strerror(int status) {
  switch (status) {
    case IPFB_OK: return "ok";
    case IPFB_ERR_INVALID: return "invalid argument";
    case IPFB_ERR_UNSUPPORTED: return "unsupported size or option";
    case IPFB_ERR_WORKSPACE: return "workspace too small";
    case IPFB_ERR_NOT_CONVERGED: return "iterative solve did not converge";
    case IPFB_ERR_TIMEOUT: return "bounded device wait timed out";
    case IPFB_ERR_CUDA: return "CUDA runtime error";
  }
  return "unknown status";
}

const char* ipfb_last_cuda_error(void) { return g_cuda_err; }

int ipfb_version(void) { return 102; }

int ipfb_stage_timing(int enable) {
  std::lock_guard<std::mutex> lk(g_tmu);
  for (auto& r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  g_timing = enable != 0;
  return IPFB_OK;
}

int ipfb_stage_times(char* names, size_t names_cap, double* ms, int* counts, int max_entries) {
  if (!names || !ms || !counts || max_entries < 1 || names_cap < 1) return IPFB_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_tmu);
  std::vector<std::string> keys;
  std::vector<double> tot;
  std::vector<int> cnt;
  for (auto& r : g_recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaEventSynchronize");
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return cuda_fail(cudaGetLastError(), "elapsed");
    size_t i = 0;
    for (; i < keys.size(); ++i)
      if (keys[i] == r.name) break;
    if (i == keys.size()) {
      keys.push_back(r.name);
      tot.push_back(0.0);
      cnt.push_back(0);
    }
    tot[i] += t;
    cnt[i] += 1;
  }
  std::string csv;
  int n = 0;
  for (size_t i = 0; i < keys.size() && n < max_entries; ++i, ++n) {
    if (i) csv += ",";
    csv += keys[i];
    ms[i] = tot[i];
    counts[i] = cnt[i];
  }
  if (csv.size() + 1 > names_cap) return IPFB_ERR_INVALID;
  std::memcpy(names, csv.c_str(), csv.size() + 1);
  return n;
}

int ipfb_set_net_wait_limit(long long cycles) {
  g_net_wait_limit.store(cycles < 0 ? -1 : cycles);
  return IPFB_OK;
}

int ipfb_set_max_column_run(int frames) {
  if (frames != 512 && frames != 8192) return IPFB_ERR_INVALID;
  g_max_column_run.store(frames);
  return IPFB_OK;
}

int ipfb_workspace_size(const ipfb_geom* g, int op, size_t* bytes) {
  if (!bytes) return IPFB_ERR_INVALID;
  *bytes = 0;
  int rc;
  switch (op) {
    case IPFB_OP_FORWARD:
      rc = check_geom(g, false);
      if (rc) return rc;
      *bytes = forward_ws_bytes(g->lblock);
      return IPFB_OK;
    case IPFB_OP_WIENER:
    case IPFB_OP_WIENER_UPCHAN:
      rc = check_geom(g, true);
      if (rc) return rc;
      // the up-channelizer's two passes keep their intermediate in a second buffer
      *bytes = (size_t)g->nframes * (size_t)g->lblock * sizeof(float) * (op == IPFB_OP_WIENER_UPCHAN ? 2 : 1);
      return IPFB_OK;
    case IPFB_OP_WIENER_STREAM:
      rc = check_geom(g, true);
      if (rc) return rc;
      // the chunk's column-pair scratch, then the chunk's time-order output
      *bytes = 2 * al256((size_t)g->nframes * (size_t)g->lblock * sizeof(float));
      return IPFB_OK;
    case IPFB_OP_ML:
    case IPFB_OP_ML_STREAM: {
      rc = check_geom(g, true);
      if (rc) return rc;
      if (g->nframes < 128) return IPFB_ERR_UNSUPPORTED;
      // columns up to the on-chip run are solved by one CTA per pair (d and x in pairs);
      // longer ones keep the CG vectors in HBM in the column transform's residue layout
      int C, S;
      column_split(g->nframes, &C, &S);
      size_t ml = 0;
      if (C == 1) {
        ml = 2 * (size_t)g->nframes * (size_t)g->lblock * sizeof(float);
      } else {
        if (S != 512 && S != 8192) return IPFB_ERR_UNSUPPORTED;  // the cluster transform's runs
        ml = mlb_workspace(g->lblock, C, S);
      }
      // the stream adds the chunk's time-order solution, its iterations and residuals
      *bytes = op == IPFB_OP_ML ? ml
                                : al256(ml) + al256((size_t)g->nframes * (size_t)g->lblock * sizeof(float)) +
                                      al256((size_t)g->lblock * sizeof(int)) +
                                      al256(2 * (size_t)g->lblock * sizeof(float));
      return IPFB_OK;
    }
    case IPFB_OP_ML_LEARNED:
    case IPFB_OP_ML_PAIRS:
      rc = check_geom(g, true);
      if (rc) return rc;
      if (g->nframes < 128 || g->nframes > 8192 || g->ntap != 4) return IPFB_ERR_UNSUPPORTED;
      *bytes = op == IPFB_OP_ML_LEARNED
                   ? fcg_layout(g->lblock, g->nframes).total
                   : 2 * (size_t)g->nframes * (size_t)g->lblock * sizeof(float) + al256((size_t)g->lblock / 2 * 4);
      return IPFB_OK;
  }
  return IPFB_ERR_INVALID;
}

int ipfb_sinc_hamming_window(int lblock, int ntap, float* window_host) {
  if (!window_host || lblock < 1 || ntap < 1) return IPFB_ERR_INVALID;
  const long long M = (long long)lblock * ntap;
  const double pi = 3.14159265358979323846;
  for (long long m = 0; m < M; ++m) {
    const double t = ((double)m - (double)M / 2.0) / (double)lblock;
    const double sinc = (t == 0.0) ? 1.0 : std::sin(pi * t) / (pi * t);
    const double taper = (M > 1) ? 0.54 - 0.46 * std::cos(2.0 * pi * (double)m / (double)(M - 1)) : 1.0;
    window_host[m] = (float)(sinc * taper);
  }
  return IPFB_OK;
}

int pfb_quantize(int lblock, int nspec, const float* spectra, const float* scale, uint8_t* codes,
                 void* stream) {
  if (!spectra || !scale || !codes || nspec < 0 || lblock < 4 || (lblock & 1)) return IPFB_ERR_INVALID;
  if (nspec == 0) return IPFB_OK;
  Stage t("k_quantize", as_stream(stream));
  CK(launch_quantize(lblock / 2, nspec, reinterpret_cast<const float2*>(spectra), scale, codes,
                     as_stream(stream)),
     "k_quantize");
  t.done();
  return IPFB_OK;
}

int pfb_forward(const ipfb_geom* g, const float* x, const float* window, const float* scale_in, uint8_t* codes,
                float* scale_out, float* spectra_out, void* ws, size_t ws_bytes, void* stream) {
  int rc = check_geom(g, false);
  if (rc) return rc;
  if (!x || !window || !codes || !scale_out) return IPFB_ERR_INVALID;
  const int H = g->lblock / 2, J = g->nframes;
  cudaStream_t st = as_stream(stream);
  if (!scale_in) {
    size_t need = 0;
    ipfb_workspace_size(g, IPFB_OP_FORWARD, &need);
    if (!ws || ws_bytes < need) return IPFB_ERR_WORKSPACE;
    double* sums = reinterpret_cast<double*>(ws);
    CK(cudaMemsetAsync(sums, 0, need, st), "cudaMemsetAsync");
    Stage t1("k1_pfb_power", st);
    CK(launch_k1_power(H, x, window, g->ntap, J, sums, st), "k1_pfb_power");
    t1.done();
    Stage t2("k1_scale_from_sums", st);
    CK(launch_k1_scale(H, J, sums, scale_out, st), "k1_scale_from_sums");
    t2.done();
  } else if (scale_out != scale_in) {
    CK(cudaMemcpyAsync(scale_out, scale_in, (size_t)(H + 1) * sizeof(float), cudaMemcpyDeviceToDevice, st),
       "cudaMemcpyAsync");
  }
  Stage t3("k1_pfb_quant", st);
  CK(launch_k1_quant(H, x, window, g->ntap, J, scale_out, codes, reinterpret_cast<float2*>(spectra_out), st),
     "k1_pfb_quant");
  t3.done();
  return IPFB_OK;
}

int ipfb_wiener(const ipfb_geom* g, const uint8_t* codes, const float* scale, const float* window,
                double noise_level, int normalize, float* x_out, void* ws, size_t ws_bytes, void* stream) {
  int rc = check_geom(g, true);
  if (rc) return rc;
  if (!codes || !scale || !window || !x_out || misaligned16(codes)) return IPFB_ERR_INVALID;
  if ((rc = check_noise(noise_level))) return rc;
  size_t need = 0;
  ipfb_workspace_size(g, IPFB_OP_WIENER, &need);
  if (!ws || ws_bytes < need) return IPFB_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  float2* d2 = reinterpret_cast<float2*>(ws);
  int C, S;
  column_split(g->nframes, &C, &S);
  rc = run_inverse_core(g, codes, scale, window, noise_level, normalize, d2, C, S, st);
  if (rc) return rc;
  Stage t("k_pairs_to_time", st);
  CK(launch_pairs_to_time(d2, x_out, g->lblock, C, S, st), "k_pairs_to_time");
  t.done();
  return IPFB_OK;
}

int ipfb_filter(const ipfb_geom* g, const uint8_t* codes, const float* scale, const float* window, int mode,
                double threshold, const float* gains, float* x_out, void* ws, size_t ws_bytes, void* stream) {
  int rc = check_geom(g, true);
  if (rc) return rc;
  if (!codes || !scale || !window || !x_out || misaligned16(codes)) return IPFB_ERR_INVALID;
  if (mode == IPFB_FILTER_THRESHOLD) {
    if (!(threshold >= 0.0) || !std::isfinite(threshold)) return IPFB_ERR_INVALID;
  } else if (mode == IPFB_FILTER_GAINS) {
    if (!gains || (reinterpret_cast<uintptr_t>(gains) & 7) != 0) return IPFB_ERR_INVALID;
  } else {
    return IPFB_ERR_INVALID;
  }
  size_t need = 0;
  ipfb_workspace_size(g, IPFB_OP_WIENER, &need);
  if (!ws || ws_bytes < need) return IPFB_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  float2* d2 = reinterpret_cast<float2*>(ws);
  int C, S;
  column_split(g->nframes, &C, &S);
  rc = run_inverse_core(g, codes, scale, window, 0.0, 0, d2, C, S, st, 0, mode, threshold,
                        reinterpret_cast<const float2*>(gains));
  if (rc) return rc;
  Stage t("k_pairs_to_time", st);
  CK(launch_pairs_to_time(d2, x_out, g->lblock, C, S, st), "k_pairs_to_time");
  t.done();
  return IPFB_OK;
}

int upchannelize(const float* x, int64_t nsamples, int64_t block, float* out, void* ws, size_t ws_bytes,
                 void* stream) {
  (void)ws;
  (void)ws_bytes;
  if (!x || !out || nsamples < 0 || block < 2) return IPFB_ERR_INVALID;
  if (!is_pow2(block) || block < 1024 || block > 262144) return IPFB_ERR_UNSUPPORTED;
  const long long nb = nsamples / block;
  if (nb == 0) return IPFB_OK;
  UpchanSrc src{x, nullptr, 0, 0, 0};
  Stage t("k4_upchan", as_stream(stream));
  CK(launch_upchan(src, (int)block, nb, reinterpret_cast<float2*>(out), nullptr, as_stream(stream)), "k4_upchan");
  t.done();
  return IPFB_OK;
}

int ipfb_wiener_stream(const ipfb_geom* g, int64_t nspec, const uint8_t* codes, const float* scale,
                       const float* window, double noise_level, int normalize, int margin, float* x_out, void* ws,
                       size_t ws_bytes, void* stream) {
  int rc = check_geom(g, true);
  if (rc) return rc;
  if (!codes || !scale || !window || !x_out || misaligned16(codes)) return IPFB_ERR_INVALID;
  if ((rc = check_noise(noise_level))) return rc;
  const int N = g->lblock, J = g->nframes;
  if (margin < 0 || J - 2 * margin < 1 || nspec < J) return IPFB_ERR_INVALID;
  if (((size_t)N / 2) % 16 != 0) return IPFB_ERR_UNSUPPORTED;  // chunk starts must stay 16-byte aligned
  size_t need = 0;
  ipfb_workspace_size(g, IPFB_OP_WIENER_STREAM, &need);
  if (!ws || ws_bytes < need) return IPFB_ERR_WORKSPACE;
  if (misaligned16(ws)) return IPFB_ERR_INVALID;
  cudaStream_t st = as_stream(stream);
  size_t wiener_bytes = 0;
  ipfb_workspace_size(g, IPFB_OP_WIENER, &wiener_bytes);
  float2* d2 = reinterpret_cast<float2*>(ws);
  float* xc = reinterpret_cast<float*>(static_cast<char*>(ws) + al256(wiener_bytes));
  int C, S;
  column_split(J, &C, &S);
  const long long step = J - 2 * margin;
  long long start = 0;
  while (true) {
    const bool last = start + J >= nspec;
    if (last) start = nspec - J;
    rc = run_inverse_core(g, codes + (size_t)start * (N / 2), scale, window, noise_level, normalize, d2, C, S, st);
    if (rc) return rc;
    CK(launch_pairs_to_time(d2, xc, N, C, S, st), "k_pairs_to_time");
    // frames margin .. J - margin of this chunk are frames start + margin .. of the run,
    // stored from x_out[(start) N] (x_out begins at frame `margin`)
    CK(cudaMemcpyAsync(x_out + (size_t)start * N, xc + (size_t)margin * N, (size_t)step * N * sizeof(float),
                       cudaMemcpyDeviceToDevice, st),
       "cudaMemcpyAsync");
    if (last) break;
    start += step;
  }
  return IPFB_OK;
}

int upchannelize_pfb(const float* x, int64_t nsamples, int64_t block, int ntap, const float* window, float* out,
                     void* ws, size_t ws_bytes, void* stream) {
  if (!x || !window || !out || nsamples < 0 || block < 2 || ntap < 1 || ntap > 64) return IPFB_ERR_INVALID;
  if (misaligned16(x) || misaligned16(window)) return IPFB_ERR_INVALID;
  if (!is_pow2(block) || block < 1024 || block > 262144) return IPFB_ERR_UNSUPPORTED;
  const long long nb = nsamples / block;
  if (nb == 0) return IPFB_OK;
  const size_t need = (size_t)nb * (size_t)block * sizeof(float);
  if (!ws || ws_bytes < need) return IPFB_ERR_WORKSPACE;
  if (misaligned16(ws)) return IPFB_ERR_INVALID;
  cudaStream_t st = as_stream(stream);
  float* xs = reinterpret_cast<float*>(ws);
  {
    Stage t("k_block_polyphase", st);
    CK(launch_block_polyphase(x, window, (int)block, ntap, nb, xs, st), "k_block_polyphase");
    t.done();
  }
  UpchanSrc src{xs, nullptr, 0, 0, 0};
  Stage t("k4_upchan", st);
  CK(launch_upchan(src, (int)block, nb, reinterpret_cast<float2*>(out), nullptr, st), "k4_upchan");
  t.done();
  return IPFB_OK;
}

int ipfb_wiener_upchannelize(const ipfb_geom* g, const uint8_t* codes, const float* scale, const float* window,
                             double noise_level, int normalize, int upfactor, float* out, float* x_out, void* ws,
                             size_t ws_bytes, void* stream) {
  int rc = check_geom(g, true);
  if (rc) return rc;
  if (!codes || !scale || !window || !out || misaligned16(codes)) return IPFB_ERR_INVALID;
  if ((rc = check_noise(noise_level))) return rc;
  if (upfactor < 1 || !is_pow2(upfactor)) return IPFB_ERR_UNSUPPORTED;
  const long long L = (long long)upfactor * g->lblock;
  if (L < 1024 || L > 262144) return IPFB_ERR_UNSUPPORTED;
  size_t need = 0;
  ipfb_workspace_size(g, IPFB_OP_WIENER_UPCHAN, &need);
  if (!ws || ws_bytes < need) return IPFB_ERR_WORKSPACE;
  if (misaligned16(ws)) return IPFB_ERR_INVALID;
  cudaStream_t st = as_stream(stream);
  float2* d2 = reinterpret_cast<float2*>(ws);
  int C, S;
  column_split(g->nframes, &C, &S);
  if (upfactor % C) return IPFB_ERR_UNSUPPORTED;
  const long long nb = (long long)g->nframes / upfactor;
  const bool two_pass = nb > 0 && upchan2_supported(g->lblock, C, upfactor);
  rc = run_inverse_core(g, codes, scale, window, noise_level, normalize, d2, C, S, st, two_pass ? 1 : 0);
  if (rc) return rc;
  if (nb == 0) return IPFB_OK;
  if (two_pass) {
    // two passes: frames DFT + pa DFT into the second half of the workspace, then
    // the pb DFTs with the real-input split and contiguous stores
    float2* W = d2 + (size_t)g->nframes * (size_t)(g->lblock / 2);
    {
      Stage ta("k4a_upchan_frames", st);
      CK(launch_k4a(d2, g->lblock, g->nframes, nb, W, x_out, st), "k4a_upchan_frames");
      ta.done();
    }
    Stage tb("k4b_upchan_pairs", st);
    CK(launch_k4b(W, g->lblock, nb, reinterpret_cast<float2*>(out), st), "k4b_upchan_pairs");
    tb.done();
    return IPFB_OK;
  }
  UpchanSrc src{nullptr, d2, g->lblock, C, S};
  Stage t("k4_upchan", st);
  CK(launch_upchan(src, (int)L, nb, reinterpret_cast<float2*>(out), x_out, st), "k4_upchan");
  t.done();
  return IPFB_OK;
}

}  // extern "C"

namespace {
MLParams ml_params(const ipfb_geom* g, const ipfb_ml_params* prm, int use_x0) {
  MLParams mp;
  mp.inv_s2 = (float)(1.0 / prm->noise_var);
  mp.lam = (float)prm->prior_weight;
  mp.tol = (float)prm->tol;
  mp.max_iter = prm->max_iter;
  mp.ntap = g->ntap;
  mp.precond = prm->precond;
  mp.use_x0 = use_x0 ? 1 : 0;
  mp.net_from = prm->net_from;
  return mp;
}

// ---------------------------------------------------------------- learned solve
// The learned solve is one CUDA graph (no host synchronisation, no read-back):
//   k2, [initial guess to pairs], net pack, counters cleared,
//   FCG phase 0 (net_from = 0) or, when the net joins later, the Wiener-only
//   iterations on chip (k5_ml_cg with the hand-over) and FCG phase 3,
//   loop control, WHILE { net, FCG step, net, FCG step, loop control },
//   FCG finish, fallback check, IF { [initial guess to pairs], plain CG },
//   pairs to time order.
// The WHILE body is two flexible-CG iterations with the two request counters in
// fixed roles; the loop control kernel keeps it running while a column is active.
// When the caller's stream is not capturing, the graph is captured on a private stream,
// instantiated and launched on the caller's stream, and released by a later call once
// an event recorded after the launch reports it finished; when the caller's stream is
// capturing, the same nodes go into the caller's graph.
struct Capture {
  cudaStream_t user = nullptr, cap = nullptr, body = nullptr;
  cudaStream_t own_cap = nullptr;
  bool own = false, active = false, body_active = false;
  ~Capture() {
    end_body();
    if (own && active) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(own_cap, &g);
      if (g) cudaGraphDestroy(g);
    }
    if (own_cap) cudaStreamDestroy(own_cap);
    if (body) cudaStreamDestroy(body);
  }
  void end_body() {
    if (body_active) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(body, &g);
      body_active = false;
    }
  }
};

int capture_begin(Capture& c, cudaStream_t user) {
  c.user = user;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(user, &cs), "cudaStreamIsCapturing");
  CK(cudaStreamCreateWithFlags(&c.body, cudaStreamNonBlocking), "cudaStreamCreateWithFlags");
  if (cs == cudaStreamCaptureStatusActive) {
    c.cap = user;
    c.own = false;
    return IPFB_OK;
  }
  if (cs != cudaStreamCaptureStatusNone) return IPFB_ERR_INVALID;  // an invalidated capture
  CK(cudaStreamCreateWithFlags(&c.own_cap, cudaStreamNonBlocking), "cudaStreamCreateWithFlags");
  CK(cudaStreamBeginCapture(c.own_cap, cudaStreamCaptureModeRelaxed), "cudaStreamBeginCapture");
  c.cap = c.own_cap;
  c.own = true;
  c.active = true;
  return IPFB_OK;
}

// a conditional handle on the graph being captured
int capture_handle(Capture& c, unsigned int dflt, cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  CK(cudaStreamGetCaptureInfo(c.cap, &cs, nullptr, &g, nullptr, nullptr, nullptr), "cudaStreamGetCaptureInfo");
  CK(cudaGraphConditionalHandleCreate(h, g, dflt, cudaGraphCondAssignDefault), "cudaGraphConditionalHandleCreate");
  return IPFB_OK;
}

// append a conditional node after the captured work and start capturing its body on c.body
int capture_conditional(Capture& c, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(c.cap, &cs, nullptr, &g, &deps, &ed, &nd), "cudaStreamGetCaptureInfo");
  cudaGraphNodeParams prm = {};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = h;
  prm.conditional.type = type;
  prm.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  CK(cudaGraphAddNode(&node, g, deps, ed, nd, &prm), "cudaGraphAddNode");
  CK(cudaStreamUpdateCaptureDependencies(c.cap, &node, nullptr, 1, cudaStreamSetCaptureDependencies),
     "cudaStreamUpdateCaptureDependencies");
  CK(cudaStreamBeginCaptureToGraph(c.body, prm.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                   cudaStreamCaptureModeRelaxed),
     "cudaStreamBeginCaptureToGraph");
  c.body_active = true;
  return IPFB_OK;
}

int capture_end_body(Capture& c) {
  cudaGraph_t g = nullptr;
  c.body_active = false;
  CK(cudaStreamEndCapture(c.body, &g), "cudaStreamEndCapture");
  return IPFB_OK;
}

// Executable graphs launched by the library, each with an event recorded after its
// launch.  Destroying an executable graph that holds conditional nodes waits on the host
// until its launch has finished, so a graph is released only once its event reports
// completion, by a later call's sweep (cudaEventQuery does not block).
struct LaunchedGraph {
  cudaGraphExec_t exec;
  cudaEvent_t done;
};
std::mutex g_graph_mu;
std::vector<LaunchedGraph> g_graphs;

void sweep_finished_graphs() {
  std::lock_guard<std::mutex> lk(g_graph_mu);
  size_t keep = 0;
  for (size_t i = 0; i < g_graphs.size(); ++i) {
    const cudaError_t q = cudaEventQuery(g_graphs[i].done);
    if (q == cudaErrorNotReady) {
      g_graphs[keep++] = g_graphs[i];
      continue;
    }
    if (q != cudaSuccess) (void)cudaGetLastError();  // e.g. a context reset since: drop the entry
    cudaGraphExecDestroy(g_graphs[i].exec);
    cudaEventDestroy(g_graphs[i].done);
  }
  g_graphs.resize(keep);
}

int capture_finish(Capture& c) {
  if (!c.own) return IPFB_OK;
  cudaGraph_t g = nullptr;
  c.active = false;
  CK(cudaStreamEndCapture(c.cap, &g), "cudaStreamEndCapture");
  sweep_finished_graphs();
  cudaGraphExec_t ex = nullptr;
  cudaEvent_t done = nullptr;
  cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaGraphLaunch(ex, c.user);
  if (e == cudaSuccess) e = cudaEventRecord(done, c.user);
  if (e != cudaSuccess) {
    // nothing was enqueued, or the launch itself failed: nothing of ours is in flight
    if (ex) cudaGraphExecDestroy(ex);
    if (done) cudaEventDestroy(done);
    CK(e, "cudaGraphLaunch");
  }
  std::lock_guard<std::mutex> lk(g_graph_mu);
  g_graphs.push_back({ex, done});
  return IPFB_OK;
}

int ml_solve_learned(const ipfb_geom* g, const uint8_t* codes, const float* scale, const float* window,
                     const ipfb_ml_params* prm, const uint8_t* mask, const float* prior, const float* theta,
                     float* x_inout, int use_x0, int* iters, float* resid, void* ws, size_t ws_bytes,
                     cudaStream_t st) {
  size_t need = 0;
  int rc = ipfb_workspace_size(g, IPFB_OP_ML_LEARNED, &need);
  if (rc) return rc;
  if (!ws || ws_bytes < need) return IPFB_ERR_WORKSPACE;
  const int N = g->lblock, J = g->nframes;
  const FcgLayout L = fcg_layout(N, J);
  uint8_t* w = static_cast<uint8_t*>(ws);
  const float2* d2 = reinterpret_cast<const float2*>(w + L.d2);
  FcgBufs b;
  b.X = reinterpret_cast<float2*>(w + L.X);
  b.R = reinterpret_cast<float2*>(w + L.R);
  b.P = reinterpret_cast<float2*>(w + L.P);
  b.Z = reinterpret_cast<float2*>(w + L.Z);
  b.U = reinterpret_cast<float2*>(w + L.U);
  b.Y = reinterpret_cast<float*>(w + L.Y);
  b.netin = reinterpret_cast<float*>(w + L.netin);
  b.cs = reinterpret_cast<FcgCol*>(w + L.cs);
  b.mb = reinterpret_cast<uint32_t*>(w + L.mb);
  // counters: [0], [1] open requests (alternating roles), [2] loop trips, [3] net
  // status, [4] fallback taken
  int* cnt = reinterpret_cast<int*>(w + L.cnt);
  uint8_t* packed = w + L.pack;
  const MLParams mp = ml_params(g, prm, use_x0);
  const int max_trips = (prm->max_iter + 1) / 2;
  const long long wl = g_net_wait_limit.load();

  Stage t("k5_fcg_solve", st);
  Capture c;
  if ((rc = capture_begin(c, st))) return rc;
  cudaStream_t s = c.cap;
  CK(launch_k2(N / 2, codes, scale, const_cast<float2*>(d2), 1, J, s), "k2_unpack_irfft");
  if (use_x0) CK(launch_time_to_pairs(x_inout, b.X, N, J, s), "k_time_to_pairs");
  CK(launch_net_pack(theta, packed, s), "k6_net_pack");
  CK(cudaMemsetAsync(cnt, 0, kFcgCounters * sizeof(int), s), "cudaMemsetAsync");
  if (prm->net_from >= 1) {
    // The applications before the net joins use the Wiener step alone, so those
    // iterations are Wiener-preconditioned CG: they run on chip (k5_ml_cg, one CTA per
    // column pair, vectors in registers and shared memory), which hands its state over
    // to the flexible-CG kernels; phase 3 takes the next step from it and asks the net
    // for the columns still active.
    MLParams wp = mp;
    wp.precond = 1;
    wp.max_iter = std::min(prm->net_from - 1, prm->max_iter);
    CK(launch_k5_handover(J, d2, mask, prior, window, N, wp, b, prm->max_iter, iters, resid, s), "k5_ml_cg");
    CK(launch_fcg_step(J, 3, d2, b, mask, prior, window, N, mp, cnt, s), "k5_fcg_step");
  } else {
    CK(launch_fcg_step(J, 0, d2, b, mask, prior, window, N, mp, cnt, s), "k5_fcg_step");
  }
  cudaGraphConditionalHandle hl;
  if ((rc = capture_handle(c, 0, &hl))) return rc;
  CK(launch_fcg_loop_ctrl(b, N, cnt + 2, max_trips, hl, s), "k_fcg_loop_ctrl");
  if ((rc = capture_conditional(c, hl, cudaGraphCondTypeWhile))) return rc;
  {
    cudaStream_t bs = c.body;
    for (int h = 0; h < 2; ++h) {
      CK(launch_net_forward(packed, b.netin, b.Y, J, 0, cnt + h, cnt + (h ^ 1), N, wl, cnt + 3, bs),
         "k6_net_forward");
      CK(launch_fcg_step(J, 2, d2, b, mask, prior, window, N, mp, cnt + (h ^ 1), bs), "k5_fcg_step");
    }
    CK(launch_fcg_loop_ctrl(b, N, cnt + 2, max_trips, hl, bs), "k_fcg_loop_ctrl");
  }
  if ((rc = capture_end_body(c))) return rc;
  CK(launch_fcg_finish(J, d2, b, mask, prior, window, N, mp, iters, resid, s), "k5_fcg_finish");
  // Fallback: a net that returns a non-finite value leaves a non-finite residual in the
  // columns it touched (flexible CG cannot recover from it), and a net that gave up
  // waiting left some of its outputs unwritten.  Then the whole solve is redone by plain
  // CG from the same start, so the caller gets plain CG's answer, iterations and residuals.
  cudaGraphConditionalHandle hf;
  if ((rc = capture_handle(c, 0, &hf))) return rc;
  CK(launch_fcg_fallback_check(resid, 2 * N, cnt + 3, cnt + 4, hf, s), "k_fcg_fallback_check");
  if ((rc = capture_conditional(c, hf, cudaGraphCondTypeIf))) return rc;
  {
    cudaStream_t bs = c.body;
    if (use_x0) CK(launch_time_to_pairs(x_inout, b.X, N, J, bs), "k_time_to_pairs");
    MLParams plain = mp;
    plain.precond = 0;
    CK(launch_k5(J, d2, b.X, mask, prior, window, N, plain, iters, resid, bs), "k5_ml_cg");
  }
  if ((rc = capture_end_body(c))) return rc;
  CK(launch_pairs_to_time(b.X, x_inout, N, 1, J, s), "k_pairs_to_time");
  if ((rc = capture_finish(c))) return rc;
  t.done();
  return IPFB_OK;
}
// Plain / Wiener-preconditioned ML solve with the CG vectors in HBM (columns longer than
// the on-chip run), one CUDA graph:
//   k2 (d in the residue layout), transpose of mask / prior / initial guess, right-hand
//   side and r0, init, [K3 on z with r.z], control, WHILE { two CG iterations }, true
//   residual and report, back to time order.
// Each iteration is mlb_ap, then K3 with the ML gain fused with the residual update
// (listed pairs; r.r and r.z) or, without a preconditioner, mlb_xr, then mlb_ctl; the
// two iterations of the body alternate the search-direction buffers, and the second
// control sets the loop condition (a pair still listed and iterations left).  The
// finish applies each pair's last step and writes the solution through Q.
int ml_solve_big(const ipfb_geom* g, const uint8_t* codes, const float* scale, const float* window,
                 const MLParams& mp, const uint8_t* mask, const float* prior, float* x_inout, int* iters,
                 float* resid, void* ws, int C, int S, cudaStream_t st) {
  const int N = g->lblock, J = g->nframes;
  const MlbGeom G = mlb_geom(N, C, S);
  MlbBufs b = mlb_carve(ws, N, C, S);
  if (mp.precond == 0) b.Z = b.R;
  MlGainParams gp;
  gp.phi2 = 0.0f;
  gp.gnorm = 1.0f;
  gp.invJ = 1.0f / (float)J;
  gp.J = J;
  gp.ntap = g->ntap;
  gp.out_block_major = 0;
  gp.inv_s2 = mp.inv_s2;
  gp.lam_m = b.lam_m;
  gp.rz_out = b.rzk;
  // in the loop the transform also forms r -= alpha q on its way in
  MlGainParams gl = gp;
  gl.pair_list = b.list;
  gl.pair_count = b.ctl;
  gl.r_io = b.R;
  gl.q_in = b.Q;
  gl.pq_part = b.part;
  gl.nt = G.NT;
  gl.ps = b.ps;
  gl.rr_out = b.rrk;
  int rc;
  Stage t("k5_mlbig_solve", st);
  Capture c;
  if ((rc = capture_begin(c, st))) return rc;
  cudaStream_t s = c.cap;
  CK(launch_k2(N / 2, codes, scale, b.Q, C, S, s), "k2_unpack_irfft");
  CK(launch_mlb_transpose(mask, prior, mp.use_x0 ? x_inout : nullptr, mp.lam, G, b, s), "k_mlb_transpose");
  CK(launch_mlb_rhs(window, mp, G, b, s), "k_mlb_rhs");
  CK(launch_mlb_init(mp, G, b, s), "k_mlb_init");
  if (mp.precond == 1) CK(launch_k3_ml(C, S, b.Z, window, N, gp, s), "k3_column_ml");
  cudaGraphConditionalHandle h;
  if ((rc = capture_handle(c, 0, &h))) return rc;
  CK(launch_mlb_ctl(1, 1, h, mp, G, b, s), "k_mlb_ctl");
  if ((rc = capture_conditional(c, h, cudaGraphCondTypeWhile))) return rc;
  {
    cudaStream_t bs = c.body;
    for (int half = 0; half < 2; ++half) {
      CK(launch_mlb_ap(half, mp, G, b, bs), "k_mlb_ap");
      if (mp.precond == 1) {
        CK(launch_k3_ml(C, S, b.Z, window, N, gl, bs), "k3_column_ml");
      } else {
        CK(launch_mlb_xr(mp, G, b, bs), "k_mlb_xr");
      }
      CK(launch_mlb_ctl(0, half, h, mp, G, b, bs), "k_mlb_ctl");
    }
  }
  if ((rc = capture_end_body(c))) return rc;
  CK(launch_mlb_finish(mp, G, b, iters, resid, s), "k_mlb_finish");
  CK(launch_pairs_to_time(b.Q, x_inout, N, C, S, s), "k_pairs_to_time");
  if ((rc = capture_finish(c))) return rc;
  t.done();
  return IPFB_OK;
}

// Plain / Wiener-preconditioned ML solve (precond 0 or 1) of one J-frame block:
// unpack + per-frame inverse FFT, [initial guess to pairs], k5_ml_cg, back to time order;
// columns longer than the on-chip run take ml_solve_big.
int ml_solve_core(const ipfb_geom* g, const uint8_t* codes, const float* scale, const float* window,
                  const ipfb_ml_params* prm, const uint8_t* prior_mask, const float* prior_values, float* x_inout,
                  int use_x0, int* iters, float* resid, void* ws, cudaStream_t st) {
  const int N = g->lblock, J = g->nframes;
  {
    int C, S;
    column_split(J, &C, &S);
    if (C > 1)
      return ml_solve_big(g, codes, scale, window, ml_params(g, prm, use_x0), prior_mask, prior_values, x_inout,
                          iters, resid, ws, C, S, st);
  }
  float2* d2 = reinterpret_cast<float2*>(ws);
  float2* x2 = d2 + (size_t)J * (N / 2);
  {
    Stage t("k2_unpack_irfft", st);
    CK(launch_k2(N / 2, codes, scale, d2, 1, J, st), "k2_unpack_irfft");
    t.done();
  }
  if (use_x0) {
    Stage t("k_time_to_pairs", st);
    CK(launch_time_to_pairs(x_inout, x2, N, J, st), "k_time_to_pairs");
    t.done();
  }
  const MLParams mp = ml_params(g, prm, use_x0);
  {
    Stage t("k5_ml_cg", st);
    CK(launch_k5(J, d2, x2, prior_mask, prior_values, window, N, mp, iters, resid, st), "k5_ml_cg");
    t.done();
  }
  Stage t("k_pairs_to_time", st);
  CK(launch_pairs_to_time(x2, x_inout, N, 1, J, st), "k_pairs_to_time");
  t.done();
  return IPFB_OK;
}
}  // namespace

extern "C" {

int ipfb_ml_solve(const ipfb_geom* g, const uint8_t* codes, const float* scale, const float* window,
                  const ipfb_ml_params* prm, const uint8_t* prior_mask, const float* prior_values, const void* net,
                  float* x_inout, int use_x0, int* iters, float* resid, void* ws, size_t ws_bytes, void* stream) {
  int rc = check_geom(g, true);
  if (rc) return rc;
  if (!codes || !scale || !window || !prm || !prior_mask || !prior_values || !x_inout || !iters || !resid ||
      misaligned16(codes))
    return IPFB_ERR_INVALID;
  if (!(prm->noise_var > 0.0) || !std::isfinite(prm->noise_var) || !(prm->prior_weight >= 0.0) ||
      !std::isfinite(prm->prior_weight) || !(prm->tol >= 0.0) || prm->max_iter < 0 || prm->net_from < 0)
    return IPFB_ERR_INVALID;
  if (prm->precond < 0 || prm->precond > 2) return IPFB_ERR_INVALID;
  if (prm->precond == 2) {
    if (!net) return IPFB_ERR_INVALID;
    return ml_solve_learned(g, codes, scale, window, prm, prior_mask, prior_values, static_cast<const float*>(net),
                            x_inout, use_x0, iters, resid, ws, ws_bytes, as_stream(stream));
  }
  (void)net;
  size_t need = 0;
  if ((rc = ipfb_workspace_size(g, IPFB_OP_ML, &need))) return rc;
  if (!ws || ws_bytes < need) return IPFB_ERR_WORKSPACE;
  if (g->nframes / 16 < g->ntap - 1 && g->ntap > 4) return IPFB_ERR_UNSUPPORTED;
  return ml_solve_core(g, codes, scale, window, prm, prior_mask, prior_values, x_inout, use_x0, iters, resid, ws,
                       as_stream(stream));
}

int ipfb_ml_solve_stream(const ipfb_geom* g, int64_t nspec, const uint8_t* codes, const float* scale,
                         const float* window, const ipfb_ml_params* prm, const uint8_t* prior_mask,
                         const float* prior_values, const float* x0, int margin, float* x_out, int* iters,
                         float* resid, void* ws, size_t ws_bytes, void* stream) {
  int rc = check_geom(g, true);
  if (rc) return rc;
  if (!codes || !scale || !window || !prm || !prior_mask || !prior_values || !x_out || !iters || !resid ||
      misaligned16(codes))
    return IPFB_ERR_INVALID;
  if (!(prm->noise_var > 0.0) || !std::isfinite(prm->noise_var) || !(prm->prior_weight >= 0.0) ||
      !std::isfinite(prm->prior_weight) || !(prm->tol >= 0.0) || prm->max_iter < 0 || prm->net_from < 0)
    return IPFB_ERR_INVALID;
  if (prm->precond < 0 || prm->precond > 2) return IPFB_ERR_INVALID;
  if (prm->precond == 2) return IPFB_ERR_UNSUPPORTED;
  const int N = g->lblock, J = g->nframes;
  if (margin < 0 || J - 2 * margin < 1 || nspec < J) return IPFB_ERR_INVALID;
  if (((size_t)N / 2) % 16 != 0) return IPFB_ERR_UNSUPPORTED;  // chunk starts must stay 16-byte aligned
  if (J / 16 < g->ntap - 1 && g->ntap > 4) return IPFB_ERR_UNSUPPORTED;
  size_t need = 0;
  if ((rc = ipfb_workspace_size(g, IPFB_OP_ML_STREAM, &need))) return rc;
  if (!ws || ws_bytes < need) return IPFB_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  size_t ml_bytes = 0;
  ipfb_workspace_size(g, IPFB_OP_ML, &ml_bytes);
  const size_t chunk_vals = (size_t)J * (size_t)N;
  uint8_t* w = static_cast<uint8_t*>(ws);
  float* xc = reinterpret_cast<float*>(w + al256(ml_bytes));
  int* itc = reinterpret_cast<int*>(w + al256(ml_bytes) + al256(chunk_vals * sizeof(float)));
  float* rc2 = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(itc) + al256((size_t)N * sizeof(int)));
  const long long step = J - 2 * margin;
  long long start = 0;
  bool first = true;
  while (true) {
    const bool last = start + J >= nspec;
    if (last) start = nspec - J;
    const size_t off = (size_t)start * (size_t)N;
    if (x0)
      CK(cudaMemcpyAsync(xc, x0 + off, chunk_vals * sizeof(float), cudaMemcpyDeviceToDevice, st), "cudaMemcpyAsync");
    rc = ml_solve_core(g, codes + (size_t)start * (N / 2), scale, window, prm, prior_mask + off, prior_values + off,
                       xc, x0 ? 1 : 0, first ? iters : itc, first ? resid : rc2, ws, st);
    if (rc) return rc;
    if (!first) CK(launch_max_merge(iters, itc, resid, rc2, N, st), "k_max_merge");
    // frames margin .. J - margin of this chunk are frames start + margin .. of the run,
    // stored from x_out[start N] (x_out begins at frame `margin`)
    CK(cudaMemcpyAsync(x_out + off, xc + (size_t)margin * N, (size_t)step * N * sizeof(float),
                       cudaMemcpyDeviceToDevice, st),
       "cudaMemcpyAsync");
    first = false;
    if (last) break;
    start += step;
  }
  return IPFB_OK;
}

int ipfb_ml_training_pairs(const ipfb_geom* g, const float* window, const ipfb_ml_params* prm,
                           const uint8_t* prior_mask, const float* x_star, const float* x_k, const int* pair_index,
                           int npairs, float* xin, float* target, void* ws, size_t ws_bytes, void* stream) {
  int rc = check_geom(g, true);
  if (rc) return rc;
  if (!window || !prm || !prior_mask || !x_star || !x_k || !pair_index || !xin || !target || npairs < 0 ||
      npairs > g->lblock / 2)
    return IPFB_ERR_INVALID;
  for (int i = 0; i < npairs; ++i)
    if (pair_index[i] < 0 || pair_index[i] >= g->lblock / 2) return IPFB_ERR_INVALID;
  if (!(prm->noise_var > 0.0) || !std::isfinite(prm->noise_var) || !(prm->prior_weight >= 0.0) ||
      !std::isfinite(prm->prior_weight))
    return IPFB_ERR_INVALID;
  size_t need = 0;
  if ((rc = ipfb_workspace_size(g, IPFB_OP_ML_PAIRS, &need))) return rc;
  if (!ws || ws_bytes < need) return IPFB_ERR_WORKSPACE;
  if (npairs == 0) return IPFB_OK;
  const int N = g->lblock, J = g->nframes;
  cudaStream_t st = as_stream(stream);
  float2* xs2 = reinterpret_cast<float2*>(ws);
  float2* xk2 = xs2 + (size_t)J * (N / 2);
  int* pl = reinterpret_cast<int*>(xk2 + (size_t)J * (N / 2));
  CK(cudaMemcpyAsync(pl, pair_index, (size_t)npairs * sizeof(int), cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
  CK(launch_time_to_pairs(x_star, xs2, N, J, st), "k_time_to_pairs");
  CK(launch_time_to_pairs(x_k, xk2, N, J, st), "k_time_to_pairs");
  const MLParams mp = ml_params(g, prm, 0);
  Stage t("k5_net_pairs", st);
  CK(launch_net_pairs(J, xs2, xk2, pl, npairs, prior_mask, window, N, mp, xin, target, st), "k5_net_pairs");
  t.done();
  return IPFB_OK;
}

int ipfb_net_nparams(void) { return net_nparams(); }

int ipfb_net_workspace_size(int op, int nslots, int nframes, size_t* bytes) {
  if (!bytes || nslots < 1 || nframes < 1) return IPFB_ERR_INVALID;
  *bytes = 0;
  if (op == IPFB_NET_FORWARD) {
    *bytes = al256(net_pack_bytes());
    return IPFB_OK;
  }
  if (op == IPFB_NET_GRAD) {
    *bytes = al256(net_pack_bytes()) + (size_t)net_bwd_items(nslots, nframes) * (size_t)(net_nparams() + 1) * 4;
    return IPFB_OK;
  }
  return IPFB_ERR_INVALID;
}

int ipfb_net_forward(const float* theta, int nslots, int nframes, const float* xin, float* y, void* ws,
                     size_t ws_bytes, void* stream) {
  if (!theta || !xin || !y || nslots < 1 || nframes < 1) return IPFB_ERR_INVALID;
  size_t need = 0;
  int rc = ipfb_net_workspace_size(IPFB_NET_FORWARD, nslots, nframes, &need);
  if (rc) return rc;
  if (!ws || ws_bytes < need) return IPFB_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  uint8_t* packed = static_cast<uint8_t*>(ws);
  CK(launch_net_pack(theta, packed, st), "k6_net_pack");
  Stage t("k6_net_forward", st);
  CK(launch_net_forward(packed, xin, y, nframes, nslots, nullptr, nullptr, nslots, g_net_wait_limit.load(), nullptr,
                        st),
     "k6_net_forward");
  t.done();
  return IPFB_OK;
}

int ipfb_net_grad(const float* theta, int nslots, int nframes, const float* xin, const float* target, float* loss,
                  float* grad, void* ws, size_t ws_bytes, void* stream) {
  if (!theta || !xin || !target || (!loss && !grad) || nslots < 1 || nframes < 1) return IPFB_ERR_INVALID;
  size_t need = 0;
  int rc = ipfb_net_workspace_size(IPFB_NET_GRAD, nslots, nframes, &need);
  if (rc) return rc;
  if (!ws || ws_bytes < need) return IPFB_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  uint8_t* packed = static_cast<uint8_t*>(ws);
  float* part = reinterpret_cast<float*>(packed + al256(net_pack_bytes()));
  const double n = (double)nslots * (double)nframes;
  CK(launch_net_pack(theta, packed, st), "k6_net_pack");
  {
    Stage t("k6_net_backward", st);
    CK(launch_net_backward(packed, xin, target, nframes, nslots, (float)(1.0 / n), part, st), "k6_net_backward");
    t.done();
  }
  Stage t("k6_net_reduce", st);
  CK(launch_net_reduce(part, net_bwd_items(nslots, nframes), grad, loss, st), "k6_net_reduce");
  t.done();
  return IPFB_OK;
}

int ipfb_net_adam(float* theta, float* m, float* v, const float* grad, int n, int step, double lr, double beta1,
                  double beta2, double eps, void* stream) {
  if (!theta || !m || !v || !grad || n < 1 || step < 1) return IPFB_ERR_INVALID;
  if (!(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
    return IPFB_ERR_INVALID;
  const double c1 = 1.0 - std::pow(beta1, step), c2 = 1.0 - std::pow(beta2, step);
  cudaStream_t st = as_stream(stream);
  Stage t("k6_adam", st);
  CK(launch_adam(theta, m, v, grad, n, (float)lr, (float)beta1, (float)beta2, (float)eps, (float)c1, (float)c2, st),
     "k6_adam");
  t.done();
  return IPFB_OK;
}

}  // extern "C"
