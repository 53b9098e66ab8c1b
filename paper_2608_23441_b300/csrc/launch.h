// Host-side launch functions, one translation unit per kernel family so that the
// library compiles in parallel.  All return a cudaError_t (cudaErrorNotSupported
// for shapes without an instantiation).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ipfb {

struct GainParams {
  float phi2;
  float gnorm;
  float invJ;
  int J;
  int ntap;
  int out_block_major;  // k3 output layout: 0 = the d2 residue runs, 1 = block-major (k4a input)
  // eigenvalue filter: 0 = Wiener (phi2, gnorm); 1 = thresholded pseudo-inverse
  // (|W|^2 >= thresh2 kept as 1 / conj W, else 0); 2 = caller gains [N][J/2 + 1]
  int mode = 0;
  float thresh2 = 0.0f;
  const float2* gains = nullptr;
};

// K3 with the ML solve's preconditioner gain (k3_column_ml): 1 / sigma^2, lam times the
// mask fraction of each column, and an optional list of the pairs to transform
// (*pair_count entries)
struct MlbPair;
struct MlGainParams : GainParams {
  float inv_s2 = 0.0f;
  const float* lam_m = nullptr;
  const int* pair_list = nullptr;
  const int* pair_count = nullptr;
  double* rz_out = nullptr;  // [P][C][2]: each CTA's r.z of both columns (Parseval), or nullptr
  // the CG residual update fused into the transform's load (r_io != nullptr): alpha of
  // each active column from the stencil's per-tile p.q (pq_part [P][nt][8], slots 0, 1)
  // and the pair state, r = r - alpha q written back to r_io, and each CTA's r.r to
  // rr_out [P][C][2]; the transform then runs on r and writes z to d2
  float2* r_io = nullptr;
  const float2* q_in = nullptr;
  const double* pq_part = nullptr;
  int nt = 0;
  const MlbPair* ps = nullptr;
  double* rr_out = nullptr;
};

struct UpchanSrc {
  const float* x;    // time order, or nullptr
  const float2* d2;  // column-pair scratch, or nullptr
  int N;             // lblock of d2 (P = N/2 pairs)
  int C, S;          // residue split of d2 (J = C*S)
};

// threads per frame and frames per CTA for the N/2 = H point per-frame transforms
constexpr int tpf_for(int H) { return H / 16 < 32 ? 32 : (H / 16 > 256 ? 256 : H / 16); }
constexpr int fpc_for(int H) { return H >= 8192 ? 1 : (H >= 4096 ? 2 : 4); }
// threads for the S-point column transform
constexpr int t_for(int S) { return S / 16 < 32 ? 32 : (S / 16 > 256 ? 256 : S / 16); }

cudaError_t launch_k1_power(int H, const float* x, const float* window, int ntap, int J, double* sums,
                            cudaStream_t st);
cudaError_t launch_k1_scale(int H, int J, const double* sums, float* scale, cudaStream_t st);
cudaError_t launch_k1_quant(int H, const float* x, const float* window, int ntap, int J, const float* scale,
                            uint8_t* codes, float2* spectra, cudaStream_t st);
cudaError_t launch_quantize(int H, long long nspec, const float2* spec, const float* scale, uint8_t* codes,
                            cudaStream_t st);
cudaError_t launch_k2(int H, const uint8_t* codes, const float* scale, float2* d2, int C, int S,
                      cudaStream_t st);
cudaError_t launch_k3(int C, int S, float2* d2, const float* window, int N, GainParams gp, cudaStream_t st);
// K3 with the ML preconditioner gain on the residue splits C = 2, 4, 8 with S = 512 or
// 8192; fused with the CG residual update when gp.r_io is set
cudaError_t launch_k3_ml(int C, int S, float2* z2, const float* window, int N, const MlGainParams& gp,
                         cudaStream_t st);
cudaError_t launch_pairs_to_time(const float2* d2, float* x, int N, int C, int S, cudaStream_t st);
struct MLParams {
  float inv_s2;  // 1 / sigma^2
  float lam;     // prior weight (Q^-1 on saved samples)
  float tol;     // relative residual target per column
  int max_iter;
  int ntap;
  int precond;   // 0 none, 1 Wiener, 2 learned (flexible CG)
  int use_x0;    // 1: x2 holds the initial guess
  int net_from = 0;  // learned: preconditioner applications before the net joins (Wiener alone)
};

cudaError_t launch_k5(int J, const float2* d2, float2* x2, const uint8_t* mask, const float* prior,
                      const float* window, int N, const MLParams& mp, int* iters, float* resid, cudaStream_t st);
cudaError_t launch_time_to_pairs(const float* x, float2* x2, int N, int J, cudaStream_t st);
// iters[n] = max(iters[n], iters_c[n]), resid[i] = max(resid[i], resid_c[i]) (NaN kept), i < 2N
cudaError_t launch_max_merge(int* iters, const int* iters_c, float* resid, const float* resid_c, int N,
                             cudaStream_t st);
cudaError_t launch_block_polyphase(const float* x, const float* w, int L, int ntap, long long nb, float* xs,
                                   cudaStream_t st);
cudaError_t launch_upchan(const UpchanSrc& src, int L, long long nblocks, float2* out, float* x_out,
                          cudaStream_t st);
// Two-pass up-channelizer of the column-pair scratch (k4a: d2 -> W, then k4b: W ->
// spectra), upfactor 64, lblock 1024/2048/4096; W holds nblocks * 32 N complex values.
// k4a reads d2 in the block-major layout that k3 writes with out_block_major = 1:
// frame j of pair p at d2[p J + 64 (j >> 6) + 8 (j & 7) + ((j >> 3) & 7)].
bool upchan2_supported(int N, int C, int U);
cudaError_t launch_k4a(const float2* d2, int N, int J, long long nblocks, float2* W, float* x_out,
                       cudaStream_t st);
cudaError_t launch_k4b(const float2* W, int N, long long nblocks, float2* out, cudaStream_t st);

// ---- ML solve with the CG vectors in HBM (columns longer than the on-chip run)
// Every vector is [P C][S] in the column transform's residue layout: frame j = C m + r
// of pair p at v[(p C + r) S + m], columns 2p and 2p+1 as the real and imaginary parts.
struct MlbPair {
  double rz[2];    // r.z of each column's current residual
  float bn[2];     // |b| (1 where b = 0)
  float beta[2];
  float rel[2];    // recursive relative residual at the last test
  float apend[2];  // alpha of the last iteration, whose x += alpha p is still to be applied
  int act;         // bit c: column 2p + c still iterating
  int it[2];
  int pbuf;        // the search-direction buffer that holds that p
};
struct MlbBufs {
  float2 *B, *X, *R, *Q, *Z;  // Q holds d until the right-hand side is built; Z = R without a preconditioner
  float2* Pv[2];              // search direction, read from one and written to the other
  uint8_t* mk;                // mask bits per pair-frame (bit c: column 2p + c saved)
  float2* acoef;              // [P][16] stencil taps a_s / sigma^2 of both columns
  double* part;               // [P][NT][8] per-tile partial sums
  double* rzk;                // [P][8][2] r.z of both columns from each CTA of the preconditioner
  double* rrk;                // [P][8][2] r.r of both columns from each CTA of the fused update
  MlbPair* ps;                // [P]
  float* lam_m;               // [N] lam * mask fraction of each column
  int* list;                  // [P] active pairs, ascending
  int* ctl;                   // [0] active pairs, [1] iterations done, [2] block ticket
};
struct MlbGeom {
  int N, C, S, logC;
  int TM, logTM, NT;  // tile: TM positions of all C residues (TF = C TM frames), NT tiles per pair
};
MlbGeom mlb_geom(int N, int C, int S);
size_t mlb_workspace(int N, int C, int S);
MlbBufs mlb_carve(void* ws, int N, int C, int S);
// mask, prior, initial guess (time order [J][N]) -> mask bits, lam m prior (in B), X
cudaError_t launch_mlb_transpose(const uint8_t* mask, const float* prior, const float* x0, float lam,
                                 const MlbGeom& g, const MlbBufs& b, cudaStream_t st);
// b = C^T d / sigma^2 + lam m prior, r0 = b - A x0, [Z = r0]; per-tile |b|^2, mask counts, r.r
cudaError_t launch_mlb_rhs(const float* window, const MLParams& mp, const MlbGeom& g, const MlbBufs& b,
                           cudaStream_t st);
// |b|, lam mbar, all pairs listed, counters cleared
cudaError_t launch_mlb_init(const MLParams& mp, const MlbGeom& g, const MlbBufs& b, cudaStream_t st);
// x += apend p (the previous iteration's step, p in Pv[src]), p' = z + beta p
// (Pv[src] -> Pv[src ^ 1]), q = A p', per-tile p'.q (listed pairs)
cudaError_t launch_mlb_ap(int src, const MLParams& mp, const MlbGeom& g, const MlbBufs& b, cudaStream_t st);
// without a preconditioner: alpha, r -= alpha q, per-tile r.r (listed pairs)
cudaError_t launch_mlb_xr(const MLParams& mp, const MlbGeom& g, const MlbBufs& b, cudaStream_t st);
// stopping test, beta, iteration counts, the next list; sets h (if set_cond) to "a pair is listed"
cudaError_t launch_mlb_ctl(int first, int set_cond, cudaGraphConditionalHandle h, const MLParams& mp,
                           const MlbGeom& g, const MlbBufs& b, cudaStream_t st);
// x = X + apend p (each pair's last step) written to Q, its true residual b - A x,
// iterations and residuals out
cudaError_t launch_mlb_finish(const MLParams& mp, const MlbGeom& g, const MlbBufs& b, int* iters, float* resid,
                              cudaStream_t st);

// ---- learned preconditioner: flexible CG state and the net
struct FcgCol;
struct FcgBufs {
  float2 *X, *R, *P, *Z, *U;  // [P][J] column-pair vectors
  FcgCol* cs;                 // [N] per-column state
  float* Y;                   // [N][J] net outputs (request slots)
  float* netin;               // [N][2][J] net inputs (request slots)
  uint32_t* mb;               // [P][fcg_threads(J)] prior-mask bits of each thread's frames
};
// threads per column pair of the flexible-CG kernels (16 frames per thread)
constexpr int fcg_threads(int J) { return J / 16 < 32 ? 32 : (J / 16 > 512 ? 512 : J / 16); }
size_t fcg_col_bytes();
cudaError_t launch_fcg_step(int J, int phase, const float2* d2, const FcgBufs& b, const uint8_t* mask,
                            const float* prior, const float* window, int N, const MLParams& mp, int* counter,
                            cudaStream_t st);
// Wiener-preconditioned CG on chip (k5_ml_cg, mp.max_iter iterations, initial guess in
// b.X in frame order when mp.use_x0) whose state is handed over to the flexible-CG
// kernels: X, R, P, Z and the mask bits lane-interleaved, the per-column state in b.cs
// (a column stays active below fcg_max_iter iterations); resumed by fcg step phase 3.
// A pair with no active column is finished in the kernel instead: its solution in
// frame order in b.X, its iters / resid entries written, b.cs marked done (pad = 1).
cudaError_t launch_k5_handover(int J, const float2* d2, const uint8_t* mask, const float* prior,
                               const float* window, int N, const MLParams& mp, const FcgBufs& b, int fcg_max_iter,
                               int* iters, float* resid, cudaStream_t st);
// device-side control of the learned solve's graph: the loop condition (a column still
// active and fewer than max_trips trips) and the plain-CG fallback condition (a
// non-finite residual among the 2 N values, or a net that gave up waiting)
cudaError_t launch_fcg_loop_ctrl(const FcgBufs& b, int ncols, int* trips, int max_trips,
                                 cudaGraphConditionalHandle h, cudaStream_t st);
cudaError_t launch_fcg_fallback_check(const float* resid, int n2, const int* net_status, int* flag,
                                      cudaGraphConditionalHandle h, cudaStream_t st);
cudaError_t launch_fcg_finish(int J, const float2* d2, const FcgBufs& b, const uint8_t* mask, const float* prior,
                              const float* window, int N, const MLParams& mp, int* iters, float* resid,
                              cudaStream_t st);
cudaError_t launch_net_pairs(int J, const float2* xs, const float2* xk, const int* pl, int npairs,
                             const uint8_t* mask, const float* window, int N, const MLParams& mp, float* xin,
                             float* target, cudaStream_t st);
size_t net_pack_bytes();
int net_nparams();
long long net_bwd_items(int nslots, int J);
long long net_fwd_items(int nslots, int J);
cudaError_t launch_net_pack(const float* theta, uint8_t* packed, cudaStream_t st);
// wait_limit < 0: the default bound on the accumulator wait (about a second);
// status (or nullptr) is set nonzero by a CTA that gave up waiting
cudaError_t launch_net_forward(const uint8_t* packed, const float* in, float* y, int J, int nslots_host,
                               const int* count, int* zero_other, int max_slots, long long wait_limit, int* status,
                               cudaStream_t st);
cudaError_t launch_net_backward(const uint8_t* packed, const float* in, const float* target, int J, int nslots,
                                float inv_n, float* part, cudaStream_t st);
cudaError_t launch_net_reduce(const float* part, long long nitems, float* grad, float* loss, cudaStream_t st);
cudaError_t launch_adam(float* theta, float* m, float* v, const float* g, int n, float lr, float beta1, float beta2,
                        float eps, float c1, float c2, cudaStream_t st);

}  // namespace ipfb
