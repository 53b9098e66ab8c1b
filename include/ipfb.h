/*
 * libipfb — circulant inverse polyphase filter bank on one B300 (sm_103a).
 *
 * Method: "Inverting and Up-channelizing Critically-Sampled Polyphase Filter
 * Banks" (arXiv 2608.23441).  Section / equation names below refer to it.
 *
 * Conventions shared by every entry point
 *   N = lblock (real samples per frame), p = ntap, J = nframes (spectra);
 *   T = J*N samples; C = N/2 + 1 real-FFT channels.
 *   DFT sign: forward exp(-2 pi i n k / N) (Sec. 2.3, operator F).
 *   Complex arrays are interleaved float pairs (re, im), i.e. float2.
 *   Time-ordered streams: x[j*N + n] = sample n of frame j.
 *   Window: float [p][N], w[r][n] = h[r*N + n] (Sec. 2.3 "reshape into [p, N]").
 *   4-bit codes: folded layout, N/2 bytes per spectrum: byte c (0 < c < N/2) =
 *     Re_c (low nibble) | Im_c (high nibble), two's complement in [-7, 7];
 *     byte 0 = Re_0 (low) | Re_{N/2} (high).  DC and Nyquist have no
 *     imaginary part in a real PFB, so nothing is lost.  Code arrays read by
 *     the inverse calls must start on a 16-byte boundary (they are read with
 *     16-byte loads); an unaligned pointer is refused with IPFB_ERR_INVALID.
 *
 * Ownership: every array pointer is owned by the caller.  Unless stated
 *   otherwise pointers are DEVICE pointers on the current CUDA device.  The
 *   library allocates no device memory: scratch comes from the caller (size
 *   from ipfb_workspace_size), 256-byte aligned.
 * Execution: every compute call is asynchronous on `stream` (a cudaStream_t
 *   passed as void*; NULL = legacy default stream).  Host-side argument checks
 *   run before anything is enqueued.
 * Errors: 0 on success, a negative IPFB_ERR_* code otherwise; nothing is
 *   enqueued when a check fails.  A launch failure returns IPFB_ERR_CUDA and
 *   the CUDA error string is available from ipfb_last_cuda_error().
 */
#ifndef IPFB_H
#define IPFB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IPFB_OK 0
#define IPFB_ERR_INVALID (-1)       /* null pointer, bad size, bad flag          */
#define IPFB_ERR_UNSUPPORTED (-2)   /* valid, but outside the built kernel range */
#define IPFB_ERR_WORKSPACE (-3)     /* workspace smaller than required           */
#define IPFB_ERR_NOT_CONVERGED (-4) /* iterative solve hit max_iter              */
#define IPFB_ERR_TIMEOUT (-5)       /* a bounded device wait gave up             */
#define IPFB_ERR_CUDA (-6)          /* a CUDA runtime call failed                */

/* operation ids for ipfb_workspace_size */
#define IPFB_OP_FORWARD 1
#define IPFB_OP_WIENER 2
#define IPFB_OP_WIENER_UPCHAN 3
#define IPFB_OP_ML 4
#define IPFB_OP_ML_LEARNED 5 /* ipfb_ml_solve with precond = 2        */
#define IPFB_OP_ML_PAIRS 6   /* ipfb_ml_training_pairs                 */
#define IPFB_OP_WIENER_STREAM 7 /* ipfb_wiener_stream (nframes = chunk) */
#define IPFB_OP_ML_STREAM 8     /* ipfb_ml_solve_stream (nframes = chunk) */

typedef struct {
  int lblock;   /* N: power of two, 32 <= N <= 16384                              */
  int ntap;     /* p: 1 <= p <= 16                                                 */
  int nframes;  /* J: spectra (= input frames for a periodic PFB); power of two,
                   16 <= J <= 65536 for the inverse                               */
  int periodic; /* 1: spectrum j uses frames j..j+p-1 mod J (the circulant model) */
} ipfb_geom;

/* Human-readable text for a status code (static storage). */
const char* ipfb_strerror(int status);
/* Text of the last CUDA error seen by this library in this thread ("" if none). */
const char* ipfb_last_cuda_error(void);
/* Library ABI version (major*100 + minor). */
int ipfb_version(void);

/*
 * Testing knob (no counterpart in the paper): the longest run of frames one CTA
 * transforms along a column (8192 by default; 512 is also accepted).  Columns
 * longer than the run are split over a thread-block cluster of up to 8 CTAs, and
 * ipfb_ml_solve (precond 0, 1) keeps their CG vectors in HBM instead of on chip, so
 * a small run exercises both paths on small inputs.  Process-wide; it also decides
 * ipfb_workspace_size's answer for IPFB_OP_ML and IPFB_OP_ML_STREAM.
 */
int ipfb_set_max_column_run(int frames);

/*
 * Testing knob (no counterpart in the paper): the bound, in SM clocks, on the net
 * forward's wait for its tensor-core accumulators (ipfb_net_forward and the learned
 * solve).  cycles < 0 restores the built-in bound of about a second.  With a bound
 * shorter than the MMAs take, every CTA gives up at once: it marks its tile's output,
 * reports the give-up to the learned solve, lets its MMAs in flight finish (within the
 * built-in bound) and stops, so the expiry path runs without anything being withheld.
 * Process-wide.
 */
int ipfb_set_net_wait_limit(long long cycles);

/*
 * Stage timing (no counterpart in the paper).  ipfb_stage_timing(1) clears the
 * record and starts bracketing every kernel launch of every compute call with two
 * CUDA events on that call's stream; ipfb_stage_timing(0) clears and stops.
 * ipfb_stage_times waits for the recorded events and writes, per kernel name, the
 * summed milliseconds and the launch count: names_csv receives the names in
 * order, comma separated (HOST buffer of names_cap bytes); ms / counts are HOST
 * arrays of max_entries.  Returns the number of names (>= 0) or an error code.
 */
int ipfb_stage_timing(int enable);
int ipfb_stage_times(char* names_csv, size_t names_cap, double* ms, int* counts, int max_entries);

/* Bytes of device scratch needed by operation `op` for geometry g (0 if none). */
int ipfb_workspace_size(const ipfb_geom* g, int op, size_t* bytes);

/*
 * Sinc x Hamming PFB window (Sec. 2.2, Eq. chan_dft read as sinc((m - M/2)/N);
 * App. A: Hamming with the cos(2 pi m/(M-1)) normalisation), M = ntap*lblock:
 *   w[m] = sinc((m - M/2)/N) * (0.54 - 0.46 cos(2 pi m / (M - 1))).
 * Computed on the host in double, rounded to float.  window_host: HOST float [M].
 */
int ipfb_sinc_hamming_window(int lblock, int ntap, float* window_host);

/*
 * Forward critically-sampled PFB with 4-bit quantization (Eq. pfb; Sec. 4.3).
 *   d[j, n] = sum_{r<p} w[r][n] x[((j + r) mod J) N + n]        (periodic)
 *   Y[j, c] = sum_n d[j, n] exp(-2 pi i n c / N),   c <= N/2
 *   scale_c = RMS_c / 2.5 with RMS_c over the real and imaginary parts of
 *     channel c (DC, Nyquist: real parts only), accumulated in FP64, rounded
 *     once to float; used as given when scale_in != NULL.
 *   code = clamp(rint(v / scale_c), -7, 7) on Re and Im (float32 IEEE divide,
 *     round half to even; scale 0 gives code 0).
 * x: float [J*N]; window: float [p][N]; scale_in: float [C] or NULL;
 * codes: uint8 [J][N/2] (folded); scale_out: float [C] (may equal scale_in);
 * spectra_out: float2 [J][C] or NULL.  Only periodic = 1 is supported.
 */
int pfb_forward(const ipfb_geom* g, const float* x, const float* window, const float* scale_in,
                uint8_t* codes, float* scale_out, float* spectra_out, void* ws, size_t ws_bytes,
                void* stream);

/*
 * pfb_forward without a workspace (the paper has no counterpart: this is a
 * calling convention, not part of the method).  Same computation and outputs as
 * pfb_forward with scale_in = NULL.  For callers that cannot give the library a
 * scratch buffer: streaming ingest code that reserves all device memory at
 * start-up and must not allocate afterwards (cudaMalloc can synchronize the
 * device and stall the stream), or host frameworks that only pass in the buffers
 * they own.  The FP64 power sums live in a fixed array inside the library sized
 * for lblock <= 16384 (131 KB held on every GPU that loads the library, until the
 * process exits); larger lblock returns IPFB_ERR_UNSUPPORTED before anything is
 * enqueued.  No device memory is allocated.  Every call looks up the array's
 * address on the current device (cudaGetSymbolAddress, a host-side query), so a
 * device reset between calls is harmless; the first call on a device also loads
 * the library's device code there, so make it before any stream capture.  All
 * calls share the array: each clears it on its own stream, and calls that overlap
 * on the GPU (other streams or host threads on the same device) race on it --
 * serialize them.  CUDA failures return IPFB_ERR_CUDA with the failing step named
 * in ipfb_last_cuda_error().
 */
int pfb_forward_noalloc(const ipfb_geom* g, const float* x, const float* window, uint8_t* codes,
                        float* scale_out, float* spectra_out, void* stream);

/*
 * The quantize-and-pack step alone (Sec. 4.3 quantizer) on given spectra:
 * spectra: float2 [nspec][lblock/2 + 1]; scale: float [lblock/2 + 1];
 * codes: uint8 [nspec][lblock/2].  Same decision rule as pfb_forward.
 */
int pfb_quantize(int lblock, int nspec, const float* spectra, const float* scale, uint8_t* codes,
                 void* stream);

/*
 * Circulant inverse PFB with Wiener filtering (Sec. 3.1 Eq. decorrelation,
 * Sec. 4.1 Eq. wiener weights, App. C):
 *   d = N-point inverse real FFT of (codes x scale) per spectrum  ("undo F")
 *   per column n: D_n = FFT_J(d[:, n]); W_n(k) = sum_r w[r][n] e^{-2 pi i r k/J}
 *   x_hat_n = IFFT_J( G D_n ),  G = W_n (1 + phi^2) / (|W_n|^2 + phi^2)
 *   (= H_n / conj(W_n)); noise_level = phi^2 (= N/S); noise_level = 0 is the
 *   exact inverse 1/conj(W_n) (modes with W_n == 0 exactly are dropped).
 *   normalize = 0 drops the optional (1 + phi^2) factor.
 * codes: uint8 [J][N/2]; scale: float [C]; window: float [p][N];
 * x_out: float [J*N], time order.  Requires periodic = 1 (J spectra -> J frames).
 * Workspace: ipfb_workspace_size(g, IPFB_OP_WIENER).
 */
int ipfb_wiener(const ipfb_geom* g, const uint8_t* codes, const float* scale, const float* window,
                double noise_level, int normalize, float* x_out, void* ws, size_t ws_bytes,
                void* stream);

/*
 * ipfb_filter: the circulant inverse PFB of ipfb_wiener with another eigenvalue filter
 * on the frame-axis modes (Sec. 3.2: the circulant form exposes every eigenmode, so
 * any per-mode filter costs the same as the Wiener one).  Per column n and mode k
 * the reconstruction multiplies the column spectrum by G_n(k):
 *   mode IPFB_FILTER_THRESHOLD: thresholded pseudo-inverse, G = 1 / conj W_n(k) where
 *     |W_n(k)| >= threshold (threshold >= 0), G = 0 elsewhere; threshold 0 is the
 *     exact inverse.  |W|^2 below 1e-4 is evaluated in FP64, the keep-or-drop decision
 *     included; above that it is decided in FP32.
 *   mode IPFB_FILTER_GAINS: caller gains, a DEVICE array of complex float pairs
 *     (re, im) laid out [N][J/2 + 1]: gains[n (J/2 + 1) + k] = G_n(k) for k <= J/2;
 *     G_n(J - k) = conj G_n(k) (real output), 8-byte aligned.  The 1/J of the inverse
 *     transform is applied by the library.
 * codes, scale, window, x_out as for ipfb_wiener (same sizes, same workspace:
 * ipfb_workspace_size(g, IPFB_OP_WIENER)).  Errors: IPFB_ERR_INVALID for an unknown
 * mode, a negative or non-finite threshold, or a null / unaligned gains array.
 */
#define IPFB_FILTER_THRESHOLD 1
#define IPFB_FILTER_GAINS 2
int ipfb_filter(const ipfb_geom* g, const uint8_t* codes, const float* scale, const float* window, int mode,
                double threshold, const float* gains, float* x_out, void* ws, size_t ws_bytes, void* stream);

/*
 * Up-channelization (Sec. 4.3, re-channelization with frames `block` samples
 * long; read here as a plain real DFT of consecutive blocks, no window):
 *   X_b[c] = sum_{t<L} x[b L + t] exp(-2 pi i t c / L),  c <= L/2,
 *   b < floor(nsamples / L); a trailing partial block is ignored.
 * x: float [nsamples] time order; out: float2 [nsamples/L][L/2 + 1].
 * L: power of two, 1024 <= L <= 262144.
 */
int upchannelize(const float* x, int64_t nsamples, int64_t block, float* out, void* ws,
                 size_t ws_bytes, void* stream);

/*
 * ipfb_wiener_stream: overlap-save inverse of a run of nspec spectra longer than one
 * circulant block (App. C: the Wiener decorrelation kernels are tens of frames long,
 * so a chunk inverted as if periodic is exact up to the kernel's tail beyond the
 * margin).  g->nframes is the chunk length J (power of two); chunks of J spectra step
 * by S = J - 2 margin, the last one aligned to the end of the run; each is inverted
 * as ipfb_wiener does and its frames margin .. J - margin are kept.
 * codes: uint8 [nspec][N/2] (16-byte aligned; N/2 a multiple of 16), scale: float
 * [N/2 + 1] of the whole run, window: float [p][N]; x_out: float
 * [(nspec - 2 margin) N], frames margin .. nspec - margin - 1 in time order.
 * 0 <= margin, J - 2 margin >= 1, nspec >= J.  The first and last `margin` frames
 * of the run have no context on one side and are not produced.
 * Workspace: ipfb_workspace_size(g, IPFB_OP_WIENER_STREAM), 16-byte aligned.
 */
int ipfb_wiener_stream(const ipfb_geom* g, int64_t nspec, const uint8_t* codes, const float* scale,
                       const float* window, double noise_level, int normalize, int margin, float* x_out, void* ws,
                       size_t ws_bytes, void* stream);

/*
 * Windowed re-channelization (Sec. 4.3: the inverted stream "channelized again using
 * a PFB with 64-times longer frame size"): a PFB with frames L = block samples long
 * and p = ntap taps, periodic over the nb = floor(nsamples / L) blocks:
 *   s_b[t] = sum_{r<p} window[r L + t] x[((b + r) mod nb) L + t],   X_b = rfft_L(s_b).
 * x: float [nsamples] time order; window: float [p][L] (e.g. ipfb_sinc_hamming_window
 * with lblock = L); out: float2 [nb][L/2 + 1].  L: power of two, 1024 <= L <= 262144;
 * 1 <= ntap <= 64.  Workspace: nb * L floats (the summed blocks).  x, window and ws
 * must start on a 16-byte boundary.
 */
int upchannelize_pfb(const float* x, int64_t nsamples, int64_t block, int ntap, const float* window, float* out,
                     void* ws, size_t ws_bytes, void* stream);

/*
 * ipfb_wiener followed by upchannelize with block = upfactor * lblock, without
 * a round trip of the reconstructed stream through time order.  x_out (time
 * order) is optional (NULL = not written).  out: float2 [J/upfactor][L/2 + 1].
 * Workspace: ipfb_workspace_size(g, IPFB_OP_WIENER_UPCHAN) (2 J N floats: the
 * column-pair scratch and the up-channelizer's intermediate); it must start on a
 * 16-byte boundary (the up-channelizer moves it with 16-byte copies), else
 * IPFB_ERR_INVALID.
 */
int ipfb_wiener_upchannelize(const ipfb_geom* g, const uint8_t* codes, const float* scale,
                             const float* window, double noise_level, int normalize,
                             int upfactor, float* out, float* x_out, void* ws, size_t ws_bytes,
                             void* stream);

/*
 * Maximum-likelihood inverse PFB with a time-domain prior (Sec. 4.2,
 * Eq. chi squared), by conjugate gradient on the per-column normal equations
 *   (C_n^T C_n / sigma^2 + lam M_n) x_n = C_n^T d_n / sigma^2 + lam M_n p_n
 * with d = N-point inverse real FFT of (codes x scale) ("undo F"), the circulant
 * sub-filter correlation (C x)[j] = sum_r w[r][n] x[(j + r) mod J], sigma^2 =
 * noise_var, lam = prior_weight, M_n = the prior mask of column n, p = prior values.
 * C^T C is applied as its exact circular (2p-1)-tap stencil; inner products are
 * reduced in FP64, vectors are FP32.  Each column stops on its own when
 * ||b - A x|| / ||b|| <= tol (recursively updated residual), or after max_iter.
 * precond: 0 none; 1 Wiener, z = F^dagger[F r / (|W_n|^2/sigma^2 + lam mean(M_n))];
 * 2 learned: net = device pointer to the net parameters (float [IPFB_NET_NPARAMS],
 * see ipfb_net_forward), z = u + lam mean(M_n) M_W(s g(u/s, m)) with u = M_W r the
 * Wiener z above, M_W that Wiener step, s = RMS(u) over the column (1 if u = 0), m
 * the column's prior mask; the outer iteration is then flexible CG (Notay 2000) with
 * the Polak-Ribiere beta r_new.(z_new - z_old) / r_old.z_old.  The first net_from
 * applications use u alone: with net_from >= 1 those iterations (Wiener-PCG) run in
 * the on-chip CG kernel, which hands x, r, p, z and r.z over to the flexible-CG
 * kernels for the columns still active.  precond 2 requires ntap = 4; its workspace
 * is ipfb_workspace_size(g, IPFB_OP_ML_LEARNED).  It is enqueued as one CUDA graph
 * whose loop (two launches per iteration) is ended on the device once no column is
 * active, so the call neither synchronizes nor reads anything back: when `stream` is
 * capturing, the graph's nodes (conditional WHILE and IF nodes among them) join the
 * caller's capture; otherwise the library captures it privately, launches it on
 * `stream` and releases it.  If any column ends with a non-finite residual (a net
 * that returns NaN or Inf), or the net gave up waiting for its accumulators, the
 * solve is redone on the device by plain CG (precond 0) from the same start, and
 * x_inout, iters and resid are plain CG's.
 * prior_mask: uint8 [J*N] time order (nonzero = saved sample); prior_values:
 * float [J*N]; x_inout: float [J*N], the initial guess when use_x0 != 0 (else
 * zero is used), the solution on return.  iters: int [N] iterations per column;
 * resid: float [2][N], recursive then true relative residual per column (the
 * true one recomputed from the final x).  Non-convergence is reported through
 * these arrays (the call itself returns 0).  Requires 128 <= J (a power of two);
 * precond 0 and 1 take J up to 65536, precond 2 up to 8192.  Columns up to the
 * on-chip run (8192 frames) are solved by one CTA per column pair with the vectors
 * in shared memory and registers; longer ones keep the CG vectors in HBM in the
 * column transform's residue layout (J = C S, C = 2, 4, 8), iterate as one CUDA graph
 * whose loop is ended on the device (no host synchronisation, capturable like
 * precond 2), take the Wiener step through the cluster column transform and drop
 * converged column pairs from each iteration's work.
 * Workspace: ipfb_workspace_size(g, IPFB_OP_ML): 2 J N floats up to the on-chip run,
 * else about 28 J N bytes (seven pair-packed vectors, the mask bits, small state).
 */
typedef struct {
  double noise_var;    /* sigma^2 (> 0) in units of d                        */
  double prior_weight; /* lam >= 0 (1 in the paper)                           */
  double tol;          /* relative residual target per column (e.g. 1e-6)     */
  int max_iter;        /* iteration cap per column                            */
  int precond;         /* 0 none, 1 Wiener, 2 learned                         */
  int net_from;        /* learned: iterations that use the Wiener step alone
                          before the net joins (>= 0; 0 = from the start)     */
} ipfb_ml_params;

int ipfb_ml_solve(const ipfb_geom* g, const uint8_t* codes, const float* scale, const float* window,
                  const ipfb_ml_params* prm, const uint8_t* prior_mask, const float* prior_values,
                  const void* net, float* x_inout, int use_x0, int* iters, float* resid, void* ws,
                  size_t ws_bytes, void* stream);

/*
 * ipfb_ml_solve_stream: the ML reconstruction of ipfb_ml_solve (precond 0 or 1) for a
 * run of nspec spectra longer than one solve, overlap-save like ipfb_wiener_stream
 * (Sec. 4.2 solved block by block; the solution's dependence on data far away decays
 * along the frame axis, so a chunk solved as if periodic agrees with the solve of the
 * whole run away from the chunk's edges).  g->nframes is the chunk length J
 * (128 <= J <= 65536, a power of two); chunks of J spectra step by J - 2 margin, the
 * last one aligned to the end of the run; each is solved with its own stretch of
 * prior_mask, prior_values and (when x0 != NULL) initial guess x0, and its frames
 * margin .. J - margin are kept.  codes: uint8 [nspec][N/2] (16-byte aligned; N/2 a
 * multiple of 16); scale: float [N/2 + 1] of the whole run; window: float [p][N];
 * prior_mask: uint8 [nspec*N]; prior_values, x0: float [nspec*N], time order;
 * x_out: float [(nspec - 2 margin) N], frames margin .. nspec - margin - 1; iters:
 * int [N] and resid: float [2][N], the largest over the chunks of ipfb_ml_solve's
 * per-column counts and residuals.  0 <= margin, J - 2 margin >= 1, nspec >= J;
 * precond 2 returns IPFB_ERR_UNSUPPORTED.  Workspace:
 * ipfb_workspace_size(g, IPFB_OP_ML_STREAM).
 */
int ipfb_ml_solve_stream(const ipfb_geom* g, int64_t nspec, const uint8_t* codes, const float* scale,
                         const float* window, const ipfb_ml_params* prm, const uint8_t* prior_mask,
                         const float* prior_values, const float* x0, int margin, float* x_out, int* iters,
                         float* resid, void* ws, size_t ws_bytes, void* stream);

/*
 * Learned preconditioner net.  The paper has no learned component: this is the
 * learned variant of the Sec. 4.2 solve.  Per column (a sequence of J frames) a
 * 1-D convolutional net along the frame axis with circular padding:
 *   a1 = GELU(conv(x0, w1) + b1)   2 -> 32 channels, 9 taps
 *   a2 = GELU(conv(a1, w2) + b2)   32 -> 32
 *   y  = conv(a2, w3) + b3         32 -> 1
 * conv(x, w)[co][j] = sum_{ci,t} w[co][ci][t] x[ci][(j + t - 4) mod J];
 * GELU(x) = x Phi(x) = 0.5 x (1 + erf(x / sqrt 2)).
 * theta: device float [IPFB_NET_NPARAMS] = w1[32][2][9], b1[32], w2[32][32][9],
 * b2[32], w3[1][32][9], b3[1].  Weights and the activations x0, a1, a2 are rounded
 * to BF16 (nearest even) and every convolution accumulates in FP32 on the tensor
 * cores; biases, GELU and the loss are FP32.
 * xin: device float [nslots][2][J] (channel 0 = u/s, channel 1 = mask);
 * y, target: device float [nslots][J].
 *
 * ipfb_net_forward: y = net(xin).  Workspace ipfb_net_workspace_size(IPFB_NET_FORWARD).
 *   Layer 2 waits for its tensor-core accumulators with a bound of about a second
 *   of SM clocks (ipfb_set_net_wait_limit); a CTA that gives up writes NaN at the
 *   first output frame of its tile, waits for its MMAs in flight and stops (a
 *   learned solve then falls back to plain CG).  The call itself returns 0: the
 *   status is in y.
 * ipfb_net_grad: loss = sum over slots and frames of (y - target)^2 / (nslots J)
 *   (device float [1], may be NULL) and its gradient with respect to theta
 *   (device float [IPFB_NET_NPARAMS], may be NULL), the BF16 rounding of weights
 *   and activations treated as the identity in the backward pass; partial sums
 *   are reduced in a fixed order, so results are deterministic.
 *   Workspace ipfb_net_workspace_size(IPFB_NET_GRAD).
 * ipfb_net_adam: one Adam step (Kingma and Ba 2015) on theta with moment buffers
 *   m, v (device float [n], zero before step 1); step counts from 1.
 * ipfb_ml_training_pairs: training examples for the net from two iterates of a
 *   solve with the same operator (g, window, prm: noise_var, prior_weight): for
 *   each listed column pair i (pair_index: HOST int [npairs], npairs <= N/2, each
 *   0 <= p < N/2, checked before anything is enqueued; pair p = columns 2p, 2p+1)
 *   and h = 0, 1: e = x_star - x_k, r = A e, u = M_W r, s = RMS(u),
 *   xin[2i+h] = (u/s, mask), target[2i+h] = (e - u)/s, i.e. what the net has to
 *   add so that z = u + s g = A^{-1} r.  x_star, x_k: device float [J*N] time
 *   order.  Requires ntap = 4.  Workspace ipfb_workspace_size(g, IPFB_OP_ML_PAIRS).
 */
#define IPFB_NET_NPARAMS 10145
#define IPFB_NET_FORWARD 1
#define IPFB_NET_GRAD 2

int ipfb_net_nparams(void);
int ipfb_net_workspace_size(int op, int nslots, int nframes, size_t* bytes);
int ipfb_net_forward(const float* theta, int nslots, int nframes, const float* xin, float* y, void* ws,
                     size_t ws_bytes, void* stream);
int ipfb_net_grad(const float* theta, int nslots, int nframes, const float* xin, const float* target, float* loss,
                  float* grad, void* ws, size_t ws_bytes, void* stream);
int ipfb_net_adam(float* theta, float* m, float* v, const float* grad, int n, int step, double lr, double beta1,
                  double beta2, double eps, void* stream);
int ipfb_ml_training_pairs(const ipfb_geom* g, const float* window, const ipfb_ml_params* prm,
                           const uint8_t* prior_mask, const float* x_star, const float* x_k, const int* pair_index,
                           int npairs, float* xin, float* target, void* ws, size_t ws_bytes, void* stream);

/*
 * Batched inverse PFB of many independent streams of uneven shape (lblock in
 * {1024, 2048, 4096}, any integer number of frames 1024 <= J <= 16384), each the
 * Wiener inverse of ipfb_wiener (Eq. decorrelation, Eq. wiener weights).  The
 * J-point column DFT for arbitrary J uses Bluestein's chirp-z identity with
 * FFTs of length M on thread-block clusters, M the smallest of the powers of two,
 * 20480 and 24576 that is >= 2J - 1 (the two non-powers of two only above 16384); the
 * work (spectra groups, column pairs, output tiles) is pulled from counters by
 * persistent kernels, longest items first.
 *
 * ipfb_batched_plan builds the host-side plan (no device work) and returns the
 * workspace size; tune_cache (a file path, or NULL) supplies per-M kernel
 * variants written by ipfb_batched_autotune.  ipfb_batched_prepare uploads the
 * descriptors (from host arrays the plan owns until ipfb_batched_free) and builds the
 * chirp and FFT(chirp) tables in the workspace, asynchronously on `stream`; its
 * copies come from pageable host memory, so it cannot be captured in a CUDA graph
 * (replan and prepare outside the capture).  ipfb_batched_run enqueues the
 * inversion (a counter reset and the persistent kernels, no host
 * synchronization); after a prepare with the same workspace it can be captured
 * in a CUDA graph and replayed.  ipfb_batched_autotune times every kernel
 * variant per M class on the plan's own work items, keeps the fastest, and
 * writes the choice to cache_path (if not NULL); it overwrites the outputs.
 * ipfb_batched_variant reports the variant chosen for M (a power of two from 2048
 * to 32768, or 20480 / 24576, whose kernels are fixed).  Stream descriptors:
 * device pointers codes [J][N/2], scale [N/2+1], window [ntap][N], x_out [J*N].
 */
typedef struct {
  int lblock;
  int ntap;
  int nframes;
  const uint8_t* codes;
  const float* scale;
  const float* window;
  double noise_level; /* phi^2 of this stream */
  float* x_out;
} ipfb_stream_desc;

int ipfb_batched_plan(const ipfb_stream_desc* streams, int nstreams, int normalize, const char* tune_cache,
                      void** plan, size_t* ws_bytes);
int ipfb_batched_prepare(void* plan, void* ws, size_t ws_bytes, void* stream);
int ipfb_batched_run(void* plan, void* ws, size_t ws_bytes, void* stream);
int ipfb_batched_autotune(void* plan, void* ws, size_t ws_bytes, void* stream, const char* cache_path);
int ipfb_batched_variant(void* plan, int M, char* name, size_t cap);
int ipfb_batched_free(void* plan);

#ifdef __cplusplus
}
#endif

#endif /* IPFB_H */
