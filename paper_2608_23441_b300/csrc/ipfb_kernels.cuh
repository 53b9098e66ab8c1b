// Inverse-PFB kernels (Sec. 3.1, Sec. 4.1, App. C).
//
// Scratch layout "d2" (column-pair, residue-major), shared by the iPFB, the ML
// solve and the up-channelizer:  columns 2p and 2p+1 of the [J, N] polyphase
// array are packed as one complex sequence z_p[j] = d[j, 2p] + i d[j, 2p+1];
// with J = C*S (C = CTAs per column cluster) frame j = C*m + r is stored at
//     d2[(p*C + r)*S + m]          (float2)
// so each of the C CTAs that transform column pair p reads and writes one
// contiguous S-element run.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"
#include "launch.h"

namespace ipfb {
namespace cg = cooperative_groups;

// ----------------------------------------------------------------------------
// K2: 4-bit unpack x scale  ->  N-point inverse real FFT per spectrum ("undoing F")
// ----------------------------------------------------------------------------
// One CTA inverts F spectra j = C*m + r, m in [m0, m0+F), with TPF threads per
// spectrum.  The real inverse FFT of length N = 2H runs as an H-point complex
// inverse FFT of Z[k] = E[k] + i O[k] with
//     E[k] = (Y[k] + conj Y[H-k]) / 2,  O[k] = (Y[k] - conj Y[H-k]) e^{+2 pi i k/N} / 2,
// so that z[m] = x[2m] + i x[2m+1] -- exactly the column-pair value of pair m.
// The 1/H normalisation is folded into the pre-scale.
// frame stride in smem (float2): padded length rounded to 4 (mod 16), so that the
// F interleaved frames of the transposed store fall in distinct banks
__host__ __device__ constexpr int k2_frame_stride(int H) { return ((padded_len(H) + 15) / 16) * 16 + 4; }

// One group of F spectra (frames C*(m0 + f) + r, f < nvalid) -> d2.  Called by every
// thread of the CTA (TPF*F threads); smem holds F frame buffers plus 256 twiddles.
template <int H, int TPF, int F>
__device__ __forceinline__ void k2_group(const uint8_t* __restrict__ codes, const float* __restrict__ scale,
                                         float2* __restrict__ d2, int C, int S, int r, int m0, int nvalid,
                                         float2* smem) {
  const int f = threadIdx.x / TPF;
  const int tid = threadIdx.x % TPF;
  float2* sm = smem + f * k2_frame_stride(H);
  const bool live = f < nvalid;
  const float pre = 0.5f / (float)H;
  // exp(+2 pi i k / N), N = 2H, from two tables of 128 entries shared by the CTA
  float2* tw_hi = smem + F * k2_frame_stride(H);
  float2* tw_lo = tw_hi + 128;
  // the F code rows (H bytes each) and the H+1 channel steps, staged with 16-byte loads
  uint8_t* crow = reinterpret_cast<uint8_t*>(tw_lo + 128);
  float* sscale = reinterpret_cast<float*>(crow + F * H);
  twid2_fill<7, true>(tw_hi, tw_lo, 2 * H, threadIdx.x, TPF * F);
  {
    constexpr int V = H / 16;  // 16-byte vectors per row
    for (int i = threadIdx.x; i < F * V; i += TPF * F) {
      const int ff = i / V, c = i % V;
      if (ff < nvalid) {
        const size_t jj = (size_t)C * (m0 + ff) + r;
        reinterpret_cast<uint4*>(crow + ff * H)[c] = reinterpret_cast<const uint4*>(codes + jj * H)[c];
      }
    }
    for (int i = threadIdx.x; i <= H; i += TPF * F) sscale[i] = scale[i] * pre;  // 1/(2H) folded in
  }
  __syncthreads();
  const Twid2<7> tw{tw_hi, tw_lo};
  const uint8_t* row = crow + f * H;

  // pre-processing: Z[k] and Z[H-k] for k in [0, H/2], four consecutive k per step
  // (one 4-byte load of codes k..k+3, two of the mirror bytes H-k-3..H-k, float4
  // loads of the steps and the twiddles).  With d = Y[k] - conj Y[H-k]:
  //   E = Y[k] + conj Y[H-k],  O = d w,  Z[k] = E + i O,  Z[H-k] = conj E + i conj O
  // (w = e^{+2 pi i k/N}; the 1/2 and 1/H are in the staged steps).  A nibble q
  // (two's complement) becomes a float exactly as (2^23 + (q ^ 8)) - (2^23 + 8).
  auto nib = [](uint32_t v, int hi) -> float {
    return __uint_as_float(((hi ? v >> 4 : v) & 0xFu) ^ 0x4B000008u) - 8388616.0f;
  };
  auto emit = [&](int k, float2 yk, float2 ym, float2 w) {
    const float2 e = cadd(yk, cconj(ym));
    const float2 o = cmul(csub(yk, cconj(ym)), w);
    sm[pidx(k)] = make_float2(e.x - o.y, e.y + o.x);
    if (k != 0 && 2 * k != H) sm[pidx(H - k)] = make_float2(e.x + o.y, o.x - e.y);
  };
  for (int g = tid; live && g < H / 8; g += TPF) {
    const int k0 = 4 * g;
    const uint32_t cw = *reinterpret_cast<const uint32_t*>(row + k0);
    const uint32_t mlo = *reinterpret_cast<const uint32_t*>(row + (H - k0 - 4));  // bytes H-k0-4 .. H-k0-1
    const uint32_t mhi = g ? row[H - k0] : 0u;                                     // byte H-k0
    const float4 sk = *reinterpret_cast<const float4*>(sscale + k0);
    const float4 smv = *reinterpret_cast<const float4*>(sscale + (H - k0 - 4));
    const float sm0 = sscale[H - k0];  // g = 0: the Nyquist step
    const float2 th = tw_hi[k0 >> 7];
    const float4 tl01 = *reinterpret_cast<const float4*>(tw_lo + (k0 & 127));
    const float4 tl23 = *reinterpret_cast<const float4*>(tw_lo + (k0 & 127) + 2);
    const float skj[4] = {sk.x, sk.y, sk.z, sk.w};
    const float smj[4] = {sm0, smv.w, smv.z, smv.y};
    const uint32_t bmj[4] = {mhi, mlo >> 24, mlo >> 16, mlo >> 8};
    const float2 tlj[4] = {make_float2(tl01.x, tl01.y), make_float2(tl01.z, tl01.w), make_float2(tl23.x, tl23.y),
                           make_float2(tl23.z, tl23.w)};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t bk = cw >> (8 * j);
      float2 yk, ym;
      if (j == 0 && g == 0) {  // DC and Nyquist share byte 0
        yk = make_float2(nib(bk, 0) * skj[0], 0.0f);
        ym = make_float2(nib(bk, 1) * smj[0], 0.0f);
      } else {
        yk = make_float2(nib(bk, 0) * skj[j], nib(bk, 1) * skj[j]);
        ym = make_float2(nib(bmj[j], 0) * smj[j], nib(bmj[j], 1) * smj[j]);
      }
      emit(k0 + j, yk, ym, cmul(th, tlj[j]));
    }
  }
  if (live && tid == 0) {  // k = H/2, its own mirror
    const uint32_t bk = row[H / 2];
    const float2 y = make_float2(nib(bk, 0) * sscale[H / 2], nib(bk, 1) * sscale[H / 2]);
    emit(H / 2, y, y, tw(H / 2));
  }
  __syncthreads();
  block_fft<H, TPF, true>(sm, tid, SPad{sm}, SPad{sm});
  __syncthreads();
  // transposed store: for each pair p, the valid consecutive m of residue r
  for (int idx = threadIdx.x; idx < H * F; idx += TPF * F) {
    const int p = idx / F, ff = idx % F;
    if (ff < nvalid) d2[((size_t)p * C + r) * S + m0 + ff] = smem[ff * k2_frame_stride(H) + pidx(p)];
  }
}

template <int H, int TPF, int F>
__global__ void __launch_bounds__(TPF* F)
k2_unpack_irfft(const uint8_t* __restrict__ codes, const float* __restrict__ scale,
                float2* __restrict__ d2, int C, int S) {
  extern __shared__ float2 smem[];
  const int per_res = S / F;
  const int r = blockIdx.x / per_res;
  const int m0 = (blockIdx.x % per_res) * F;
  k2_group<H, TPF, F>(codes, scale, d2, C, S, r, m0, F, smem);
}

// ----------------------------------------------------------------------------
// Gain per frame-axis mode (Eq. decorrelation with Eq. wiener weights):
//   W_n(k) = sum_t w[t, n] e^{-2 pi i t k / J}
//   G = W gnorm / (|W|^2 + phi^2) / J      (phi^2 = 0, gnorm = 1: 1/conj(W) / J)
// |W|^2 below kFp64Below is recomputed in FP64 (near-zero eigenvalues, App. A).
// An exactly zero denominator gives G = 0 (the mode is dropped).
// ----------------------------------------------------------------------------
constexpr float kFp64Below = 1e-4f;
constexpr int kMaxTaps = 16;

// FP64 re-evaluation of one gain where |W|^2 is tiny (near-zero eigenvalues of
// nearly symmetric windows, App. A).  Kept out of line: it runs for a few modes per
// million, and inlining its FP64 code into the FP32 loop slows every mode.
static __device__ __noinline__ float2 gain_fp64(const float* taps, int ntap, int k, GainParams gp) {
  double s, c;
  sincospi(2.0 * (double)k / (double)gp.J, &s, &c);
  double wx = 0.0, wy = 0.0;
  for (int t = ntap - 1; t >= 0; --t) {
    const double nx = wx * c + wy * s;  // (wx + i wy)(c - i s)
    const double ny = wy * c - wx * s;
    wx = nx + (double)taps[t];
    wy = ny;
  }
  const double den = wx * wx + wy * wy + (double)gp.phi2;
  if (den == 0.0) return make_float2(0.0f, 0.0f);
  const double g = (double)gp.gnorm * (double)gp.invJ / den;
  return make_float2((float)(wx * g), (float)(wy * g));
}

template <int NT>
__device__ __forceinline__ float2 gain_at(const float* taps, int k, float2 e1, const GainParams& gp) {
  // Horner in e1 = e^{-2 pi i k/J}.  NT > 0: exactly NT taps (compile time);
  // NT == 0: gp.ntap <= kMaxTaps taps, loop unrolled with a uniform guard.
  constexpr int NMAX = NT > 0 ? NT : kMaxTaps;
  float2 W = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int t = NMAX - 1; t >= 0; --t) {
    if (NT > 0 || t < gp.ntap) {
      W = cmul(W, e1);
      W.x += taps[t];
    }
  }
  const float a2 = fmaf(W.x, W.x, W.y * W.y);
  if (a2 < kFp64Below) return gain_fp64(taps, NT > 0 ? NT : gp.ntap, k, gp);
  const float g = __fdividef(gp.gnorm * gp.invJ, a2 + gp.phi2);
  return make_float2(W.x * g, W.y * g);
}

// Filters other than Wiener (GainParams::mode 1, 2), for the generic-tap kernels:
//   1: thresholded pseudo-inverse G = W / |W|^2 / J where |W|^2 >= thresh2, else 0
//      (|W|^2 below kFp64Below is formed in FP64, decision included);
//   2: caller gains G = gains[col][k] / J for k <= J/2, conj(gains[col][J - k]) / J above.
static __device__ __noinline__ float2 pinv_gain_fp64(const float* taps, int ntap, int k, const GainParams& gp) {
  double s, c;
  sincospi(2.0 * (double)k / (double)gp.J, &s, &c);
  double wx = 0.0, wy = 0.0;
  for (int t = ntap - 1; t >= 0; --t) {
    const double nx = wx * c + wy * s;
    const double ny = wy * c - wx * s;
    wx = nx + (double)taps[t];
    wy = ny;
  }
  const double a2 = wx * wx + wy * wy;
  if (!(a2 >= (double)gp.thresh2) || a2 == 0.0) return make_float2(0.0f, 0.0f);
  const double g = (double)gp.invJ / a2;
  return make_float2((float)(wx * g), (float)(wy * g));
}

template <int NT>
__device__ __forceinline__ float2 filter_gain(const float* taps, int k, float2 e1, const GainParams& gp, int col) {
  if constexpr (NT == 0) {
    if (gp.mode == 1) {
      float2 W = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int t = kMaxTaps - 1; t >= 0; --t) {
        if (t < gp.ntap) {
          W = cmul(W, e1);
          W.x += taps[t];
        }
      }
      const float a2 = fmaf(W.x, W.x, W.y * W.y);
      if (a2 < kFp64Below) return pinv_gain_fp64(taps, gp.ntap, k, gp);
      if (a2 < gp.thresh2) return make_float2(0.0f, 0.0f);
      const float g = __fdividef(gp.invJ, a2);
      return make_float2(W.x * g, W.y * g);
    }
    if (gp.mode == 2) {
      const int half = gp.J / 2;
      const float2 G = __ldg(gp.gains + (size_t)col * (half + 1) + (k <= half ? k : gp.J - k));
      return make_float2(G.x * gp.invJ, (k <= half ? G.y : -G.y) * gp.invJ);
    }
  }
  return gain_at<NT>(taps, k, e1, gp);
}

// Column-pair split, per-column gain, recombination for modes k and -k:
//   A = (Z_k + conj Z_-k)/2, B = (Z_k - conj Z_-k)/(2i)      (spectra of columns a, b)
//   Z'_k = Ga A + i Gb B,   Z'_-k = conj(Ga A) + i conj(Gb B)
__device__ __forceinline__ void split_gain(float2& zk, float2& zm, float2 ga, float2 gb) {
  const float2 A = cscale(cadd(zk, cconj(zm)), 0.5f);
  const float2 d = csub(zk, cconj(zm));
  const float2 B = make_float2(0.5f * d.y, -0.5f * d.x);
  const float2 ya = cmul(ga, A), yb = cmul(gb, B);
  zk = cadd(ya, cmul_i(yb));
  zm = cadd(cconj(ya), cmul_i(cconj(yb)));
}

// The same for a compile-time tap count NT > 0, in one step: W_a and W_b share the
// powers of e1, and the split, the gains and the recombination fold into
//   s = Z_k + conj Z_-k,  d = Z_k - conj Z_-k,  P = (Ga/2) s,  Q = (Gb/2) d,
//   Z'_k = P + Q,  Z'_-k = conj(P - Q).
// Where either |W|^2 falls below kFp64Below both gains come from gain_at.
template <int NT>
__device__ __forceinline__ void pair_gain(float2& zk, float2& zm, const float* ta, const float* tb, int k,
                                          float2 e1, const GainParams& gp) {
  static_assert(NT > 0, "compile-time tap count");
  float2 ep[NT];
  ep[0] = make_float2(1.0f, 0.0f);
  if constexpr (NT > 1) ep[1] = e1;
#pragma unroll
  for (int q = 2; q < NT; ++q) ep[q] = cmul(ep[q / 2], ep[q - q / 2]);
  float2 Wa = make_float2(ta[0], 0.0f), Wb = make_float2(tb[0], 0.0f);
#pragma unroll
  for (int q = 1; q < NT; ++q) {
    Wa.x = fmaf(ta[q], ep[q].x, Wa.x);
    Wa.y = fmaf(ta[q], ep[q].y, Wa.y);
    Wb.x = fmaf(tb[q], ep[q].x, Wb.x);
    Wb.y = fmaf(tb[q], ep[q].y, Wb.y);
  }
  const float a2a = fmaf(Wa.x, Wa.x, Wa.y * Wa.y), a2b = fmaf(Wb.x, Wb.x, Wb.y * Wb.y);
  float2 Ga, Gb;
  if (fminf(a2a, a2b) < kFp64Below) {
    Ga = cscale(gain_at<NT>(ta, k, e1, gp), 0.5f);
    Gb = cscale(gain_at<NT>(tb, k, e1, gp), 0.5f);
  } else {
    const float half = 0.5f * gp.gnorm * gp.invJ;
    Ga = cscale(Wa, __fdividef(half, a2a + gp.phi2));
    Gb = cscale(Wb, __fdividef(half, a2b + gp.phi2));
  }
  const float2 sv = make_float2(zk.x + zm.x, zk.y - zm.y);
  const float2 dv = make_float2(zk.x - zm.x, zk.y + zm.y);
  const float2 P = cmul(Ga, sv), Q = cmul(Gb, dv);
  zk = cadd(P, Q);
  zm = make_float2(P.x - Q.x, Q.y - P.y);
}

// Gain policy of K3 (k3_pair): load(), the forward local FFT of step 1; pair() and
// single(), the per-mode step on modes k and -k of both columns of pair p; finish(),
// after the cross stage.  WienerGain applies the eigenvalue filter of GainParams (Wiener
// in one fused step for a compile-time tap count; any filter mode with the generic
// taps); the ML solve's preconditioner policy lives with its kernel (k3_ml.cuh).
template <int NT>
struct WienerGain {
  __device__ __forceinline__ static void pair(float2& zk, float2& zm, const float* ta, const float* tb, int k,
                                              float2 e1, const GainParams& gp, int p) {
    if constexpr (NT > 0) {
      pair_gain<NT>(zk, zm, ta, tb, k, e1, gp);
    } else {
      const float2 ga = filter_gain<NT>(ta, k, e1, gp, 2 * p), gb = filter_gain<NT>(tb, k, e1, gp, 2 * p + 1);
      split_gain(zk, zm, ga, gb);
    }
  }
  __device__ __forceinline__ static void single(float2& a, float2& b, const float* ta, const float* tb, int k,
                                                float2 e1, const GainParams& gp, int p, bool self) {
    (void)self;
    const float2 ga = filter_gain<NT>(ta, k, e1, gp, 2 * p), gb = filter_gain<NT>(tb, k, e1, gp, 2 * p + 1);
    split_gain(a, b, ga, gb);
  }
  __device__ __forceinline__ static void finish(const GainParams&, int) {}
  // step 1's forward local FFT: this CTA's run of the pair, global -> smem
  template <int S, int T>
  __device__ __forceinline__ static void load(float2* sm, int tid, float2* base, const GainParams&, int, size_t) {
    block_fft<S, T, false>(sm, tid, GMem{base}, SPad{sm});
  }
};

// ----------------------------------------------------------------------------
// K3: per column pair: FFT_J along frames -> gain -> inverse FFT_J, in place on d2.
// A cluster of C CTAs handles one pair; CTA r owns z[C m + r], m < S.
//   1. local S-point FFT:      U_r[kb] = sum_m z[Cm + r] e^{-2 pi i m kb / S}
//   2. cross stage (DSMEM):    Z[kb + S ka] = sum_r e^{-2 pi i r ka / C} e^{-2 pi i r kb/J} U_r[kb]
//   3. gains on modes k and -k; -k of (kb, ka) is (S-kb, C-1-ka) (kb != 0), so one
//      thread owns both and nothing crosses CTAs between 2 and 4
//   4. inverse cross stage, pushed back to the owners, then local inverse FFT.
// ----------------------------------------------------------------------------
template <int C, int S, int T, int NT, class GAIN, class GP>
__device__ __forceinline__ void k3_pair(float2* __restrict__ d2, const float* __restrict__ window, int N, GP gp,
                                        const int p) {
  extern __shared__ float2 sm[];
  const int tid = threadIdx.x;
  int r = 0;
  if constexpr (C > 1) r = (int)cg::this_cluster().block_rank();
  float2* base = d2 + ((size_t)p * C + r) * S;
  const int J = C * S;

  constexpr int NMAX = NT > 0 ? NT : kMaxTaps;
  float ta[NMAX], tb[NMAX];
#pragma unroll
  for (int t = 0; t < NMAX; ++t) {
    ta[t] = (t < gp.ntap) ? __ldg(window + (size_t)t * N + 2 * p) : 0.0f;
    tb[t] = (t < gp.ntap) ? __ldg(window + (size_t)t * N + 2 * p + 1) : 0.0f;
  }

  // 1. forward local FFT: global -> smem
  GAIN gn;
  gn.template load<S, T>(sm, tid, base, gp, p, ((size_t)p * C + r) * S);
  if constexpr (C > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }

  // peer q's shared array (mapped on use, to keep the addresses out of registers)
  auto peer = [](int q) -> float2* {
    if constexpr (C > 1)
      return cg::this_cluster().map_shared_rank(sm, q);
    else
      return sm;
  };

  // 2-4. tasks t < S/2: the pair (t, S - t); t = 0 takes the two self-paired groups
  // kb = 0 and kb = S/2 together (each holds C modes whose partners lie in the same
  // group, so together they weigh one pair task, and the S/2 tasks fill the C T
  // threads' slots evenly instead of leaving one thread a third task)
  for (int t = r * T + tid; t < S / 2; t += C * T) {
    const bool pairtask = t != 0;
    const int kb0 = t, kb1 = pairtask ? S - t : S / 2;
    float2 z0[C], z1[C];
    float2 w0[C];
    // gather + cross-stage twiddle + C-point DFT over r.  The twiddle of kb1 = S - kb0
    // is e^{-2 pi i q (S - kb0)/J} = e^{-2 pi i q / C} conj(w0[q]); for kb0 = 0 it is 1,
    // and kb1 = S/2 takes its own.
    if constexpr (C > 1) twiddle_powers<C>(twiddle<false>(pairtask ? kb0 : S / 2, J), w0);
#pragma unroll
    for (int q = 0; q < C; ++q) {
      z0[q] = peer(q)[pidx(kb0)];
      z1[q] = peer(q)[pidx(kb1)];
    }
    if constexpr (C > 1) {
#pragma unroll
      for (int q = 1; q < C; ++q) {
        if (pairtask) {
          z0[q] = cmul(z0[q], w0[q]);
          z1[q] = rotq<C, false>(cmul(z1[q], cconj(w0[q])), q);
        } else {
          z1[q] = cmul(z1[q], w0[q]);
        }
      }
      DFT<C, false>::run(z0);
      DFT<C, false>::run(z1);
    }
    // gains: z0[ka] is mode k = kb0 + S*ka, e^{-2 pi i k/J} = e0 e^{-2 pi i ka/C} (e0 of
    // kb = S/2 in the t = 0 task)
    float2 e0;
    if constexpr (C > 1)
      e0 = w0[1];
    else
      e0 = twiddle<false>(pairtask ? kb0 : S / 2, J);
    if (pairtask) {
#pragma unroll
      for (int ka = 0; ka < C; ++ka) {
        const int k = kb0 + S * ka;
        const float2 e1 = rotq<C, false>(e0, ka);
        gn.pair(z0[ka], z1[C - 1 - ka], ta, tb, k, e1, gp, p);
      }
    } else {
      // kb = 0 in z0: modes S*ka; -k is S*((C-ka) mod C)
#pragma unroll
      for (int ka = 0; ka <= C / 2; ++ka) {
        const int km = (C - ka) % C;
        const int k = S * ka;
        const float2 e1 = rotq<C, false>(make_float2(1.0f, 0.0f), ka);
        float2 a = z0[ka], b = z0[km];
        gn.single(a, b, ta, tb, k, e1, gp, p, km == ka);
        z0[ka] = a;
        if (km != ka) z0[km] = b;
      }
      // kb = S/2 in z1: modes S/2 + S*ka; -k is S/2 + S*(C-1-ka)
#pragma unroll
      for (int ka = 0; ka < (C + 1) / 2; ++ka) {
        const int km = C - 1 - ka;
        const int k = S / 2 + S * ka;
        const float2 e1 = rotq<C, false>(e0, ka);
        float2 a = z1[ka], b = z1[km];
        gn.single(a, b, ta, tb, k, e1, gp, p, km == ka);
        z1[ka] = a;
        if (km != ka) z1[km] = b;
      }
    }
    // inverse C-point DFT over ka, conj twiddle, push back to owner q
    if constexpr (C > 1) {
      DFT<C, true>::run(z0);
      DFT<C, true>::run(z1);
#pragma unroll
      for (int q = 1; q < C; ++q) {
        if (pairtask) {
          z0[q] = cmul(z0[q], cconj(w0[q]));
          z1[q] = rotq<C, true>(cmul(z1[q], w0[q]), q);
        } else {
          z1[q] = cmul(z1[q], cconj(w0[q]));
        }
      }
    }
#pragma unroll
    for (int q = 0; q < C; ++q) {
      peer(q)[pidx(kb0)] = z0[q];
      peer(q)[pidx(kb1)] = z1[q];
    }
  }
  if constexpr (C > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
  gn.finish(gp, p * C + r);
  // 4. inverse local FFT: smem -> global, in place over this CTA's input run, or (for
  // the up-channelizer) in place over the pair's J frames in block-major order: frame
  // j at 64 (j >> 6) + 8 (j & 7) + ((j >> 3) & 7), i.e. each 64-frame block contiguous
  // with its 8 residues as runs of 8.  Every CTA of the cluster has read its input
  // before the cluster barrier above, so the reordering cannot overwrite unread data.
  const bool bm = gp.out_block_major != 0;
  float2* pbase = d2 + (size_t)p * J;
  block_fft<S, T, true>(sm, tid, SPad{sm}, fn_st([=](int m, float2 v) {
    if (bm) {
      const int j = C * m + r;
      pbase[64 * (j >> 6) + 8 * (j & 7) + ((j >> 3) & 7)] = v;
    } else {
      base[m] = v;
    }
  }));
}

template <int C, int S, int T, int NT>
__global__ void __launch_bounds__(T, (S >= 4096 ? 2 : 1))
k3_column_wiener(float2* __restrict__ d2, const float* __restrict__ window, int N, GainParams gp) {
  k3_pair<C, S, T, NT, WienerGain<NT>, GainParams>(d2, window, N, gp, blockIdx.x / C);
}

// ----------------------------------------------------------------------------
// d2 (column-pair, residue-major) -> time-ordered x[j*N + n]
// Tile: TJ consecutive frames x 32 pairs.
// ----------------------------------------------------------------------------
template <int TJ>
__global__ void __launch_bounds__(256)
k_pairs_to_time(const float2* __restrict__ d2, float* __restrict__ x, int N, int C, int S) {
  __shared__ float2 tile[TJ][33];
  const int H = N / 2;
  const int p0 = blockIdx.x * 32;
  const int j0 = blockIdx.y * TJ;
  // load: for pair p0+pp, frames j0..j0+TJ-1
  for (int idx = threadIdx.x; idx < 32 * TJ; idx += 256) {
    const int pp = idx / TJ, jj = idx % TJ;
    const int j = j0 + jj;
    const int p = p0 + pp;
    if (p < H) tile[jj][pp] = d2[((size_t)p * C + (j % C)) * S + j / C];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 32 * TJ; idx += 256) {
    const int jj = idx / 32, pp = idx % 32;
    const int p = p0 + pp;
    if (p < H) reinterpret_cast<float2*>(x + (size_t)(j0 + jj) * N)[p] = tile[jj][pp];
  }
}

}  // namespace ipfb
