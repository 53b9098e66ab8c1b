// Forward-PFB kernels: polyphase sum + real FFT + per-channel RMS, then 4-bit
// quantization and packing (Eq. pfb, Sec. 2.3; quantizer of Sec. 4.3).
#pragma once

#include "common.cuh"

namespace ipfb {

// Real N-point FFT (N = 2H) of the polyphase sum of frame j as an H-point complex
// FFT of z[m] = d[2m] + i d[2m+1]; the polyphase sum is formed while loading:
//   z[m] = sum_r (w[r][2m], w[r][2m+1]) * (x[(j+r) mod J][2m], x[(j+r) mod J][2m+1]).
// Result: Z[k] in sm (natural order, padded).
// NT > 0: the tap count is a compile-time constant (NT == ntap), so the 2 NT loads
// of each element are independent and issued together; NT == 0: any ntap.
template <int H, int TPF, int NT>
__device__ __forceinline__ void frame_rfft_core(const float2* __restrict__ x2, const float2* __restrict__ w2,
                                                int ntap, int J, int j, float2* sm, int tid) {
  auto ldp = [=](int m) {
    float2 acc = make_float2(0.0f, 0.0f);
    if constexpr (NT > 0) {
      float2 xv[NT], wv[NT];
#pragma unroll
      for (int r = 0; r < NT; ++r) {
        int jj = j + r;
        if (jj >= J) jj -= J;  // J >= NT
        xv[r] = x2[(size_t)jj * H + m];
        wv[r] = __ldg(w2 + (size_t)r * H + m);
      }
#pragma unroll
      for (int r = 0; r < NT; ++r) {
        acc.x = fmaf(wv[r].x, xv[r].x, acc.x);
        acc.y = fmaf(wv[r].y, xv[r].y, acc.y);
      }
    } else {
      int jj = j;
      for (int r = 0; r < ntap; ++r) {
        const float2 xv = x2[(size_t)jj * H + m];
        const float2 wv = __ldg(w2 + (size_t)r * H + m);
        acc.x = fmaf(wv.x, xv.x, acc.x);
        acc.y = fmaf(wv.y, xv.y, acc.y);
        jj = (jj + 1 == J) ? 0 : jj + 1;
      }
    }
    return acc;
  };
  block_fft<H, TPF, false>(sm, tid, fn_ld(ldp), SPad{sm});
}

// The polyphase sums of the F consecutive frames jb .. jb+F-1 of a CTA, for a
// compile-time tap count NT: each element m loads the F + NT - 1 rows it needs once
// (instead of NT rows per frame) and the NT window values once, then writes the F
// sums z_f[m] into the frames' padded buffers (frame f at smem + f * stride).
template <int H, int F, int NT, int NTH>
__device__ __forceinline__ void polyphase_group(const float2* __restrict__ x2, const float2* __restrict__ w2,
                                                int J, int jb, float2* smem, int stride) {
  constexpr int NR = F + NT - 1;
  for (int m = threadIdx.x; m < H; m += NTH) {
    float2 xr[NR], wv[NT];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      int jj = jb + r;
      while (jj >= J) jj -= J;
      xr[r] = x2[(size_t)jj * H + m];
    }
#pragma unroll
    for (int t = 0; t < NT; ++t) wv[t] = __ldg(w2 + (size_t)t * H + m);
#pragma unroll
    for (int f = 0; f < F; ++f) {
      float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        acc.x = fmaf(wv[t].x, xr[f + t].x, acc.x);
        acc.y = fmaf(wv[t].y, xr[f + t].y, acc.y);
      }
      smem[f * stride + pidx(m)] = acc;
    }
  }
}

// Polyphase sum + H-point complex FFT of the CTA's frames: with a compile-time tap
// count the sums of all F frames are formed together first; otherwise each frame's
// first FFT pass forms its own sums while loading.
template <int H, int TPF, int F, int NT>
__device__ __forceinline__ void frames_rfft(const float2* __restrict__ x2, const float2* __restrict__ w2, int ntap,
                                            int J, int jb, float2* smem, int tid, int f) {
  float2* sm = smem + f * padded_len(H);
  if constexpr (NT > 0) {
    polyphase_group<H, F, NT, TPF * F>(x2, w2, J, jb, smem, padded_len(H));
    __syncthreads();
    block_fft<H, TPF, false>(sm, tid, SPad{sm}, SPad{sm});
  } else {
    const int j = jb + f;
    frame_rfft_core<H, TPF, 0>(x2, w2, ntap, J, j < J ? j : 0, sm, tid);
  }
}

// Post-processing of the half-length FFT into the real-input spectrum:
//   E = (Z[k] + conj Z[H-k])/2, O = (Z[k] - conj Z[H-k])/(2i),
//   Y[k] = E + e^{-2 pi i k/N} O,   Y[H-k] = conj(E) - e^{+2 pi i k/N} conj(O)... (see below)
// Computes Y[k] and Y[H-k] for k in [0, H/2]; k = 0 also gives Y[H] (Nyquist).
__device__ __forceinline__ void rfft_post(const float2* sm, int H, int k, const Twid2<7>& tw, float2& yk,
                                          float2& ym) {
  const int km = H - k;
  const float2 zk = sm[pidx(k)];
  const float2 zm = sm[pidx(km == H ? 0 : km)];
  const float2 E = cscale(cadd(zk, cconj(zm)), 0.5f);
  const float2 dd = csub(zk, cconj(zm));
  const float2 O = make_float2(0.5f * dd.y, -0.5f * dd.x);  // dd / (2i)
  const float2 w = tw(k);                                     // e^{-2 pi i k / N}
  yk = cadd(E, cmul(w, O));
  // at H-k: E' = conj(E), O' = conj(O), twiddle e^{-2 pi i (H-k)/N} = -conj(w)
  ym = csub(cconj(E), cmul(cconj(w), cconj(O)));
}

// Pass A: per-channel sums of Re^2 and Im^2 over all spectra (FP64 atomics at the
// end of each CTA).  CTA processes frames blockIdx.x*F + f, stepping gridDim.x*F.
template <int H, int TPF, int F, int NT>
__global__ void __launch_bounds__(TPF* F, 2)
k1_pfb_power(const float* __restrict__ x, const float* __restrict__ window, int ntap, int J,
             double* __restrict__ sums /* [2][H+1] */) {
  extern __shared__ float2 smem[];
  constexpr int KPT = (H / 2 + TPF) / TPF;  // channels k in [0, H/2] per thread
  const int f = threadIdx.x / TPF, tid = threadIdx.x % TPF;
  float2* sm = smem + f * padded_len(H);
  const float2* x2 = reinterpret_cast<const float2*>(x);
  const float2* w2 = reinterpret_cast<const float2*>(window);
  float2* tw_hi = smem + F * padded_len(H);
  twid2_fill<7, false>(tw_hi, tw_hi + 128, 2 * H, threadIdx.x, TPF * F);
  const Twid2<7> tw{tw_hi, tw_hi + 128};
  float re_k[KPT], im_k[KPT], re_m[KPT], im_m[KPT];
#pragma unroll
  for (int i = 0; i < KPT; ++i) re_k[i] = im_k[i] = re_m[i] = im_m[i] = 0.0f;
  for (int jb = blockIdx.x * F; jb < J; jb += gridDim.x * F) {
    const int j = jb + f;
    const bool live = j < J;
    frames_rfft<H, TPF, F, NT>(x2, w2, ntap, J, jb, smem, tid, f);
    __syncthreads();
    if (live) {
#pragma unroll
      for (int i = 0; i < KPT; ++i) {
        const int k = tid + i * TPF;
        if (k <= H / 2) {
          float2 yk, ym;
          rfft_post(sm, H, k, tw, yk, ym);
          re_k[i] = fmaf(yk.x, yk.x, re_k[i]);
          im_k[i] = fmaf(yk.y, yk.y, im_k[i]);
          re_m[i] = fmaf(ym.x, ym.x, re_m[i]);
          im_m[i] = fmaf(ym.y, ym.y, im_m[i]);
        }
      }
    }
    __syncthreads();
  }
  // reduce the F frame groups through smem, then one FP64 atomic per value
  float* red = reinterpret_cast<float*>(smem);  // [F][4][H/2+1]
  const int L = H / 2 + 1;
#pragma unroll
  for (int i = 0; i < KPT; ++i) {
    const int k = tid + i * TPF;
    if (k <= H / 2) {
      red[(f * 4 + 0) * L + k] = re_k[i];
      red[(f * 4 + 1) * L + k] = im_k[i];
      red[(f * 4 + 2) * L + k] = re_m[i];
      red[(f * 4 + 3) * L + k] = im_m[i];
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 4 * L; idx += TPF * F) {
    const int q = idx / L, k = idx % L;
    float s = 0.0f;
    for (int ff = 0; ff < F; ++ff) s += red[(ff * 4 + q) * L + k];
    // q: 0 re(k), 1 im(k), 2 re(H-k), 3 im(H-k)
    const int c = (q < 2) ? k : H - k;
    if (q >= 2 && (c == k)) continue;  // k == H/2 counted once
    atomicAdd(&sums[(q & 1) * (H + 1) + c], (double)s);
  }
}

// scale_c = RMS_c / 2.5 from the FP64 sums, rounded once to float.
__global__ void k1_scale_from_sums(const double* __restrict__ sums, int H, int J, float* __restrict__ scale) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c > H) return;
  const double re2 = sums[c], im2 = sums[(H + 1) + c];
  double rms;
  if (c == 0 || c == H)
    rms = sqrt(re2 / (double)J);
  else
    rms = sqrt((re2 + im2) / (2.0 * (double)J));
  scale[c] = (float)(rms / 2.5);
}

// Quantizer decision on float32 (v, scale): clamp(rint(v / s), -7, 7), s == 0 -> 0.
__device__ __forceinline__ int quant4(float v, float s) {
  if (s == 0.0f) return 0;
  float q = rintf(__fdiv_rn(v, s));
  q = fminf(fmaxf(q, -7.0f), 7.0f);
  return (int)q;
}
// The same decision from a precomputed reciprocal r = 1/s (correctly rounded): d =
// v r lies within 1.5 2^-23 |v/s| of the rounded quotient fl(v/s), so for |d| < 8
// the two round to the same integer unless d is within 3e-6 of a half-integer
// (then the exact quotient is formed); |d| >= 8 clamps to +-7 either way.
__device__ __forceinline__ int quant4r(float v, float s, float r) {
  if (s == 0.0f) return 0;
  const float d = v * r;
  float q = rintf(d);
  if (fabsf(d) < 8.0f && 0.5f - fabsf(d - q) < 3.0e-6f) q = rintf(__fdiv_rn(v, s));
  q = fminf(fmaxf(q, -7.0f), 7.0f);
  return (int)q;
}
__device__ __forceinline__ uint8_t pack2(int lo, int hi) {
  return (uint8_t)((lo & 0xF) | ((hi & 0xF) << 4));
}

// Pass B: recompute spectra, quantize, pack (and optionally write spectra).
template <int H, int TPF, int F, int NT>
__global__ void __launch_bounds__(TPF* F, 2)
k1_pfb_quant(const float* __restrict__ x, const float* __restrict__ window, int ntap, int J,
             const float* __restrict__ scale, uint8_t* __restrict__ codes, float2* __restrict__ spectra) {
  extern __shared__ float2 smem[];
  const int f = threadIdx.x / TPF, tid = threadIdx.x % TPF;
  float2* sm = smem + f * padded_len(H);
  const float2* x2 = reinterpret_cast<const float2*>(x);
  const float2* w2 = reinterpret_cast<const float2*>(window);
  float2* tw_hi = smem + F * padded_len(H);
  twid2_fill<7, false>(tw_hi, tw_hi + 128, 2 * H, threadIdx.x, TPF * F);
  const Twid2<7> tw{tw_hi, tw_hi + 128};
  // reciprocal steps 1/scale[c], c <= H (0 where the step is 0), once per CTA
  float* rstep = reinterpret_cast<float*>(tw_hi + 256);
  for (int c = threadIdx.x; c <= H; c += TPF * F) rstep[c] = scale[c] == 0.0f ? 0.0f : __frcp_rn(scale[c]);
  for (int jb = blockIdx.x * F; jb < J; jb += gridDim.x * F) {
    const int j = jb + f;
    const bool live = j < J;
    frames_rfft<H, TPF, F, NT>(x2, w2, ntap, J, jb, smem, tid, f);
    __syncthreads();
    if (live) {
      uint8_t* row = codes + (size_t)j * H;
      float2* srow = spectra ? spectra + (size_t)j * (H + 1) : nullptr;
      for (int k = tid; k <= H / 2; k += TPF) {
        float2 yk, ym;
        rfft_post(sm, H, k, tw, yk, ym);
        const int km = H - k;
        if (k == 0) {
          row[0] = pack2(quant4r(yk.x, scale[0], rstep[0]), quant4r(ym.x, scale[H], rstep[H]));
          if (srow) {
            srow[0] = make_float2(yk.x, 0.0f);
            srow[H] = make_float2(ym.x, 0.0f);
          }
        } else {
          const float sk = scale[k], rk = rstep[k];
          row[k] = pack2(quant4r(yk.x, sk, rk), quant4r(yk.y, sk, rk));
          if (km != k) {
            const float sm_ = scale[km], rm = rstep[km];
            row[km] = pack2(quant4r(ym.x, sm_, rm), quant4r(ym.y, sm_, rm));
          }
          if (srow) {
            srow[k] = yk;
            if (km != k) srow[km] = ym;
          }
        }
      }
    }
    __syncthreads();
  }
}

// Quantize given spectra (float2 [nspec][H+1]) with the same rule.
__global__ void k_quantize(const float2* __restrict__ spec, const float* __restrict__ scale, int H,
                           long long nspec, uint8_t* __restrict__ codes) {
  const long long total = nspec * H;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long j = idx / H;
    const int c = (int)(idx % H);
    const float2* row = spec + j * (H + 1);
    if (c == 0)
      codes[idx] = pack2(quant4(row[0].x, scale[0]), quant4(row[H].x, scale[H]));
    else
      codes[idx] = pack2(quant4(row[c].x, scale[c]), quant4(row[c].y, scale[c]));
  }
}

}  // namespace ipfb
