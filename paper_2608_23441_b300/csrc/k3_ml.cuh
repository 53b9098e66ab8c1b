// Launch helper for K3 with the ML solve's preconditioner gain (k3_column_ml) on the
// residue splits of the HBM-resident ML solve (C = 2, 4, 8; S = 512 or 8192).
#pragma once

#include "ipfb_kernels.cuh"
#include "launch.h"

namespace ipfb {
// First-pass accessor of the fused CG update: element i of the CTA's run is
// r_i - alpha q_i, written back to r and added to the CTA's r.r (each element is read
// once by the first pass)
struct MlResidLoad {
  float2* rp;
  const float2* qp;
  float aa, ab;
  float* rr;
  template <int R, int NB>
  __device__ __forceinline__ int lbase(int b) const { return b; }
  template <int R, int NB>
  __device__ __forceinline__ float2 ld(int base, int r) const {
    const int i = base + r * NB;
    float2 v = rp[i];
    const float2 q = __ldg(qp + i);
    v.x = fmaf(-aa, q.x, v.x);
    v.y = fmaf(-ab, q.y, v.y);
    rp[i] = v;
    rr[0] = fmaf(v.x, v.x, rr[0]);
    rr[1] = fmaf(v.y, v.y, rr[1]);
    return v;
  }
};

// Gain policy of the ML solve's Wiener preconditioner (Sec. 4.2): the real gain
// G = 1 / (|W|^2 inv_s2 + lam_m[col]) / J, 0 where the denominator vanishes.
template <int NT, bool FUSED>
struct MlGain {
  // With the real gain g, z = M r has r.z = sum_k g(k) |R(k)|^2 (Parseval for the
  // unnormalised transform pair), accumulated here per column while the gains are applied
  float acc_a = 0.0f, acc_b = 0.0f;
  float rr[2] = {0.0f, 0.0f};  // FUSED: the CTA's r.r of the updated residual

  // 1 / (|W|^2 inv_s2 + lam_m) / J from |W|^2; a preconditioner only needs a fixed
  // positive gain, so the fast division serves (denominators below 1e-30 give 0)
  __device__ __forceinline__ static float from_w2(float a2, const MlGainParams& gp, int col) {
    const float P = fmaf(a2, gp.inv_s2, __ldg(gp.lam_m + col));
    return P > 1e-30f ? __fdividef(gp.invJ, P) : 0.0f;
  }
  // modes k and -k (w = 1), or one self-conjugate mode passed as both (w = 1/2)
  __device__ __forceinline__ void apply(float2& zk, float2& zm, const float* ta, const float* tb, float2 e1,
                                        const MlGainParams& gp, int p, float w) {
    float2 Wa, Wb;
    if constexpr (NT > 0) {
      // both columns share the powers of e1
      float2 ep[NT];
      ep[0] = make_float2(1.0f, 0.0f);
      if constexpr (NT > 1) ep[1] = e1;
#pragma unroll
      for (int q = 2; q < NT; ++q) ep[q] = cmul(ep[q / 2], ep[q - q / 2]);
      Wa = make_float2(ta[0], 0.0f);
      Wb = make_float2(tb[0], 0.0f);
#pragma unroll
      for (int q = 1; q < NT; ++q) {
        Wa.x = fmaf(ta[q], ep[q].x, Wa.x);
        Wa.y = fmaf(ta[q], ep[q].y, Wa.y);
        Wb.x = fmaf(tb[q], ep[q].x, Wb.x);
        Wb.y = fmaf(tb[q], ep[q].y, Wb.y);
      }
    } else {
      Wa = make_float2(0.0f, 0.0f);
      Wb = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int t = kMaxTaps - 1; t >= 0; --t) {
        if (t < gp.ntap) {
          Wa = cmul(Wa, e1);
          Wa.x += ta[t];
          Wb = cmul(Wb, e1);
          Wb.x += tb[t];
        }
      }
    }
    const float ga = from_w2(fmaf(Wa.x, Wa.x, Wa.y * Wa.y), gp, 2 * p);
    const float gb = from_w2(fmaf(Wb.x, Wb.x, Wb.y * Wb.y), gp, 2 * p + 1);
    // real gains: Z'_k = ga A + i gb B, Z'_-k = conj(ga A) + i conj(gb B) with
    // A = (Z_k + conj Z_-k)/2 = sv/2 and B = (Z_k - conj Z_-k)/(2i) = dv/(2i)
    const float2 sv = make_float2(zk.x + zm.x, zk.y - zm.y);
    const float2 dv = make_float2(zk.x - zm.x, zk.y + zm.y);
    const float2 P = cscale(sv, 0.5f * ga), Q = cscale(dv, 0.5f * gb);
    zk = cadd(P, Q);
    zm = make_float2(P.x - Q.x, Q.y - P.y);
    // modes k and -k add 2 g |A|^2 = g |sv|^2 / 2 (half that for a self-conjugate mode)
    acc_a = fmaf(0.5f * w * ga, fmaf(sv.x, sv.x, sv.y * sv.y), acc_a);
    acc_b = fmaf(0.5f * w * gb, fmaf(dv.x, dv.x, dv.y * dv.y), acc_b);
  }
  __device__ __forceinline__ void pair(float2& zk, float2& zm, const float* ta, const float* tb, int k, float2 e1,
                                       const MlGainParams& gp, int p) {
    (void)k;
    apply(zk, zm, ta, tb, e1, gp, p, 1.0f);
  }
  __device__ __forceinline__ void single(float2& a, float2& b, const float* ta, const float* tb, int k, float2 e1,
                                         const MlGainParams& gp, int p, bool self) {
    (void)k;
    apply(a, b, ta, tb, e1, gp, p, self ? 0.5f : 1.0f);
  }
  // step 1.  FUSED: alpha = r.z / p.q per active column (the pair's per-tile p.q
  // summed by one warp in a fixed order, FP64; the ratio in FP32), then the first pass
  // forms r - alpha q on the fly
  template <int S, int T>
  __device__ __forceinline__ void load(float2* sm, int tid, float2* base, const MlGainParams& gp, int p,
                                       size_t off) {
    if constexpr (!FUSED) {
      block_fft<S, T, false>(sm, tid, GMem{base}, SPad{sm});
    } else {
      __shared__ float al[2];
      if (tid < 32) {
        double a = 0.0, b = 0.0;
        if (tid < gp.nt) {
          const double* q = gp.pq_part + ((size_t)p * gp.nt + tid) * 8;
          a = __ldcg(q);
          b = __ldcg(q + 1);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (tid == 0) {
          const int act = __ldcg(&gp.ps[p].act);
          const double rz0 = __ldcg(&gp.ps[p].rz[0]), rz1 = __ldcg(&gp.ps[p].rz[1]);
          al[0] = ((act & 1) && a != 0.0) ? (float)rz0 / (float)a : 0.0f;
          al[1] = ((act & 2) && b != 0.0) ? (float)rz1 / (float)b : 0.0f;
        }
      }
      __syncthreads();
      block_fft<S, T, false>(sm, tid, MlResidLoad{gp.r_io + off, gp.q_in + off, al[0], al[1], rr}, SPad{sm});
    }
  }
  // the CTA's r.z (and, FUSED, r.r) of both columns to rz_out / rr_out[2 slot + c]
  // (FP32 within a warp, FP64 across)
  __device__ __forceinline__ void finish(const MlGainParams& gp, int slot) {
    if (!gp.rz_out) return;
    __shared__ float red[4][32];
    float v[4] = {acc_a, acc_b, rr[0], rr[1]};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) red[k][threadIdx.x >> 5] = v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum[4] = {0.0, 0.0, 0.0, 0.0};
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
#pragma unroll
        for (int k = 0; k < 4; ++k) sum[k] += (double)red[k][w];
      }
      gp.rz_out[2 * slot] = sum[0];
      gp.rz_out[2 * slot + 1] = sum[1];
      if constexpr (FUSED) {
        gp.rr_out[2 * slot] = sum[2];
        gp.rr_out[2 * slot + 1] = sum[3];
      }
    }
  }
};

// The ML solve's preconditioner (FUSED: with the residual update r -= alpha q in its
// load, so the transform's input is the new residual).  With a pair list (the solve's
// active pairs, ascending) cluster c transforms pair pair_list[c] if c < *pair_count
// and exits otherwise; every CTA of a cluster takes the same branch, before any cluster
// barrier.  (A persistent loop over the list keeps the transform's state live across
// trips and spills.)
template <int C, int S, int T, int NT, bool FUSED>
__global__ void __launch_bounds__(T, (S >= 4096 ? 2 : 1))
k3_column_ml(float2* __restrict__ d2, const float* __restrict__ window, int N, MlGainParams gp) {
  int p = blockIdx.x / C;
  if (gp.pair_list) {
    if (p >= __ldg(gp.pair_count)) return;
    p = __ldg(gp.pair_list + p);
  }
  k3_pair<C, S, T, NT, MlGain<NT, FUSED>, MlGainParams>(d2, window, N, gp, p);
}

template <int C, int S, int NT, bool FUSED>
cudaError_t k3_ml(float2* z2, const float* window, int N, const MlGainParams& gp, cudaStream_t st) {
  constexpr int T = t_for(S);
  const size_t smem = (size_t)padded_len(S) * sizeof(float2);
  auto kern = k3_column_ml<C, S, T, NT, FUSED>;
  cudaError_t e;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((N / 2) * C);
  cfg.blockDim = dim3(T);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, z2, window, N, gp);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int NT, bool FUSED>
cudaError_t k3_ml_cs(int C, int S, float2* z2, const float* window, int N, const MlGainParams& gp,
                     cudaStream_t st) {
  if (S == 8192) {
    switch (C) {
      case 2: return k3_ml<2, 8192, NT, FUSED>(z2, window, N, gp, st);
      case 4: return k3_ml<4, 8192, NT, FUSED>(z2, window, N, gp, st);
      case 8: return k3_ml<8, 8192, NT, FUSED>(z2, window, N, gp, st);
    }
  } else if (S == 512) {
    switch (C) {
      case 2: return k3_ml<2, 512, NT, FUSED>(z2, window, N, gp, st);
      case 4: return k3_ml<4, 512, NT, FUSED>(z2, window, N, gp, st);
      case 8: return k3_ml<8, 512, NT, FUSED>(z2, window, N, gp, st);
    }
  }
  return cudaErrorNotSupported;
}

cudaError_t k3_ml_fused(int C, int S, float2* z2, const float* window, int N, const MlGainParams& gp,
                        cudaStream_t st);
}  // namespace ipfb
