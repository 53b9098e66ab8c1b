// Learned conjugate-gradient preconditioner net (the workload's learned variant of
// the ML solve of Sec. 4.2; the paper itself has no learned component).
//
// Per column a 1-D convolutional net along the frame axis, circular padding:
//   z1 = conv(x0, w1) + b1   (2 -> 32 channels, 9 taps)    a1 = GELU(z1)
//   z2 = conv(a1, w2) + b2   (32 -> 32)                     a2 = GELU(z2)
//   y  = conv(a2, w3) + b3   (32 -> 1)
// conv(x, w)[co, j] = sum_{ci, t} w[co, ci, t] x[ci, (j + t - 4) mod J]  (cross-correlation),
// GELU(x) = x Phi(x) = 0.5 x (1 + erf(x / sqrt 2)), Phi the standard normal CDF.
// Parameters theta (FP32 master copy) are laid out w1[32][2][9], b1[32],
// w2[32][32][9], b2[32], w3[1][32][9], b3[1]: 10145 values.
//
// Precision: weights and activations x0, a1, a2 are rounded to BF16 (round to
// nearest even) and every convolution is a BF16 x BF16 -> FP32 tensor-core
// contraction (mma.sync m16n8k16); biases, pre-activations, GELU and the loss are
// FP32.  Each convolution is a GEMM over positions: row = position, K = (tap,
// input channel), so the tap shift is a row offset into a [position][channel]
// tile in shared memory.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"
#include "gelu_poly.cuh"
#include "tcgen05.cuh"

namespace ipfb {
namespace netk {

constexpr int KW = 9;
constexpr int HALF = 4;
constexpr int CH = 32;
constexpr int OW1 = 0, OB1 = 576, OW2 = 608, OB2 = 9824, OW3 = 9856, OB3 = 10144, NPARAM = 10145;

// Packed BF16 weights.  Row strides of 40 and 296 elements (80 B and 592 B) put
// the 8 rows that one ldmatrix phase reads into distinct 16-byte bank groups.
constexpr int S32 = 40;
constexpr int S288 = 296;
constexpr int PW1 = 0;                 // [32 co][S32]   k = 2t + ci   (k < 18, rest 0)
constexpr int PW2 = PW1 + 32 * S32;    // [32 co][S288]  k = 32t + ci
constexpr int PW3 = PW2 + 32 * S288;   // [8][S288]      row 0: k = 32t + ci; rows 1..7 zero
constexpr int PW2T = PW3 + 8 * S288;   // [32 ci][S288]  k = 32t' + co: w2[co][ci][8 - t']
constexpr int NPACK_BF = PW2T + 32 * S288;          // 22592 bf16
constexpr int NFWD_BF = PW2T;                       // forward needs W1, W2, W3
constexpr size_t PACK_BIAS_OFF = (size_t)NPACK_BF * 2;  // bytes; FP32 b1[32] b2[32] b3[1] pad[3]
constexpr size_t PACK_BYTES = PACK_BIAS_OFF + 68 * sizeof(float);

// ---- GELU, two values at a time on the paired FP32 pipe (fma.rn.f32x2 / mul.rn.f32x2).
// With a = |x| and Q(a) = 1 - Phi(a) the upper normal tail,
//   GELU(x) = max(x, 0) - a Q(a),   Q(a) = exp(-a^2 / 2) R(a),   R(a) = erfcx(a / sqrt 2) / 2,
// R a polynomial on [0, kGeluClamp] (gelu_poly.cuh; the FP32 result is within 3e-7
// absolute of x Phi(x)), the Gaussian factor one hardware exp2; and
//   GELU'(x) = Phi(x) + x phi(x) = (x >= 0 ? 1 - Q(a) : Q(a)) + x exp(-x^2 / 2) / sqrt(2 pi).
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_splat(float c) { return f2_pack(c, c); }
__device__ __forceinline__ float ex2_fast(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Q(|x0|), Q(|x1|) and the Gaussian factors exp(-x^2 / 2)
__device__ __forceinline__ void normal_tail2(float x0, float x1, float& q0, float& q1, float& e0, float& e1) {
  const float a0 = fabsf(x0), a1 = fabsf(x1);
  const uint64_t t = f2_pack(fminf(a0, kGeluClamp), fminf(a1, kGeluClamp));
  uint64_t r = f2_fma(f2_splat(gelu_r(kGeluDeg)), t, f2_splat(gelu_r(kGeluDeg - 1)));
#pragma unroll
  for (int k = kGeluDeg - 2; k >= 0; --k) r = f2_fma(r, t, f2_splat(gelu_r(k)));
  constexpr float kHalfLog2e = 0.72134752044448170f;  // exp(-a^2 / 2) = 2^(-a^2 log2(e) / 2)
  const uint64_t aa = f2_pack(a0, a1);
  float s0, s1;
  f2_unpack(f2_mul(f2_mul(aa, aa), f2_splat(-kHalfLog2e)), s0, s1);
  e0 = ex2_fast(s0);
  e1 = ex2_fast(s1);
  f2_unpack(f2_mul(f2_pack(e0, e1), r), q0, q1);
}

// x <- GELU(x) for two values
__device__ __forceinline__ void gelu2(float& x0, float& x1) {
  float q0, q1, e0, e1;
  normal_tail2(x0, x1, q0, q1, e0, e1);
  f2_unpack(f2_fma(f2_pack(-fabsf(x0), -fabsf(x1)), f2_pack(q0, q1), f2_pack(fmaxf(x0, 0.0f), fmaxf(x1, 0.0f))),
            x0, x1);
}

// GELU (g) and GELU' (d) of two values
__device__ __forceinline__ void gelu2_grad(float x0, float x1, float& g0, float& g1, float& d0, float& d1) {
  float q0, q1, e0, e1;
  normal_tail2(x0, x1, q0, q1, e0, e1);
  g0 = fmaf(-fabsf(x0), q0, fmaxf(x0, 0.0f));
  g1 = fmaf(-fabsf(x1), q1, fmaxf(x1, 0.0f));
  constexpr float kInvSqrt2Pi = 0.39894228040143268f;
  d0 = fmaf(x0 * kInvSqrt2Pi, e0, x0 >= 0.0f ? 1.0f - q0 : q0);
  d1 = fmaf(x1 * kInvSqrt2Pi, e1, x1 >= 0.0f ? 1.0f - q1 : q1);
}

__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo (low 16 bits), .y = hi
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ float bf_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf_hi(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }
__device__ __forceinline__ float bf_at(const __nv_bfloat16* p) { return __bfloat162float(*p); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2(uint32_t& r0, uint32_t& r1, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(smem_u32(p)));
}
// D += A B, A 16x16 (row-major fragments), B 16x8 (column-major fragments), FP32 accumulators
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Lane address of an ldmatrix.x4 A tile (16 rows x 16 k) of a row-major [row][k] array:
// matrices (rows 0-7, k 0-7), (rows 8-15, k 0-7), (rows 0-7, k 8-15), (rows 8-15, k 8-15).
__device__ __forceinline__ const __nv_bfloat16* a_tile_addr(const __nv_bfloat16* base, int stride, int row0, int k0,
                                                          int lane) {
  const int mi = lane >> 3, ri = lane & 7;
  return base + (row0 + ri + (mi & 1) * 8) * stride + k0 + (mi >> 1) * 8;
}
// Lane address of an ldmatrix.x4 B pair (two n-tiles of 8 x 16 k) of an [n][k] array:
// registers 0,1 = (b0, b1) of n-tile n0, registers 2,3 = (b0, b1) of n-tile n0 + 8.
__device__ __forceinline__ const __nv_bfloat16* b_pair_addr(const __nv_bfloat16* base, int stride, int n0, int k0,
                                                          int lane) {
  const int mi = lane >> 3, ri = lane & 7;
  return base + (n0 + ri + (mi >> 1) * 8) * stride + k0 + (mi & 1) * 8;
}

// theta (FP32) -> packed BF16 weights + FP32 biases
__global__ void k6_net_pack(const float* __restrict__ theta, uint8_t* __restrict__ packed) {
  __nv_bfloat16* pw = reinterpret_cast<__nv_bfloat16*>(packed);
  float* pb = reinterpret_cast<float*>(packed + PACK_BIAS_OFF);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPACK_BF + 68; i += gridDim.x * blockDim.x) {
    if (i >= NPACK_BF) {
      const int b = i - NPACK_BF;
      float v = 0.0f;
      if (b < 32) v = theta[OB1 + b];
      else if (b < 64) v = theta[OB2 + b - 32];
      else if (b == 64) v = theta[OB3];
      pb[b] = v;
      continue;
    }
    float v = 0.0f;
    if (i < PW2) {
      const int co = i / S32, k = i % S32;
      if (k < 18) v = theta[OW1 + (co * 2 + (k & 1)) * KW + (k >> 1)];
    } else if (i < PW3) {
      const int co = (i - PW2) / S288, k = (i - PW2) % S288;
      if (k < 288) v = theta[OW2 + (co * CH + (k & 31)) * KW + (k >> 5)];
    } else if (i < PW2T) {
      const int row = (i - PW3) / S288, k = (i - PW3) % S288;
      if (row == 0 && k < 288) v = theta[OW3 + (k & 31) * KW + (k >> 5)];
    } else {
      const int ci = (i - PW2T) / S288, k = (i - PW2T) % S288;
      if (k < 288) v = theta[OW2 + ((k & 31) * CH + ci) * KW + (8 - (k >> 5))];
    }
    pw[i] = __float2bfloat16_rn(v);
  }
}

// ---------------------------------------------------------------------------
// Shared pieces of the forward and backward kernels
// ---------------------------------------------------------------------------
// Copy packed BF16 rows [0, nbf) and the biases into shared memory (16-byte copies).
__device__ __forceinline__ void load_pack(const uint8_t* __restrict__ packed, __nv_bfloat16* wsm, float* bsm, int nbf,
                                          int nbf_off = 0) {
  const uint4* src = reinterpret_cast<const uint4*>(packed + (size_t)nbf_off * 2);
  uint4* dst = reinterpret_cast<uint4*>(wsm);
  for (int i = threadIdx.x; i < nbf / 8; i += blockDim.x) dst[i] = src[i];
  const float* pb = reinterpret_cast<const float*>(packed + PACK_BIAS_OFF);
  for (int i = threadIdx.x; i < 68; i += blockDim.x) bsm[i] = pb[i];
}

// x0 rows: x0s[i] = (bf16 ch0, bf16 ch1) at position (q0 + i) mod J, i < nrows
__device__ __forceinline__ void load_x0(const float* __restrict__ in, int J, int q0, int nrows, uint32_t* x0s) {
  // positions q0 .. q0 + nrows - 1 lie in [-J, 2J) when -J <= q0 and q0 + nrows <= 2J
  // (every tile of a column with J >= nrows): one conditional wrap, no division
  const bool one_wrap = q0 >= -J && q0 + nrows <= 2 * J;
  for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
    int q = q0 + i;
    if (one_wrap) {
      q = q < 0 ? q + J : (q >= J ? q - J : q);
    } else {
      q %= J;
      if (q < 0) q += J;
    }
    x0s[i] = pack_bf2(__ldg(in + q), __ldg(in + J + q));
  }
}

// im2col of layer 1: A1[i][2t + ci] = x0[i + t][ci] (t < 9), zero for k in [18, 32)
__device__ __forceinline__ void build_a1col(const uint32_t* x0s, int nrows, __nv_bfloat16* A1s) {
  for (int idx = threadIdx.x; idx < nrows * 16; idx += blockDim.x) {
    const int i = idx >> 4, t = idx & 15;
    reinterpret_cast<uint32_t*>(A1s + i * S32)[t] = t < KW ? x0s[i + t] : 0u;
  }
}

// One conv layer as MT m-tiles (16 output rows each) x 4 n-tiles (32 output channels)
// for this warp: rows [m0, m0 + 16) of the output use A rows m0 + t + [0, 16) (tap t)
// when TAPS, else rows m0 + [0, 16) with K contiguous.  KSTEPS = K / 16.
// The epilogue receives (row, col, v0, v1) for columns col, col + 1.
template <int KSTEPS, bool TAPS, class EPI>
__device__ __forceinline__ void conv_layer_warp(const __nv_bfloat16* A, int astride, const __nv_bfloat16* B,
                                                int bstride, int m0, int lane, EPI epi) {
  float acc[4][4];
#pragma unroll
  for (int n = 0; n < 4; ++n)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[n][q] = 0.0f;
#pragma unroll 2
  for (int ks = 0; ks < KSTEPS; ++ks) {
    // with taps: k-step ks covers tap ks / 2, input channels 16 (ks % 2) .. + 15
    const int arow = TAPS ? m0 + (ks >> 1) : m0;
    const int acol = TAPS ? (ks & 1) * 16 : ks * 16;
    uint32_t a[4], b01[4], b23[4];
    ldsm_x4(a, a_tile_addr(A, astride, arow, acol, lane));
    ldsm_x4(b01, b_pair_addr(B, bstride, 0, ks * 16, lane));
    ldsm_x4(b23, b_pair_addr(B, bstride, 16, ks * 16, lane));
    mma_bf16(acc[0], a, b01[0], b01[1]);
    mma_bf16(acc[1], a, b01[2], b01[3]);
    mma_bf16(acc[2], a, b23[0], b23[1]);
    mma_bf16(acc[3], a, b23[2], b23[3]);
  }
  const int g = lane >> 2, c = lane & 3;
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    epi(m0 + g, n * 8 + 2 * c, acc[n][0], acc[n][1]);
    epi(m0 + g + 8, n * 8 + 2 * c, acc[n][2], acc[n][3]);
  }
}

// Layer 1 (2 -> 32 channels, 9 taps, K = 2t + ci padded to 32) for one m-tile, its A
// fragments read straight from the packed input rows: in the m16n8k16 layout lane
// (g = lane / 4, c = lane % 4) holds rows g and g + 8 at k = 2c, 2c + 1 (tap c, both
// channels: one packed row x0s[row + c]) and at k = 2c + 8, 2c + 9 (tap c + 4); the
// second k-step holds tap 8 (lanes with c = 0) and zeros.  bw holds the B fragments
// of W1 (two k-steps x four n-tiles), loaded once per warp.
template <class EPI>
__device__ __forceinline__ void conv1_warp(const uint32_t* x0s, const uint32_t (&bw)[16], int m0, int lane,
                                           EPI epi) {
  float acc[4][4];
#pragma unroll
  for (int n = 0; n < 4; ++n)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[n][q] = 0.0f;
  const int g = lane >> 2, c = lane & 3;
  const uint32_t* x = x0s + m0 + g;
  const uint32_t a0[4] = {x[c], x[8 + c], x[4 + c], x[12 + c]};
  const uint32_t t8a = x[8], t8b = x[16];
  const uint32_t a1[4] = {c == 0 ? t8a : 0u, c == 0 ? t8b : 0u, 0u, 0u};
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    mma_bf16(acc[n], a0, bw[2 * n], bw[2 * n + 1]);
    mma_bf16(acc[n], a1, bw[8 + 2 * n], bw[8 + 2 * n + 1]);
  }
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    epi(m0 + g, n * 8 + 2 * c, acc[n][0], acc[n][1]);
    epi(m0 + g + 8, n * 8 + 2 * c, acc[n][2], acc[n][3]);
  }
}

// B fragments of W1 for conv1_warp: bw[2n], bw[2n + 1] the n-tile n of k-step 0,
// bw[8 + 2n], bw[8 + 2n + 1] those of k-step 1
__device__ __forceinline__ void load_w1_frags(const __nv_bfloat16* W1, int lane, uint32_t (&bw)[16]) {
#pragma unroll
  for (int ks = 0; ks < 2; ++ks) {
    uint32_t b01[4], b23[4];
    ldsm_x4(b01, b_pair_addr(W1, S32, 0, ks * 16, lane));
    ldsm_x4(b23, b_pair_addr(W1, S32, 16, ks * 16, lane));
    bw[8 * ks + 0] = b01[0];
    bw[8 * ks + 1] = b01[1];
    bw[8 * ks + 2] = b01[2];
    bw[8 * ks + 3] = b01[3];
    bw[8 * ks + 4] = b23[0];
    bw[8 * ks + 5] = b23[1];
    bw[8 * ks + 6] = b23[2];
    bw[8 * ks + 7] = b23[3];
  }
}

// Layer 3 (one output channel, padded to an 8-wide n-tile) for one m-tile:
// returns through epi(row, value) for the rows this lane holds (lanes with c == 0).
template <class EPI>
__device__ __forceinline__ void conv_out_warp(const __nv_bfloat16* A, const __nv_bfloat16* W3, int m0, int lane,
                                              EPI epi) {
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  const int l16 = lane & 15;
#pragma unroll 2
  for (int ks = 0; ks < 18; ++ks) {
    uint32_t a[4], b0, b1;
    ldsm_x4(a, a_tile_addr(A, S32, m0 + (ks >> 1), (ks & 1) * 16, lane));
    // x2: lanes 0-7 address rows 0-7 at k0, lanes 8-15 rows 0-7 at k0 + 8
    ldsm_x2(b0, b1, W3 + (l16 & 7) * S288 + ks * 16 + (l16 >> 3) * 8);
    mma_bf16(acc, a, b0, b1);
  }
  const int g = lane >> 2, c = lane & 3;
  if (c == 0) {
    epi(m0 + g, acc[0]);
    epi(m0 + g + 8, acc[2]);
  }
}

// ---------------------------------------------------------------------------
// Forward: y[slot][j] for slots [0, nslots) (nslots from *count if count != null).
// Work item = (slot, tile of FT outputs); persistent CTAs of 256 threads.
// Rows: x0 i <-> p0 - 12 + i (264), a1 i <-> p0 - 8 + i (256, +8 zero rows),
//       a2 i <-> p0 - 4 + i (256, first 248 used), y i <-> p0 + i (240).
// Layers 1 and 3 run on mma.sync; layer 2 (90 % of the flops) on the fifth-generation
// tensor cores: two M = 128 row blocks x N = 32 channels x K = 288 (9 taps x 32 input
// channels) in 2 x 18 tcgen05.mma of K = 16, issued by one thread, accumulators in
// 64 TMEM columns, read back by all eight warps (warp w: lane quarter w % 4, block
// w / 4) for the bias + GELU epilogue.  Operands in shared memory as no-swizzle
// K-major core matrices: a1 as [4 channel chunks][264 rows][8] (a tap is a 16-byte
// row offset of the descriptor's start address), W2 as [36 k-chunks][32 co][8].
// ---------------------------------------------------------------------------
constexpr int FT = 240;
constexpr int F_X0 = FT + 24;   // 264
constexpr int F_A1 = FT + 16;   // 256 computed rows of a1
constexpr int F_A2 = FT + 16;   // 256 computed rows of a2 (248 valid)
constexpr int A1R = F_A1 + 8;   // a1 rows held (8 zero rows past the computed ones)
// shared-memory map of the forward (bytes)
constexpr size_t FO_W2C = 0;                                    // [36][32][8] bf16
constexpr size_t FO_A1C = FO_W2C + 36 * 32 * 16;                // [4][A1R][8] bf16
constexpr size_t FO_A2 = FO_A1C + 4 * (size_t)A1R * 16;         // [256][S32] bf16 (also layer-1 im2col)
constexpr size_t FO_W1 = FO_A2 + (size_t)F_A2 * S32 * 2;        // [32][S32] bf16
constexpr size_t FO_W3 = FO_W1 + 32 * S32 * 2;                  // [8][S288] bf16
constexpr size_t FO_B = FO_W3 + 8 * S288 * 2;                   // 68 floats
constexpr size_t FO_X0 = FO_B + 68 * 4;                         // F_X0 packed bf16 pairs
constexpr size_t fwd_smem_bytes() { return FO_X0 + (size_t)F_X0 * 4; }
static_assert(FO_A1C % 1024 == 0 && FO_A2 % 16 == 0 && FO_W1 % 16 == 0 && FO_W3 % 16 == 0, "alignment");
constexpr uint32_t kNetTmemCols = 64;
constexpr long long kNetMmaWait = 2000000000LL;  // SM clocks (~1 s)

// wait_limit: SM clocks the accumulator wait may take before the CTA gives up (the
// library passes kNetMmaWait unless a test lowers it).  A CTA that gives up marks the
// first output of its tile with NaN, sets *status (when not null), waits up to
// kNetMmaWait more for its MMAs in flight so that nothing still writes its tensor
// memory or reads its shared memory, frees its tensor memory and stops.
__global__ void __launch_bounds__(256)
k6_net_forward(const uint8_t* __restrict__ packed, const float* __restrict__ in, float* __restrict__ y, int J,
               int nslots_host, const int* __restrict__ count, int* __restrict__ zero_other, long long wait_limit,
               int* __restrict__ status) {
  extern __shared__ __align__(1024) uint8_t smfwd[];
  __shared__ __align__(8) uint64_t mma_bar;
  __shared__ uint32_t tmem_slot;
  __nv_bfloat16* w2c = reinterpret_cast<__nv_bfloat16*>(smfwd + FO_W2C);
  __nv_bfloat16* a1c = reinterpret_cast<__nv_bfloat16*>(smfwd + FO_A1C);
  __nv_bfloat16* a2s = reinterpret_cast<__nv_bfloat16*>(smfwd + FO_A2);
  __nv_bfloat16* W1 = reinterpret_cast<__nv_bfloat16*>(smfwd + FO_W1);
  __nv_bfloat16* W3 = reinterpret_cast<__nv_bfloat16*>(smfwd + FO_W3);
  float* bsm = reinterpret_cast<float*>(smfwd + FO_B);
  uint32_t* x0s = reinterpret_cast<uint32_t*>(smfwd + FO_X0);

  if (zero_other && blockIdx.x == 0 && threadIdx.x == 0) *zero_other = 0;
  const int nslots = count ? *count : nslots_host;
  const int ntile = (J + FT - 1) / FT;
  const long long nitems = (long long)nslots * ntile;
  if ((long long)blockIdx.x >= nitems) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // weights: W1, W3 and the biases as packed; W2 regrouped into k-chunk core matrices
  {
    const uint4* src = reinterpret_cast<const uint4*>(packed);
    for (int i = threadIdx.x; i < 32 * S32 / 8; i += blockDim.x)
      reinterpret_cast<uint4*>(W1)[i] = src[PW1 / 8 + i];
    for (int i = threadIdx.x; i < 8 * S288 / 8; i += blockDim.x)
      reinterpret_cast<uint4*>(W3)[i] = src[PW3 / 8 + i];
    for (int i = threadIdx.x; i < 36 * 32; i += blockDim.x) {
      const int kc = i >> 5, co = i & 31;
      reinterpret_cast<uint4*>(w2c)[i] = src[(PW2 + co * S288) / 8 + kc];
    }
    const float* pb = reinterpret_cast<const float*>(packed + PACK_BIAS_OFF);
    for (int i = threadIdx.x; i < 68; i += blockDim.x) bsm[i] = pb[i];
    // the 8 rows past a1 in every channel chunk (read by the unused a2 rows) stay zero
    for (int i = threadIdx.x; i < 4 * 8; i += blockDim.x)
      reinterpret_cast<uint4*>(a1c)[(i >> 3) * A1R + F_A1 + (i & 7)] = make_uint4(0u, 0u, 0u, 0u);
  }
  if (warp == 0) tc::alloc(smem_u32(&tmem_slot), kNetTmemCols);
  if (threadIdx.x == 0) tc::mbar_init(smem_u32(&mma_bar));
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = tmem_slot;
  uint32_t phase = 0;
  uint32_t bw1[16];
  load_w1_frags(W1, lane, bw1);
  // layer-2 operand descriptors: the start address sits in the low 14 bits (16-byte
  // units, shared memory < 256 KB), so each MMA's descriptor is a base plus a constant
  const uint64_t adesc0 = tc::desc(smem_u32(a1c), A1R * 16, 128);
  const uint64_t bdesc0 = tc::desc(smem_u32(w2c), 32 * 16, 128);

  // Tile loop, software-pipelined: while the tensor cores run layer 2 of tile i, the
  // warps run layer 3 of tile i - 1 (from a2s) and load the input rows of tile i + 1
  // (into x0s, free once layer 1 of tile i is done).
  const float b3 = bsm[64];
  auto layer3 = [&](int s3, int q3) {
    float* yo = y + (size_t)s3 * J;
#pragma unroll 1
    for (int mt = warp; mt < FT / 16; mt += 8)
      conv_out_warp(a2s, W3, mt * 16, lane, [&](int r, float v) {
        if (q3 + r < J) yo[q3 + r] = v + b3;
      });
  };
  long long item = blockIdx.x;
  int slot = (int)(item / ntile), p0 = (int)(item % ntile) * FT;
  int prev_slot = -1, prev_p0 = 0;
  bool stopped = false;
  load_x0(in + (size_t)slot * 2 * J, J, p0 - 12, F_X0, x0s);
  for (; item < nitems; item += gridDim.x) {
    __syncthreads();  // x0s holds this tile's rows; a2s, a1c and TMEM are free
    // layer 1 (mma.sync, A fragments from the packed input rows): m-tiles warp,
    // warp + 8, into the chunked a1
#pragma unroll 1
    for (int mt = warp; mt < F_A1 / 16; mt += 8)
      conv1_warp(x0s, bw1, mt * 16, lane, [&](int r, int cc, float v0, float v1) {
        v0 += bsm[cc];
        v1 += bsm[cc + 1];
        gelu2(v0, v1);
        *reinterpret_cast<uint32_t*>(a1c + ((cc >> 3) * A1R + r) * 8 + (cc & 7)) = pack_bf2(v0, v1);
      });
    tc::fence_smem_operands();
    tc::fence_before();
    __syncthreads();
    // layer 2 (tcgen05): one thread issues the 36 MMAs and commits them to mma_bar
    if (threadIdx.x == 0) {
      tc::fence_after();
      constexpr uint32_t idesc = tc::idesc_bf16(128, 32);
#pragma unroll
      for (int mb = 0; mb < 2; ++mb)
#pragma unroll
        for (int ks = 0; ks < 2 * KW; ++ks) {
          const int t = ks >> 1, h = ks & 1;
          const uint64_t ad = adesc0 + (uint64_t)((2 * h) * A1R + 128 * mb + t);
          const uint64_t bd = bdesc0 + (uint64_t)(2 * ks * 32);
          tc::mma(tbase + 32 * mb, ad, bd, idesc, ks > 0 ? 1u : 0u);
        }
      tc::commit(smem_u32(&mma_bar));
    }
    if (prev_slot >= 0) layer3(prev_slot, prev_p0);
    const long long next = item + gridDim.x;
    const int nslot = (int)(next / ntile), np0 = (int)(next % ntile) * FT;
    if (next < nitems) load_x0(in + (size_t)nslot * 2 * J, J, np0 - 12, F_X0, x0s);
    // one thread waits on the barrier; the others sleep in the block barrier below
    bool late = false;
    if (threadIdx.x == 0) late = !tc::mbar_wait(smem_u32(&mma_bar), phase, wait_limit);
    if (__syncthreads_or(late)) {  // the accumulators did not arrive in time: mark, drain, stop
      if (threadIdx.x == 0) {
        y[(size_t)slot * J + p0] = __int_as_float(0x7fc00000);
        if (status) atomicOr(status, 1);
        (void)tc::mbar_wait(smem_u32(&mma_bar), phase, kNetMmaWait);
      }
      __syncthreads();
      stopped = true;
      break;
    }
    phase ^= 1;
    tc::fence_after();
    {
      const int qd = warp & 3, mb = warp >> 2;
      const int r = 128 * mb + 32 * qd + lane;
      float v[32];
      tc::ld32(tbase + ((uint32_t)(32 * qd) << 16) + 32 * mb, v);
      uint32_t pk[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        float g0 = v[2 * c] + bsm[32 + 2 * c], g1 = v[2 * c + 1] + bsm[33 + 2 * c];
        gelu2(g0, g1);
        pk[c] = pack_bf2(g0, g1);
      }
      uint4* dst = reinterpret_cast<uint4*>(a2s + r * S32);
#pragma unroll
      for (int c = 0; c < 4; ++c) dst[c] = make_uint4(pk[4 * c], pk[4 * c + 1], pk[4 * c + 2], pk[4 * c + 3]);
    }
    tc::fence_before();
    prev_slot = slot;
    prev_p0 = p0;
    slot = nslot;
    p0 = np0;
  }
  if (!stopped && prev_slot >= 0) {
    __syncthreads();
    layer3(prev_slot, prev_p0);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::dealloc(tbase, kNetTmemCols);
}

// ---------------------------------------------------------------------------
// Backward (loss = sum over all positions of (y - target)^2 * inv_n): per work item
// the tile's forward is recomputed with the halo the gradients need, then
//   dy -> dW3, db3;  da2 = conv^T(dy, w3), dz2 = da2 GELU'(z2) -> dW2, db2;
//   da1 = conv^T(dz2, w2) (tensor cores), dz1 = da1 GELU'(z1) -> dW1, db1.
// Each item writes its partial gradient (NPARAM values) and loss to part[item].
// Rows (tile positions [p0, p0 + BT)):
//   x0  i <-> p0 - 20 + i  (264)      a1  i <-> p0 - 16 + i  (256 + 8 zero)
//   a2  i <-> p0 - 12 + i  (256, 248 valid)   y/dy i <-> p0 - 8 + i (240)
//   dz2 i <-> p0 - 4 + i   (232)      dz1 i <-> p0 + i (224)
// ---------------------------------------------------------------------------
constexpr int BT = 224;
constexpr int B_X0 = BT + 40;   // 264
constexpr int B_A1 = BT + 32;   // 256
constexpr int B_A2 = BT + 32;   // 256 computed, 248 valid
constexpr int B_Y = BT + 16;    // 240
constexpr int B_DZ2 = BT + 8;   // 232
constexpr int GP_STRIDE = 33;   // FP32 rows of 32 channels, padded

struct BwdSmem {
  static constexpr size_t w = 0;                                        // packed bf16 (all, incl. W2T)
  static constexpr size_t b = w + (size_t)NPACK_BF * 2;                 // 68 floats
  static constexpr size_t x0 = b + 68 * 4;                              // [264] u32
  static constexpr size_t a1 = x0 + (size_t)B_X0 * 4;                   // [264][S32] bf16
  static constexpr size_t a2 = a1 + (size_t)(B_A1 + 8) * S32 * 2;       // [256][S32] bf16
  static constexpr size_t dz2 = a2 + (size_t)B_A2 * S32 * 2;            // [256][S32] bf16 (also im2col)
  static constexpr size_t gp2 = dz2 + (size_t)B_A1 * S32 * 2;           // [232][33] f32 GELU'(z2)
  static constexpr size_t gp1 = gp2 + (size_t)B_DZ2 * GP_STRIDE * 4;    // [224][33] f32 GELU'(z1), then dz1
  static constexpr size_t dy = gp1 + (size_t)BT * GP_STRIDE * 4;        // [240] f32
  static constexpr size_t red = dy + (size_t)B_Y * 4;                   // [8 warps][8] f32
  static constexpr size_t total = red + 64 * 4;
};

__global__ void __launch_bounds__(256, 1)
k6_net_backward(const uint8_t* __restrict__ packed, const float* __restrict__ in, const float* __restrict__ target,
                int J, int nslots, float inv_n, float* __restrict__ part) {
  extern __shared__ __align__(16) uint8_t smraw[];
  __nv_bfloat16* wsm = reinterpret_cast<__nv_bfloat16*>(smraw + BwdSmem::w);
  float* bsm = reinterpret_cast<float*>(smraw + BwdSmem::b);
  uint32_t* x0s = reinterpret_cast<uint32_t*>(smraw + BwdSmem::x0);
  __nv_bfloat16* a1s = reinterpret_cast<__nv_bfloat16*>(smraw + BwdSmem::a1);
  __nv_bfloat16* a2s = reinterpret_cast<__nv_bfloat16*>(smraw + BwdSmem::a2);
  __nv_bfloat16* dz2s = reinterpret_cast<__nv_bfloat16*>(smraw + BwdSmem::dz2);
  float* gp2 = reinterpret_cast<float*>(smraw + BwdSmem::gp2);
  float* gp1 = reinterpret_cast<float*>(smraw + BwdSmem::gp1);
  float* dys = reinterpret_cast<float*>(smraw + BwdSmem::dy);
  float* red = reinterpret_cast<float*>(smraw + BwdSmem::red);
  const __nv_bfloat16* W1 = wsm + PW1;
  const __nv_bfloat16* W2 = wsm + PW2;
  const __nv_bfloat16* W3 = wsm + PW3;
  const __nv_bfloat16* W2T = wsm + PW2T;

  const int ntile = (J + BT - 1) / BT;
  const long long nitems = (long long)nslots * ntile;
  if ((long long)blockIdx.x >= nitems) return;
  load_pack(packed, wsm, bsm, NPACK_BF);
  for (int i = threadIdx.x; i < 8 * S32 / 2; i += blockDim.x) reinterpret_cast<uint32_t*>(a1s + B_A1 * S32)[i] = 0u;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (long long item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int slot = (int)(item / ntile), tile = (int)(item % ntile);
    const int p0 = tile * BT;
    const float* tg = target + (size_t)slot * J;
    float* pg = part + (size_t)item * (NPARAM + 1);
    __syncthreads();
    load_x0(in + (size_t)slot * 2 * J, J, p0 - 20, B_X0, x0s);
    __syncthreads();
    build_a1col(x0s, B_A1, dz2s);
    __syncthreads();
    // ---- forward recompute; keep GELU'(z) on the rows the backward uses
#pragma unroll 1
    for (int mt = warp; mt < B_A1 / 16; mt += 8)
      conv_layer_warp<2, false>(dz2s, S32, W1, S32, mt * 16, lane, [&](int r, int cc, float v0, float v1) {
        v0 += bsm[cc];
        v1 += bsm[cc + 1];
        // a1 row r <-> dz1 row r - 16
        float g0, g1, d0, d1;
        gelu2_grad(v0, v1, g0, g1, d0, d1);
        if (r >= 16 && r < 16 + BT) {
          gp1[(r - 16) * GP_STRIDE + cc] = d0;
          gp1[(r - 16) * GP_STRIDE + cc + 1] = d1;
        }
        *reinterpret_cast<uint32_t*>(a1s + r * S32 + cc) = pack_bf2(g0, g1);
      });
    __syncthreads();
#pragma unroll 1
    for (int mt = warp; mt < B_A2 / 16; mt += 8)
      conv_layer_warp<18, true>(a1s, S32, W2, S288, mt * 16, lane, [&](int r, int cc, float v0, float v1) {
        v0 += bsm[32 + cc];
        v1 += bsm[32 + cc + 1];
        // a2 row r <-> dz2 row r - 8
        float g0, g1, d0, d1;
        gelu2_grad(v0, v1, g0, g1, d0, d1);
        if (r >= 8 && r < 8 + B_DZ2) {
          gp2[(r - 8) * GP_STRIDE + cc] = d0;
          gp2[(r - 8) * GP_STRIDE + cc + 1] = d1;
        }
        *reinterpret_cast<uint32_t*>(a2s + r * S32 + cc) = pack_bf2(g0, g1);
      });
    __syncthreads();
    float loss_part = 0.0f;
    {
      const float b3 = bsm[64];
#pragma unroll 1
      for (int mt = warp; mt < B_Y / 16; mt += 8)
        conv_out_warp(a2s, W3, mt * 16, lane, [&](int r, float v) {
          // y row r <-> position p0 - 8 + r
          int q = (p0 - 8 + r) % J;
          if (q < 0) q += J;
          const float diff = v + b3 - __ldg(tg + q);
          dys[r] = 2.0f * inv_n * diff;
          if (r >= 8 && r < 8 + BT && p0 + r - 8 < J) loss_part = fmaf(diff * inv_n, diff, loss_part);
        });
    }
    __syncthreads();
    // positions past J in the last tile contribute no gradient
    const int nvalid = min(BT, J - p0);
    // ---- dW3[ci][t] = sum_pos dy[pos] a2[pos + t - 4][ci]: dy row i + 8, a2 row i + 8 + t
    for (int o = tid; o < 288 + 1; o += blockDim.x) {
      float s = 0.0f;
      if (o < 288) {
        const int ci = o / KW, t = o % KW;
        for (int i = 0; i < nvalid; ++i) s = fmaf(dys[i + 8], bf_at(a2s + (i + 8 + t) * S32 + ci), s);
        pg[OW3 + o] = s;
      } else {
        for (int i = 0; i < nvalid; ++i) s += dys[i + 8];
        pg[OB3] = s;
      }
    }
    // ---- dz2[i][ci] = GELU'(z2) * sum_t w3[ci][t] dy[i + 8 - t]  (i < 232)
    for (int idx = tid; idx < B_DZ2 * 16; idx += blockDim.x) {
      const int i = idx >> 4, c2 = (idx & 15) * 2;
      float d0 = 0.0f, d1 = 0.0f;
#pragma unroll
      for (int t = 0; t < KW; ++t) {
        const float dyv = dys[i + 8 - t];
        d0 = fmaf(bf_at(W3 + t * 32 + c2), dyv, d0);
        d1 = fmaf(bf_at(W3 + t * 32 + c2 + 1), dyv, d1);
      }
      d0 *= gp2[i * GP_STRIDE + c2];
      d1 *= gp2[i * GP_STRIDE + c2 + 1];
      // dz2 rows outside the valid positions (beyond J in the last tile) are real
      // gradients of neighbouring positions only through the circular wrap; keep them
      // (they feed da1 of valid rows) but exclude them from the weight sums below.
      gp2[i * GP_STRIDE + c2] = d0;
      gp2[i * GP_STRIDE + c2 + 1] = d1;
      *reinterpret_cast<uint32_t*>(dz2s + i * S32 + c2) = pack_bf2(d0, d1);
    }
    __syncthreads();
    // ---- da1 = conv^T(dz2, w2) on the tile rows (tensor cores), dz1 = da1 GELU'(z1)
#pragma unroll 1
    for (int mt = warp; mt < BT / 16; mt += 8)
      conv_layer_warp<18, true>(dz2s, S32, W2T, S288, mt * 16, lane, [&](int r, int cc, float v0, float v1) {
        gp1[r * GP_STRIDE + cc] *= v0;
        gp1[r * GP_STRIDE + cc + 1] *= v1;
      });
    // ---- db2, dW2[co][ci][t] = sum_pos dz2[pos][co] a1[pos + t - 4][ci]
    //   dz2 row i + 4 (FP32 in gp2), a1 row i + 12 + t, i < nvalid
    for (int o = tid; o < CH * CH * KW + CH; o += blockDim.x) {
      float s = 0.0f;
      if (o < CH * CH * KW) {
        const int co = o / (CH * KW), rem = o % (CH * KW), ci = rem / KW, t = rem % KW;
        for (int i = 0; i < nvalid; ++i)
          s = fmaf(gp2[(i + 4) * GP_STRIDE + co], bf_at(a1s + (i + 12 + t) * S32 + ci), s);
        pg[OW2 + o] = s;
      } else {
        const int co = o - CH * CH * KW;
        for (int i = 0; i < nvalid; ++i) s += gp2[(i + 4) * GP_STRIDE + co];
        pg[OB2 + co] = s;
      }
    }
    __syncthreads();
    // ---- db1, dW1[co][ci][t] = sum_pos dz1[pos][co] x0[pos + t - 4][ci]: dz1 row i, x0 row i + 16 + t
    for (int o = tid; o < CH * 2 * KW + CH; o += blockDim.x) {
      float s = 0.0f;
      if (o < CH * 2 * KW) {
        const int co = o / (2 * KW), ci = (o / KW) & 1, t = o % KW;
        for (int i = 0; i < nvalid; ++i) {
          const uint32_t xv = x0s[i + 16 + t];
          s = fmaf(gp1[i * GP_STRIDE + co], ci ? bf_hi(xv) : bf_lo(xv), s);
        }
        pg[OW1 + o] = s;
      } else {
        const int co = o - CH * 2 * KW;
        for (int i = 0; i < nvalid; ++i) s += gp1[i * GP_STRIDE + co];
        pg[OB1 + co] = s;
      }
    }
    // ---- loss of the tile
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss_part += __shfl_xor_sync(0xffffffffu, loss_part, o);
    if (lane == 0) red[warp] = loss_part;
    __syncthreads();
    if (tid == 0) {
      float s = 0.0f;
      for (int w = 0; w < 8; ++w) s += red[w];
      pg[NPARAM] = s;
    }
  }
}

// grad[k] = sum over items of part[item][k] (k <= NPARAM: the last entry is the loss),
// FP64 accumulation in item order (deterministic)
__global__ void k6_net_reduce(const float* __restrict__ part, long long nitems, float* __restrict__ grad,
                              float* __restrict__ loss) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > NPARAM) return;
  double s = 0.0;
  for (long long i = 0; i < nitems; ++i) s += (double)part[(size_t)i * (NPARAM + 1) + k];
  if (k < NPARAM) {
    if (grad) grad[k] = (float)s;
  } else if (loss) {
    *loss = (float)s;
  }
}

// Adam (Kingma and Ba 2015) with bias corrections c1 = 1 - beta1^t, c2 = 1 - beta2^t
__global__ void k6_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                        const float* __restrict__ g, int n, float lr, float beta1, float beta2, float eps, float c1,
                        float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = fmaf(beta1, m[i], (1.0f - beta1) * gi);
  const float vi = fmaf(beta2, v[i], (1.0f - beta2) * gi * gi);
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace netk
}  // namespace ipfb
