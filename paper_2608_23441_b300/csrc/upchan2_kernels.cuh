// Up-channelization of the column-pair scratch in two passes through HBM (Sec. 4.3:
// re-channelize the reconstructed stream with frames L = 64 N samples long; here a
// plain real DFT of consecutive blocks).
//
// One block of L = 2Q real samples is Q complex values z[u] = x[2u] + i x[2u+1],
// u = j P + p: 64 frames j of P = N/2 column pairs p.  The Q-point DFT factors as
// 64 (frames) x PA x PB with p = PB pa + pb (PB = 64, PA = P / 64) and output index
//   k = k1 + 64 k2,   k2 = k2a + PA k2b:
//   Z[k] = sum_pb w_PB^(pb k2b) [ w_P^(pb k2a) sum_pa w_PA^(pa k2a)
//                                   [ w_Q^(p k1) sum_j w_64^(j k1) z[j P + p] ] ]
// (w_n = exp(-2 pi i / n)), then the real-input post-processing
//   X[k] = E + exp(-2 pi i k / L) O,  E = (Z[k] + conj Z[Q-k]) / 2,
//   O = -i (Z[k] - conj Z[Q-k]) / 2,  X[Q] = Re Z[0] - Im Z[0].
//
// k4a: per tile (block b, NPB = 128 / PA consecutive pb, all pa: 128 pairs) the
//   64-point frames DFT, the w_Q twiddle, the PA-point DFT over pa and the w_P
//   twiddle; writes W[b][k2a][k1][pb] (NPB-element runs).  Its input is the scratch
//   in the block-major order the column kernel writes for it (frame j of pair p at
//   p J + 64 (j >> 6) + 8 (j & 7) + ((j >> 3) & 7)), so a tile is 128 contiguous
//   512-byte runs.
// k4b: per CTA (block b, a < PA/2) the 64-point DFTs over pb of the 128 rows
//   (k2a, k1) with k2a in {a, PA-1-a} (both contiguous 32 KB slabs of W), which
//   holds the partner Z[Q-k] of every output it writes (k1 != 0: row (PA-1-k2a,
//   64-k1)); for k1 = 0 the partner rows k2a' = PA - k2a are loaded as two extra
//   rows.  Outputs for fixed (k2a, k2b) are the 64 consecutive k1: contiguous runs.
// Both are ordinary kernels (no clusters); the cross-CTA exchange of a one-pass
// design is replaced by one round trip of the block set through HBM.
#pragma once

#include "common.cuh"
#include "launch.h"

namespace ipfb {

constexpr int kK4aThreads = 256;
constexpr int kK4bThreads = 256;

template <int P>
struct K4Shape {
  static constexpr int PB = 64;
  static constexpr int PA = P / PB;
  static constexpr int NPB = 128 / PA;  // pb per k4a tile (128 pairs per tile)
  static constexpr int Q = 64 * P;
  static_assert(PA >= 2 && PA <= 128 && NPB >= 1, "P in [128, 8192]");
};

// ---------------------------------------------------------------------------
// k4a.  Shared array [64 rows][128 columns] (no padding), column swizzled per row:
// rows hold the frames-DFT state (row = 8 k1a + rt, then 8 k1a + k1b: each thread
// reads and writes the same 8 slots), column = local pair q = pa NPB + pbl.  The
// XOR swizzle puts the PA-point reads of k4a's last stage (lanes = pbl fastest,
// then k1) into distinct banks.
// ---------------------------------------------------------------------------
template <int NPB>
__device__ __forceinline__ int k4a_slot(int row, int q) {
  constexpr int KM = 16 / NPB > 1 ? 16 / NPB - 1 : 0;
  return row * 128 + (q ^ (((row >> 3) & KM) * NPB));
}

template <int P>
__global__ void __launch_bounds__(kK4aThreads)
k4a_frames(const float2* __restrict__ d2, int J, long long nblocks, float2* __restrict__ W,
           float2* __restrict__ x2_out) {
  using K = K4Shape<P>;
  constexpr int T = kK4aThreads;
  constexpr int Q = K::Q, PA = K::PA, NPB = K::NPB;
  extern __shared__ __align__(16) float2 smk4a[];
  float2* buf = smk4a;                // 64 x 128 frames-DFT state
  float2* stage = buf + 64 * 128;     // 128 x 66 raw staging (asynchronous copies)
  float2* tw_hi = stage + 128 * 66;   // Q >> 9
  float2* tw_lo = tw_hi + (Q >> 9);   // 512
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  twid2_fill<9, false>(tw_hi, tw_lo, Q, tid, T);
  const Twid2<9> tw{tw_hi, tw_lo};
  const long long ntiles = nblocks * (K::PB / NPB);
  // pair group fastest: the PB / NPB tiles of one block, which together fill whole
  // 512-byte rows of W, run at the same time, so those rows leave L2 complete.
  // A tile's input is 128 contiguous 512-byte blocks (one per pair, the column
  // kernel's block-major output: 8 residues rt x 8 consecutive m'); warp w copies
  // blocks q = w + 8 i whole into the staging rows [q][66] (float4-aligned rows,
  // conflict-free 16-byte accesses) with asynchronous 16-byte copies, the next
  // tile's while this one is computed.
  auto prefetch = [&](long long tile) {
    const long long b = tile / (K::PB / NPB);
    const int pb0 = (int)(tile % (K::PB / NPB)) * NPB;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int q = warp + 8 * i;
      const int p = K::PB * (q / NPB) + pb0 + (q % NPB);
      cp_async16(reinterpret_cast<float4*>(stage) + q * 33 + lane,
                 reinterpret_cast<const float4*>(d2 + (long long)p * J + b * 64) + lane);
    }
    cp_async_commit();
  };
  if ((long long)blockIdx.x < ntiles) prefetch(blockIdx.x);
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long b = tile / (K::PB / NPB);
    const int pb0 = (int)(tile % (K::PB / NPB)) * NPB;
    // ---- (a) the tile's copies have landed; thread (q, rt) takes its 8 frames
    cp_async_wait_all();
    __syncthreads();
    float2 v4[4][8];
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int q = tid & 127, rt = (tid >> 7) + 2 * it;
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const float4 w4 = reinterpret_cast<const float4*>(stage)[q * 33 + rt * 4 + h];
        v4[it][2 * h] = make_float2(w4.x, w4.y);
        v4[it][2 * h + 1] = make_float2(w4.z, w4.w);
      }
    }
    __syncthreads();  // every read of the staging area is done: prefetch the next tile
    if (tile + gridDim.x < ntiles) prefetch(tile + gridDim.x);
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int q = tid & 127, rt = (tid >> 7) + 2 * it;
      const int p = K::PB * (q / NPB) + pb0 + (q % NPB);
      float2* v = v4[it];
      if (x2_out) {
#pragma unroll
        for (int m = 0; m < 8; ++m) x2_out[(b * 64 + 8 * m + rt) * P + p] = v[m];
      }
      DFT<8, false>::run(v);
      if (rt) apply_twiddles<8>(v, tw(rt * P));  // w_64^rt = w_Q^(rt P)
#pragma unroll
      for (int k = 0; k < 8; ++k) buf[k4a_slot<NPB>(8 * k + rt, q)] = v[k];
    }
    __syncthreads();
    // ---- (b) DFT over rt (k1 = k1a + 8 k1b), twiddle w_Q^(p k1); same 8 slots
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int q = tid & 127, k1a = (tid >> 7) + 2 * it;
      const int p = K::PB * (q / NPB) + pb0 + (q % NPB);
      float2 v[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) v[r] = buf[k4a_slot<NPB>(8 * k1a + r, q)];
      DFT<8, false>::run(v);
      const float2 base = tw(p * k1a), step = tw(p * 8);
      v[0] = cmul(v[0], base);
      float2 w = base;
#pragma unroll
      for (int k = 1; k < 8; ++k) {
        w = cmul(w, step);
        v[k] = cmul(v[k], w);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) buf[k4a_slot<NPB>(8 * k1a + k, q)] = v[k];
    }
    __syncthreads();
    // ---- (c) PA-point DFT over pa for each (k1, pbl), twiddle w_P^(pb k2a), store W
    constexpr int NIT = (64 * NPB + T - 1) / T;
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
      const int item = tid + it * T;
      if (item < 64 * NPB) {
        const int pbl = item % NPB, k1 = item / NPB;
        const int row = 8 * (k1 & 7) + (k1 >> 3);
        float2 v[PA];
#pragma unroll
        for (int pa = 0; pa < PA; ++pa) v[pa] = buf[k4a_slot<NPB>(row, pa * NPB + pbl)];
        DFT<PA, false>::run(v);
        const int pb = pb0 + pbl;
        apply_twiddles<PA>(v, tw(64 * pb));  // w_P^pb = w_Q^(64 pb)
        float2* wb = W + ((b * PA) * 64 + k1) * 64 + pb;
#pragma unroll
        for (int k2a = 0; k2a < PA; ++k2a) wb[(long long)k2a * 64 * 64] = v[k2a];
      }
    }
    __syncthreads();  // buf is reused by the next tile
  }
}

// ---------------------------------------------------------------------------
// k4b.  Rows rho of 64 elements, element c of row rho at rho 64 + (k4b_col(c) ^
// k4b_rowx(rho)): the column swizzle k4b_col puts the radix-8 accesses of one row
// (columns 8 bf + r and bf + 8 r, lanes bf) into distinct banks, and the row XOR
// puts the two rows of a half-warp into opposite halves of the banks (FFT passes)
// and any 16 consecutive rows at one column into distinct banks (post-processing).
// Rows: 0..63 = (a, k1), 64..127 = (PA-1-a, k1), 128 = (PA-a mod PA,
// 0), 129 = (a+1 mod PA, 0).  Tables: w_128^n (the 64-point FFT twiddles and the
// k2b part of exp(-2 pi i k / L)) and w_L^(k1 + 64 k2a) per row.
// ---------------------------------------------------------------------------
constexpr int kK4bRS = 64;
constexpr int kK4bRows = 130;
// column swizzle inside a row: the radix-8 passes access columns 8 bf + r and bf + 8 r
// (lanes bf); c ^ ((c >> 3) & 7) maps both onto distinct banks
__device__ __forceinline__ int k4b_col(int c) { return c ^ ((c >> 3) & 7); }
__device__ __forceinline__ int k4b_rowx(int rho) { return ((rho & 1) << 3) | ((rho >> 1) & 7); }
__device__ __forceinline__ int k4b_at(int rho, int c) { return rho * kK4bRS + (k4b_col(c) ^ k4b_rowx(rho)); }

template <int P>
constexpr size_t k4b_smem_bytes() {
  return (size_t)(kK4bRows * kK4bRS + 128 + kK4bRows) * sizeof(float2);
}

template <int P>
__global__ void __launch_bounds__(kK4bThreads)
k4b_pairs(const float2* __restrict__ W, float2* __restrict__ out) {
  using K = K4Shape<P>;
  constexpr int T = kK4bThreads;
  constexpr int Q = K::Q, PA = K::PA, L = 2 * Q;
  constexpr int RS = kK4bRS;
  extern __shared__ float2 smk4b[];
  float2* rows = smk4b;
  float2* t128 = rows + kK4bRows * RS;
  float2* rb = t128 + 128;
  const int tid = threadIdx.x;
  const long long b = blockIdx.x / (PA / 2);
  const int a = blockIdx.x % (PA / 2);
  // k2a of the four row groups: a, PA-1-a, and the k1 = 0 partners PA-a, a+1 (mod PA)
  auto ka = [a](int i) { return i == 0 ? a : (i == 1 ? PA - 1 - a : (i == 2 ? (PA - a) % PA : (a + 1) % PA)); };
  for (int i = tid; i < 128; i += T) t128[i] = twiddle<false>(i, 128);
  for (int i = tid; i < kK4bRows; i += T) {
    const int k1 = i < 128 ? (i & 63) : 0;
    const int k2a = ka(i < 128 ? (i >> 6) : (i - 126));
    rb[i] = twiddle<false>(k1 + 64 * k2a, L);
  }
  // ---- load: two 4096-element slabs (rows 0..127) and two 64-element rows.  With
  // 256 threads, thread tid always handles the element pair pb = 2 (tid & 31) of rows
  // k1 = (tid >> 5) + 8 i: the column and the swizzle are fixed per thread.
  static_assert(T == 256, "index plan assumes 256 threads");
  {
    const int pb = (tid & 31) * 2, k1b = tid >> 5;
    // odd lanes store their second element first: each store instruction then puts
    // the 16 lanes of a half-warp into 16 distinct bank pairs
    const bool sw = tid & 1;
    const int ca = sw ? pb + 1 : pb, cb = sw ? pb : pb + 1;
    auto put = [&](int rho, float4 u) {
      rows[k4b_at(rho, ca)] = sw ? make_float2(u.z, u.w) : make_float2(u.x, u.y);
      rows[k4b_at(rho, cb)] = sw ? make_float2(u.x, u.y) : make_float2(u.z, u.w);
    };
    const float4* s0 = reinterpret_cast<const float4*>(W + ((b * PA + ka(0)) * 64) * 64 + pb);
    const float4* s1 = reinterpret_cast<const float4*>(W + ((b * PA + ka(1)) * 64) * 64 + pb);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      float4 u[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) u[i] = (half ? s1 : s0)[(k1b + 8 * i) * 32];
#pragma unroll
      for (int i = 0; i < 8; ++i) put(half * 64 + k1b + 8 * i, u[i]);
    }
    if (tid < 64) {
      const int x = tid >> 5;
      put(128 + x, *reinterpret_cast<const float4*>(W + ((b * PA + ka(2 + x)) * 64) * 64 + pb));
    }
  }
  __syncthreads();
  // ---- 64-point forward DFT of every row: two radix-8 Stockham passes, 8 lanes per
  // row (4 rows per warp), synchronised within the warp only
  {
    const int lane = tid & 31, warp = tid >> 5;
    for (int rg = warp; rg < (kK4bRows + 3) / 4; rg += T / 32) {
      const int rho = rg * 4 + (lane >> 3), bf = lane & 7;
      const bool ok = rho < kK4bRows;
      float2* row = rows + (ok ? rho : 0) * RS;
      const int rx = k4b_rowx(ok ? rho : 0);
      float2 v[8];
      if (ok) {
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] = row[k4b_col(bf + 8 * r) ^ rx];
        DFT<8, false>::run(v);
      }
      __syncwarp();
      if (ok) {
#pragma unroll
        for (int r = 0; r < 8; ++r) row[k4b_col(8 * bf + r) ^ rx] = v[r];  // Ns = 1: output 8 bf + r
      }
      __syncwarp();
      if (ok) {
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] = row[k4b_col(bf + 8 * r) ^ rx];
        if (bf) apply_twiddles<8>(v, t128[2 * bf]);  // w_64^bf
        DFT<8, false>::run(v);
#pragma unroll
        for (int r = 0; r < 8; ++r) row[k4b_col(bf + 8 * r) ^ rx] = v[r];  // Ns = 8: output bf + 8 r
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // ---- post-processing and contiguous stores: w = (half, k2b, k1), k1 fastest.  With
  // 256 threads k1 = tid & 63 is fixed per thread, so the partner row and the per-row
  // twiddle are too; only k2b and the half change across the unrolled iterations.
  float2* ob = out + b * (long long)(Q + 1);
  {
    const int k1 = tid & 63, k2b0 = tid >> 6;
    int rho_h[2], rp_h[2], k2a_h[2];
    bool dc_wrap[2];
    float2 rb_h[2];
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      const int k2a = ka(hf);
      k2a_h[hf] = k2a;
      rho_h[hf] = hf * 64 + k1;
      rb_h[hf] = rb[hf * 64 + k1];
      dc_wrap[hf] = (k1 == 0 && k2a == 0);
      if (k1 != 0) {
        rp_h[hf] = (1 - hf) * 64 + (64 - k1);
      } else {
        const int kp = (PA - k2a) % PA;
        rp_h[hf] = kp == ka(0) ? 0 : (kp == ka(1) ? 64 : (kp == ka(2) ? 128 : 129));
      }
    }
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
#pragma unroll 4
    for (int i = 0; i < 16; ++i) {
      const int k2b = k2b0 + 4 * i;
      // partner mode: k2b' = 63 - k2b, except the DC row (k1 = 0, k2a = 0): (64 - k2b) mod 64
      const int k2bp = dc_wrap[hf] ? ((64 - k2b) & 63) : 63 - k2b;
      const float2 zk = rows[k4b_at(rho_h[hf], k2b)];
      const float2 zm = rows[k4b_at(rp_h[hf], k2bp)];
      const float2 E = cscale(cadd(zk, cconj(zm)), 0.5f);
      const float2 dd = csub(zk, cconj(zm));
      const float2 O = make_float2(0.5f * dd.y, -0.5f * dd.x);
      const long long k = k1 + 64 * k2a_h[hf] + 64LL * PA * k2b;
      ob[k] = cadd(E, cmul(cmul(rb_h[hf], t128[k2b]), O));
      if (k == 0) ob[Q] = make_float2(zk.x - zk.y, 0.0f);
    }
    }
  }
}

}  // namespace ipfb
