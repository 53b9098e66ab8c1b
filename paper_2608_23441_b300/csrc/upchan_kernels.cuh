// Up-channelization kernel (Sec. 4.3: re-channelize the reconstructed stream with
// frames L samples long; here a plain real DFT of consecutive blocks).
//
// One block of L = 2Q real samples is read as Q complex values z[u] = x[2u] + i x[2u+1]
// arranged as U rows (frames) of P pairs: u = j*P + p.  Four-step DFT:
//   (1) U-point DFT over j for every p          -> y[k1][p]
//   (2) twiddle e^{-2 pi i p k1 / Q}
//   (3) P-point DFT over p for every k1         -> Z[k1 + U k2]
// then the real-input post-processing X[k] = E + e^{-2 pi i k/L} O from Z[k], Z[Q-k].
// A cluster of CU CTAs shares one block: CTA s holds pairs [s P', (s+1) P'), P' = P/CU.
// Step (3) splits as P = CU x P' (decimation in frequency): a CU-point DFT across
// CTAs (DSMEM, in place), twiddle e^{-2 pi i p' s / P}, then local P'-point DFTs,
// giving CTA s the outputs k2 = CU k2' + s.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"
#include "launch.h"

namespace ipfb {
namespace cg = cooperative_groups;

// Batched Stockham radix-R pass over NC sequences of length S.  Work item w covers
// sequence c = w % NC, butterfly b = w / NC when CFAST (sequences interleaved in
// memory), else b = w % nb, c = w / nb (sequences contiguous).  ld(c, i) / st(c, i, v).
struct NoPost {
  __device__ __forceinline__ void operator()(int, int, int, float2*) const {}
};

template <int R, int NC, int S, int T, bool INV, bool CFAST, class LD, class ST, class POST = NoPost>
__device__ __forceinline__ void batched_pass(int Ns, int tid, LD ld, ST st, POST post = POST{}) {
  constexpr int nb = S / R;
  constexpr int IPT = (NC * nb + T - 1) / T;
  float2 v[IPT][R];
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    const int w = tid + it * T;
    if (w < NC * nb) {
      const int c = CFAST ? w % NC : w / nb, b = CFAST ? w / NC : w % nb;
#pragma unroll
      for (int r = 0; r < R; ++r) v[it][r] = ld(c, b + r * nb);
      if (Ns > 1) apply_twiddles<R>(v[it], twiddle<INV>(b % Ns, Ns * R));
      DFT<R, INV>::run(v[it]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    const int w = tid + it * T;
    if (w < NC * nb) {
      const int c = CFAST ? w % NC : w / nb, b = CFAST ? w / NC : w % nb;
      const int k = b % Ns;
      const int j = (b / Ns) * Ns * R + k;
      post(c, j, Ns, v[it]);
#pragma unroll
      for (int r = 0; r < R; ++r) st(c, j + r * Ns, v[it][r]);
    }
  }
}

template <int NC, int S, int T, bool INV, bool CFAST, int Ns, class LDI, class STI, class STL, class POST = NoPost>
struct BatchedFFT {
  __device__ __forceinline__ static void run(int tid, LDI ldi, STI sti, STL stl, POST post = POST{}) {
    constexpr int R = next_radix(S, Ns);
    if constexpr (Ns * R == S) {
      batched_pass<R, NC, S, T, INV, CFAST>(Ns, tid, ldi, stl, post);
    } else {
      batched_pass<R, NC, S, T, INV, CFAST>(Ns, tid, ldi, sti);
      __syncthreads();
      BatchedFFT<NC, S, T, INV, CFAST, Ns * R, LDI, STI, STL, POST>::run(tid, ldi, sti, stl, post);
    }
  }
};

// Step-(2) twiddle of the up-channelizer applied to the R outputs k1 = j + r*Ns of
// one butterfly of pair p = p0 + c: exp(-2 pi i p k1 / Q) = base * step^r with
// base = exp(-2 pi i p j / Q), step = exp(-2 pi i p Ns / Q) (tables over L = 2Q).
template <int R>
struct UpchanTwiddle {
  Twid2<9> tw;
  int p0;
  __device__ __forceinline__ void operator()(int c, int j, int Ns, float2* v) const {
    const int p = p0 + c;
    const float2 base = tw(2 * p * j);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = cmul(v[r], base);
    apply_twiddles<R>(v, tw(2 * p * Ns));
  }
};

template <int CU, int U, int PP, int T>
__global__ void __launch_bounds__(T)
k4_upchan(UpchanSrc src, float2* __restrict__ out, float* __restrict__ x_out) {
  extern __shared__ float2 sm[];
  constexpr int P = CU * PP;
  constexpr int Q = U * P;
  constexpr int ROW = U + 1;  // transposed row stride after step (3)
  const int tid = threadIdx.x;
  int s = 0;
  if constexpr (CU > 1) s = (int)cg::this_cluster().block_rank();
  const long long b = blockIdx.x / CU;
  const int p0 = s * PP;
  // twiddle tables exp(-2 pi i t / L), L = 2Q, after the data array
  float2* tw_hi = sm + padded_len(U * PP);
  float2* tw_lo = tw_hi + 512;
  twid2_fill<9, false>(tw_hi, tw_lo, 2 * Q, tid, T);
  const Twid2<9> tw{tw_hi, tw_lo};

  // ---- load [U][PP] (element (j, p') at pidx(j*PP + p'))
  if (src.x) {
    const float2* x2 = reinterpret_cast<const float2*>(src.x) + b * (long long)Q;
#pragma unroll 8
    for (int idx = tid; idx < U * PP; idx += T) {
      const int j = idx / PP, pp = idx % PP;
      sm[pidx(idx)] = x2[(long long)j * P + p0 + pp];
    }
  } else {
    // d2[((p*C + r)*S + m)] holds frame C*m + r of pair p; this block is frames
    // [U b, U b + U).  Each thread reads the mpr consecutive m of one (pair, residue)
    // with 16-byte loads and scatters them to rows j = C*mm + r; consecutive lanes
    // take consecutive pairs, so the shared-memory writes are conflict free.
    const int C = src.C;
    const int mpr = U / C;  // frames per residue in this block (8 for U = 64, C = 8)
    const long long mbase = b * (long long)mpr;
    for (int idx = tid; idx < PP * C; idx += T) {
      const int pp = idx % PP, r = idx / PP;
      const float2* srcp = src.d2 + ((long long)(p0 + pp) * C + r) * src.S + mbase;
      if ((mpr & 1) == 0) {
        const float4* s4 = reinterpret_cast<const float4*>(srcp);
#pragma unroll 4
        for (int h = 0; h < mpr / 2; ++h) {
          const float4 v = s4[h];
          sm[pidx((C * (2 * h) + r) * PP + pp)] = make_float2(v.x, v.y);
          sm[pidx((C * (2 * h + 1) + r) * PP + pp)] = make_float2(v.z, v.w);
        }
      } else {
        for (int mm = 0; mm < mpr; ++mm) sm[pidx((C * mm + r) * PP + pp)] = srcp[mm];
      }
    }
  }
  __syncthreads();
  if (x_out) {
    float2* xo = reinterpret_cast<float2*>(x_out) + b * (long long)Q;
    for (int idx = tid; idx < U * PP; idx += T) {
      const int j = idx / PP, pp = idx % PP;
      xo[(long long)j * P + p0 + pp] = sm[pidx(idx)];
    }
  }

  // ---- (1) U-point DFT over j for each p', then (2) twiddle e^{-2 pi i p k1 / Q}
  {
    auto ld = [](int c, int i) { return sm[pidx(i * PP + c)]; };
    auto st = [](int c, int i, float2 v) { sm[pidx(i * PP + c)] = v; };
    constexpr int RL = last_radix(U);
    if constexpr (CU == 1) {
      const UpchanTwiddle<RL> post{tw, p0};
      BatchedFFT<PP, U, T, false, true, 1, decltype(ld), decltype(st), decltype(st), UpchanTwiddle<RL>>::run(
          tid, ld, st, st, post);
    } else {
      // the step-(2) twiddle is applied in the cross stage below
      BatchedFFT<PP, U, T, false, true, 1, decltype(ld), decltype(st), decltype(st)>::run(tid, ld, st, st);
    }
  }
  if constexpr (CU > 1) {
    cg::this_cluster().sync();
    // ---- cross-CTA CU-point DFT over q at each (k1, p'), twiddle e^{-2 pi i p' s'/P}
    float2* peer[CU];
#pragma unroll
    for (int q = 0; q < CU; ++q) peer[q] = cg::this_cluster().map_shared_rank(sm, q);
    for (int w = s * T + tid; w < U * PP; w += CU * T) {
      const int pp = w % PP, k1 = w / PP;
      float2 v[CU];
#pragma unroll
      for (int q = 0; q < CU; ++q) v[q] = peer[q][pidx(w)];
      // step (2): element (k1, p = q P' + p') of CTA q gets exp(-2 pi i p k1 / Q)
      //   = exp(-2 pi i p' k1 / Q) * exp(-2 pi i P' k1 / Q)^q
      {
        const float2 base = tw(2 * pp * k1);
#pragma unroll
        for (int q = 0; q < CU; ++q) v[q] = cmul(v[q], base);
        apply_twiddles<CU>(v, tw(2 * PP * k1));
      }
      DFT<CU, false>::run(v);
      float2 wr[CU];
      twiddle_powers<CU>(tw(2 * U * pp), wr);  // exp(-2 pi i p' / P)
#pragma unroll
      for (int q = 0; q < CU; ++q) peer[q][pidx(w)] = cmul(v[q], wr[q]);
    }
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
  // ---- (3) local P'-point DFT over p' for each k1; last pass stores transposed [k2'][k1]
  {
    auto ld = [](int c, int i) { return sm[pidx(c * PP + i)]; };
    auto st = [](int c, int i, float2 v) { sm[pidx(c * PP + i)] = v; };
    auto stl = [](int c, int i, float2 v) { sm[i * ROW + c] = v; };
    BatchedFFT<U, PP, T, false, false, 1, decltype(ld), decltype(st), decltype(stl)>::run(tid, ld, st, stl);
  }
  if constexpr (CU > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
  // ---- real-input post-processing, output k = k1 + U (CU k2' + s)
  float2* ob = out + b * (long long)(Q + 1);
  for (int w = tid; w < U * PP; w += T) {
    const int k1 = w % U, k2p = w / U;
    const float2 zk = sm[k2p * ROW + k1];
    float2 zm;
    int ps, pk1, pk2p;
    if (k1 != 0) {
      ps = CU - 1 - s;
      pk1 = U - k1;
      pk2p = PP - 1 - k2p;
    } else if (s == 0) {
      ps = 0;
      pk1 = 0;
      pk2p = (PP - k2p) % PP;
    } else {
      ps = CU - s;
      pk1 = 0;
      pk2p = PP - k2p - 1;
    }
    if constexpr (CU > 1)
      zm = cg::this_cluster().map_shared_rank(sm, ps)[pk2p * ROW + pk1];
    else
      zm = sm[pk2p * ROW + pk1];
    const int k = k1 + U * (CU * k2p + s);
    const float2 E = cscale(cadd(zk, cconj(zm)), 0.5f);
    const float2 dd = csub(zk, cconj(zm));
    const float2 O = make_float2(0.5f * dd.y, -0.5f * dd.x);
    const float2 wk = tw(k);
    ob[k] = cadd(E, cmul(wk, O));
    if (k == 0) ob[Q] = make_float2(zk.x - zk.y, 0.0f);
  }
  // Peers may still read this CTA's shared memory: wait for them before exiting.  The
  // arrive is relaxed (no release fence): nothing written here is read after the
  // barrier, and a release would hold every thread until its output stores drain.
  if constexpr (CU > 1) {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.aligned;\n" ::: "memory");
  }
}

}  // namespace ipfb
