// Batched inverse PFB of many independent streams with uneven shapes (lblock and
// any integer number of frames J), processed by persistent kernels that pull work
// items from a global counter.
//
// The per-column circulant decorrelation (Eq. decorrelation, Eq. wiener weights)
// needs the J-point DFT for an arbitrary J.  It is computed with Bluestein's
// chirp-z identity (Bluestein 1970):  n k = (n^2 + k^2 - (k - n)^2) / 2, so with
// w[n] = exp(-i pi n^2 / J)
//     X[k] = w[k] * sum_n (x[n] w[n]) conj(w[k - n]),
// a circular convolution of length M >= 2J - 1 (a power of two) evaluated as
// FFT_M -> x FFT_M(b) -> IFFT_M with b[m] = conj(w[m]) (and b[M - m] = b[m]).
// The inverse J-point DFT uses the same convolution on conj(X).  A cluster of C
// CTAs holds one length-M sequence, CTA r owning indices C m + r (the K3 layout).
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"
#include "ipfb_kernels.cuh"
#include "launch.h"

namespace ipfb {
namespace cg = cooperative_groups;

struct BStream {
  int N, J, M, ntap;
  float phi2, gnorm, invJ;
  int pad_;
  const uint8_t* codes;   // [J][N/2]
  const float* scale;     // [N/2 + 1]
  const float* window;    // [ntap][N]
  float* x_out;           // [J*N] time order
  float2* d2;             // [N/2][J] column pairs (workspace)
  const float2* chirp;    // [J]  w[n] = exp(-i pi n^2 / J)   (workspace, shared per J)
  const float2* bhat;     // [M]  FFT_M(b)                     (workspace, shared per J)
};

// Work item lists (host-built, sorted longest first):
//   kb2: (stream, first frame)      kb3: (stream, column pair)      kb4: (stream, tile)
struct BItem {
  int s, a;
};

// The non-template kernels below are compiled in one translation unit only
// (batched.cu defines IPFB_BATCHED_HOST_KERNELS); the kb3 variant units skip them.
#ifdef IPFB_BATCHED_HOST_KERNELS
// ---------------------------------------------------------------- chirp tables
// w[n] = exp(-i pi (n^2 mod 2J) / J) for n < J, per distinct J
__global__ void kb_chirp(const int* __restrict__ Js, float2* const* __restrict__ out, int nJ) {
  const int t = blockIdx.y;
  if (t >= nJ) return;
  const int J = Js[t];
  float2* w = out[t];
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < J; n += gridDim.x * blockDim.x) {
    const long long q = ((long long)n * n) % (2LL * J);
    float s, c;
    sincospif(__fdiv_rn((float)q, (float)J), &s, &c);
    w[n] = make_float2(c, -s);
  }
}

#endif  // IPFB_BATCHED_HOST_KERNELS

// C-point DFT of the cluster cross stage: the radix-2 form of DFT<C> for a power of
// two, otherwise (the 5- and 6-CTA clusters) the direct sum out[k] = sum_j v[j] W_C^{jk}
// with j k reduced mod C at compile time.
template <int R, bool INV, int K, int... Js>
__device__ __forceinline__ float2 direct_dft_term(const float2* v, std::integer_sequence<int, Js...>) {
  float2 acc = v[0];
  ((acc = cadd(acc, rot_const<((Js + 1) * K) % R, R, INV>(v[Js + 1]))), ...);
  return acc;
}
template <int R, bool INV, int... Ks>
__device__ __forceinline__ void direct_dft(float2* v, std::integer_sequence<int, Ks...>) {
  float2 out[R];
  ((out[Ks] = direct_dft_term<R, INV, Ks>(v, std::make_integer_sequence<int, R - 1>{})), ...);
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = out[k];
}
template <int R, bool INV>
__device__ __forceinline__ void cluster_dft(float2* v) {
  if constexpr ((R & (R - 1)) == 0)
    DFT<R, INV>::run(v);
  else
    direct_dft<R, INV>(v, std::make_integer_sequence<int, R>{});
}

// ---------------------------------------------------------------- cluster engine
// In: this CTA's S values a[C m + r] at sm[pidx(m)].  Out (CONV): the unnormalised
// circular convolution (a (*) b)[C m + r] * M at sm[pidx(m)], with bhat = FFT_M(b).
// Out (forward only): FFT_M(a)[k] written to fwd_out[k] (global), sm clobbered.
template <int C, int S, int T, int MAXR, bool FWD_ONLY>
__device__ __forceinline__ void conv_engine(float2* sm, const float2* __restrict__ bhat, float2* fwd_out, int r) {
  constexpr int M = C * S;
  const int tid = threadIdx.x;
  block_fft<S, T, false, MAXR>(sm, tid, SPad{sm}, SPad{sm});
  if constexpr (C > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
  auto peer = [sm](int q) -> float2* {
    if constexpr (C > 1)
      return cg::this_cluster().map_shared_rank(sm, q);
    else
      return sm;
  };
  for (int kb = r * T + tid; kb < S; kb += C * T) {
    float2 z[C];
    float2 w0[C];
    if constexpr (C > 1) twiddle_powers<C>(twiddle<false>(kb, M), w0);
#pragma unroll
    for (int q = 0; q < C; ++q) z[q] = peer(q)[pidx(kb)];
    if constexpr (C > 1) {
#pragma unroll
      for (int q = 1; q < C; ++q) z[q] = cmul(z[q], w0[q]);
      cluster_dft<C, false>(z);
    }
    if constexpr (FWD_ONLY) {
#pragma unroll
      for (int ka = 0; ka < C; ++ka) fwd_out[kb + S * ka] = z[ka];
    } else {
#pragma unroll
      for (int ka = 0; ka < C; ++ka) z[ka] = cmul(z[ka], __ldg(bhat + kb + S * ka));
      if constexpr (C > 1) {
        cluster_dft<C, true>(z);
#pragma unroll
        for (int q = 1; q < C; ++q) z[q] = cmul(z[q], cconj(w0[q]));
      }
#pragma unroll
      for (int q = 0; q < C; ++q) peer(q)[pidx(kb)] = z[q];
    }
  }
  if constexpr (C > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
  if constexpr (!FWD_ONLY) {
    block_fft<S, T, true, MAXR>(sm, tid, SPad{sm}, SPad{sm});
    __syncthreads();
  }
}

// ---------------------------------------------------------------- B-hat tables
// One cluster per distinct J: b[m] = conj(w[m]) (m < J), b[M - m] = conj(w[m]) (0 < m < J)
template <int C, int S, int T, int MAXR>
__device__ __forceinline__ void bhat_item(const float2* __restrict__ w, int J, float2* bhat, float2* sm, int r) {
  constexpr int M = C * S;
  for (int m = threadIdx.x; m < S; m += T) {
    const int n = C * m + r;
    float2 v = make_float2(0.0f, 0.0f);
    if (n < J)
      v = cconj(w[n]);
    else if (n > M - J)
      v = cconj(w[M - n]);
    sm[pidx(m)] = v;
  }
  __syncthreads();
  conv_engine<C, S, T, MAXR, true>(sm, nullptr, bhat, r);
}

// ---------------------------------------------------------------- column item
// One column pair of one stream: forward Bluestein, pair split + Wiener gain,
// inverse Bluestein, in place on d2.
template <int C, int S, int T, int MAXR>
__device__ __forceinline__ void column_item(const BStream& st, int p, float2* sm, int r) {
  const int J = st.J;
  constexpr int M = C * S;
  float2* col = st.d2 + (size_t)p * J;
  const float2* w = st.chirp;
  const float invM = 1.0f / (float)M;
  // 1. a[n] = z[n] w[n], zero padded
#pragma unroll 1
  for (int m = threadIdx.x; m < S; m += T) {
    const int n = C * m + r;
    sm[pidx(m)] = (n < J) ? cmul(col[n], __ldg(w + n)) : make_float2(0.0f, 0.0f);
  }
  __syncthreads();
  conv_engine<C, S, T, MAXR, false>(sm, st.bhat, nullptr, r);
  // 2. X[k] = w[k] conv[k] / M for own k
#pragma unroll 1
  for (int m = threadIdx.x; m < S; m += T) {
    const int k = C * m + r;
    if (k < J) sm[pidx(m)] = cscale(cmul(__ldg(w + k), sm[pidx(m)]), invM);
  }
  if constexpr (C > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
  // 3. pair split + gain: partner -k mod J lives in CTA (-k mod J) % C, so X'[k] may
  //    overwrite X only once every partner read is done.  S >= 4096: X'[k] stays in
  //    registers across a cluster barrier, then goes in place (one buffer, two CTAs per
  //    SM at S = 8192); smaller S: it goes to a second buffer sm2 (holding 8 or more
  //    values per thread across the rare out-of-line FP64 gain call spills there).  One
  //    CTA (C = 1) holds both modes of every pair, so one thread splits k and J - k in
  //    place.
  float ta[4], tb[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    ta[t] = __ldg(st.window + (size_t)t * st.N + 2 * p);
    tb[t] = __ldg(st.window + (size_t)t * st.N + 2 * p + 1);
  }
  GainParams gp;
  gp.phi2 = st.phi2;
  gp.gnorm = st.gnorm;
  gp.invJ = st.invJ;
  gp.J = J;
  gp.out_block_major = 0;
  gp.ntap = 4;
  if constexpr (C == 1) {
#pragma unroll 1
    for (int k = threadIdx.x; k <= J / 2; k += T) {
      const int km = (J - k) % J;
      float2 xk = sm[pidx(k)], xm = sm[pidx(km)];
      const float2 e1 = twiddle<false>(k, J);
      const float2 ga = gain_at<4>(ta, k, e1, gp), gb = gain_at<4>(tb, k, e1, gp);
      split_gain(xk, xm, ga, gb);
      // 4. the inverse transform's input: a'[k] = conj(X'[k]) w[k]
      sm[pidx(k)] = cmul(cconj(xk), __ldg(w + k));
      if (km != k) sm[pidx(km)] = cmul(cconj(xm), __ldg(w + km));
    }
#pragma unroll 1
    for (int k = J + threadIdx.x; k < S; k += T) sm[pidx(k)] = make_float2(0.0f, 0.0f);  // zero padding
    __syncthreads();
  } else if constexpr (S < 4096) {
    float2* sm2 = sm + padded_len(S);
#pragma unroll 1
    for (int m = threadIdx.x; m < S; m += T) {
      const int k = C * m + r;
      float2 xk = make_float2(0.0f, 0.0f);
      if (k < J) {
        const int km = (k == 0) ? 0 : J - k;
        const float2* src = cg::this_cluster().map_shared_rank(sm, km % C);
        float2 zm = src[pidx(km / C)];
        xk = sm[pidx(m)];
        const float2 e1 = twiddle<false>(k, J);
        const float2 ga = gain_at<4>(ta, k, e1, gp), gb = gain_at<4>(tb, k, e1, gp);
        split_gain(xk, zm, ga, gb);
        xk = cmul(cconj(xk), __ldg(w + k));  // 4. a'[k] = conj(X'[k]) w[k]
      }
      sm2[pidx(m)] = xk;
    }
    cg::this_cluster().sync();
#pragma unroll 1
    for (int m = threadIdx.x; m < S; m += T) sm[pidx(m)] = sm2[pidx(m)];
    __syncthreads();
  } else {
    constexpr int PER = (S + T - 1) / T;
    float2 xo[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int m = threadIdx.x + i * T;
      const int k = C * m + r;
      float2 xk = make_float2(0.0f, 0.0f);
      if (m < S && k < J) {
        const int km = (k == 0) ? 0 : J - k;
        const float2* src = sm;
        if constexpr (C > 1) src = cg::this_cluster().map_shared_rank(sm, km % C);
        float2 zm = src[pidx(km / C)];
        xk = sm[pidx(m)];
        const float2 e1 = twiddle<false>(k, J);
        const float2 ga = gain_at<4>(ta, k, e1, gp), gb = gain_at<4>(tb, k, e1, gp);
        split_gain(xk, zm, ga, gb);
        // 4. the inverse transform's input: a'[k] = conj(X'[k]) w[k]
        xk = cmul(cconj(xk), __ldg(w + k));
      }
      xo[i] = xk;
    }
    if constexpr (C > 1) {
      cg::this_cluster().sync();  // every CTA has read its partners' unmodified X
    } else {
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int m = threadIdx.x + i * T;
      if (m < S) sm[pidx(m)] = xo[i];
    }
    __syncthreads();
  }
  conv_engine<C, S, T, MAXR, false>(sm, st.bhat, nullptr, r);
  // 5. x[j] = conj(w[j] conv'[j] / M)
#pragma unroll 1
  for (int m = threadIdx.x; m < S; m += T) {
    const int j = C * m + r;
    if (j < J) col[j] = cconj(cscale(cmul(__ldg(w + j), sm[pidx(m)]), invM));
  }
}

// ---------------------------------------------------------------- persistent kernels
// Work fetch: one thread takes the next item index from the counter and the CTA
// (or the whole cluster, through rank 0's shared memory) reads it.
__device__ __forceinline__ int fetch_item_cta(int* counter, int* slot) {
  if (threadIdx.x == 0) *slot = atomicAdd(counter, 1);
  __syncthreads();
  const int v = *slot;
  __syncthreads();
  return v;
}

template <int C>
__device__ __forceinline__ int fetch_item_cluster(int* counter, int* slot, int r) {
  if constexpr (C == 1) {
    return fetch_item_cta(counter, slot);
  } else {
    if (r == 0 && threadIdx.x == 0) *slot = atomicAdd(counter, 1);
    cg::this_cluster().sync();
    const int v = *cg::this_cluster().map_shared_rank(slot, 0);
    cg::this_cluster().sync();
    return v;
  }
}

// kb2: unpack + per-frame inverse real FFT, one kernel per lblock N = 2H (the items of
// the streams of that lblock; F spectra of TPF threads each per item, as k2), so each
// is register-allocated for its own shape (one kernel switching over the three took
// 128 registers and spilled).  FULL: items of exactly F spectra (the group size is a
// compile-time constant, as in k2); otherwise the last, shorter item of each stream.
constexpr int kKb2Threads = 512;
#ifdef IPFB_BATCHED_HOST_KERNELS
template <int H, int TPF, int F, bool FULL>
__global__ void __launch_bounds__(TPF* F, (H == 512 ? 1 : 2))
kb2_unpack(const BStream* __restrict__ streams, const BItem* __restrict__ items, int nitems, int* counter) {
  static_assert(TPF * F == kKb2Threads, "512 threads");
  extern __shared__ float2 smem[];
  __shared__ int slot;
  for (int guard = 0; guard < nitems + 1; ++guard) {
    const int it = fetch_item_cta(counter, &slot);
    if (it >= nitems) break;
    const BItem item = items[it];
    const BStream& st = streams[item.s];
    if (st.N == 2 * H)  // always true within the list
      k2_group<H, TPF, F>(st.codes, st.scale, st.d2, 1, st.J, 0, item.a, FULL ? F : min(F, st.J - item.a), smem);
    __syncthreads();
  }
}

#endif  // IPFB_BATCHED_HOST_KERNELS

// kb3: columns (4-tap windows); a cluster of C CTAs per item, M = C * S with S
// picked per item.  Dynamic smem: one padded S-element buffer (two for a cluster
// with S < 4096).
// One launch per M class: every item of the class has M = C * S, so each kernel is
// specialised to its S (one kernel switching over all S was register-allocated for
// the largest and spilled ~3.7 KB per thread), and limited to 128 registers so two
// CTAs share an SM (measured faster than one CTA with 255 registers).
// CTAs per SM the register budget is set for: two (at most 128 registers) in general,
// three (at most 80) for the 5- and 6-CTA clusters and the single-CTA 4096-point run
// (measured faster despite 88-160 bytes of spills per thread), one for the single-CTA
// 512-thread variant and the 16384-element runs.
template <int C, int S, int T>
constexpr int kb3_min_blocks() {
  if (C == 1) return (S == 4096 && T == 256) ? 3 : ((T <= 256 && S <= 32 * T) ? 2 : 1);
  if (S > 8192) return 1;
  return (C == 5 || C == 6) ? 3 : 2;
}
template <int C, int S, int T, int MAXR>
__global__ void __launch_bounds__(T, kb3_min_blocks<C, S, T>())
kb3_columns(const BStream* __restrict__ streams, const BItem* __restrict__ items, int nitems, int* counter) {
  extern __shared__ float2 smem[];
  (void)counter;
  int r = 0;
  if constexpr (C > 1) r = (int)cg::this_cluster().block_rank();
  // Static round-robin over the class's items (all of one M, so of nearly one cost;
  // the host sorts them longest first): every CTA of a cluster walks the same item
  // sequence, so no cluster barrier is spent on fetching work.  No barrier is needed
  // between items either: an item's last remote shared-memory access precedes its
  // last cluster barrier, and the next item's first one follows the next item's
  // first cluster barrier.
  const int ncl = (int)gridDim.x / C, cl = (int)blockIdx.x / C;
  for (int it = cl; it < nitems; it += ncl) {
    const BItem item = items[it];
    const BStream& st = streams[item.s];
    if (st.M == C * S) column_item<C, S, T, MAXR>(st, item.a, smem, r);  // always true within a class
    if constexpr (C == 1) __syncthreads();
  }
}

// Launch of the class-M kernel of one variant: a persistent grid of as many clusters
// as fit, each CTA with S padded elements of shared memory.
template <int C, int T, int MAXR>
struct Kb3Launch {
  template <int S>
  static cudaError_t go(const BStream* s, const BItem* it, int n, int* ctr, cudaStream_t stream, int* nclusters) {
    auto kern = kb3_columns<C, S, T, MAXR>;
    // one buffer (the pair split in place: one CTA, or across a cluster barrier for
    // S >= 4096), two for a cluster with S < 4096 (the split through a second buffer)
    const size_t smem = (C > 1 && S < 4096 ? 2 : 1) * (size_t)padded_len(S) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(T);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(C);
    int nc = 0;
    e = cudaOccupancyMaxActiveClusters(&nc, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (nc < 1) nc = 1;
    if (nc > n) nc = n;
    *nclusters = nc;
    cfg.gridDim = dim3(nc * C);
    e = cudaLaunchKernelEx(&cfg, kern, s, it, n, ctr);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  static cudaError_t launch(int M, const BStream* s, const BItem* it, int n, int* ctr, cudaStream_t stream,
                            int* nclusters) {
    if constexpr (C == 1) {
      if (M == 16384) return go<16384>(s, it, n, ctr, stream, nclusters);
    }
    switch (M / C) {
      case 512: return go<512>(s, it, n, ctr, stream, nclusters);
      case 1024: return go<1024>(s, it, n, ctr, stream, nclusters);
      case 2048: return go<2048>(s, it, n, ctr, stream, nclusters);
      case 4096: return go<4096>(s, it, n, ctr, stream, nclusters);
      case 8192: return go<8192>(s, it, n, ctr, stream, nclusters);
    }
    return cudaErrorNotSupported;
  }
};

// Variants whose thread count follows S (16 elements per thread, S = 512 .. 2048): with
// 256 threads those small runs hold 8 or fewer elements per thread and the kernel
// spills about 900 bytes per thread; with S / 16 threads it does not.
template <int C, int MAXR>
struct Kb3LaunchAutoT {
  static cudaError_t launch(int M, const BStream* s, const BItem* it, int n, int* ctr, cudaStream_t stream,
                            int* nclusters) {
    switch (M / C) {
      case 512: return Kb3Launch<C, 32, MAXR>::template go<512>(s, it, n, ctr, stream, nclusters);
      case 1024: return Kb3Launch<C, 64, MAXR>::template go<1024>(s, it, n, ctr, stream, nclusters);
      case 2048: return Kb3Launch<C, 128, MAXR>::template go<2048>(s, it, n, ctr, stream, nclusters);
    }
    return cudaErrorNotSupported;
  }
};

// FFT_M(b) for the distinct J whose Bluestein length is exactly M = C * S (the odd
// cluster lengths; the other J are left to kb_bhat)
template <int C, int S, int T, int MAXR>
__global__ void __launch_bounds__(T, 1)
kb_bhat_s(const int* __restrict__ Js, const int* __restrict__ Ms, const float2* const* __restrict__ chirps,
          float2* const* __restrict__ bhats, int nJ) {
  extern __shared__ float2 smem[];
  int r = 0;
  if constexpr (C > 1) r = (int)cg::this_cluster().block_rank();
  const int t = blockIdx.x / C;
  if (t >= nJ || Ms[t] != C * S) return;  // uniform over the cluster
  bhat_item<C, S, T, MAXR>(chirps[t], Js[t], bhats[t], smem, r);
}

template <int C, int T, int MAXR>
__global__ void __launch_bounds__(T, 1)
kb_bhat(const int* __restrict__ Js, const int* __restrict__ Ms, const float2* const* __restrict__ chirps,
        float2* const* __restrict__ bhats, int nJ) {
  extern __shared__ float2 smem[];
  int r = 0;
  if constexpr (C > 1) r = (int)cg::this_cluster().block_rank();
  const int t = blockIdx.x / C;
  if (t >= nJ) return;  // uniform over the cluster
  const int J = Js[t];
  switch (Ms[t] / C) {
    case 512: bhat_item<C, 512, T, MAXR>(chirps[t], J, bhats[t], smem, r); break;
    case 1024: bhat_item<C, 1024, T, MAXR>(chirps[t], J, bhats[t], smem, r); break;
    case 2048: bhat_item<C, 2048, T, MAXR>(chirps[t], J, bhats[t], smem, r); break;
    case 4096: bhat_item<C, 4096, T, MAXR>(chirps[t], J, bhats[t], smem, r); break;
    case 8192: bhat_item<C, 8192, T, MAXR>(chirps[t], J, bhats[t], smem, r); break;
    default: break;
  }
}

#ifdef IPFB_BATCHED_HOST_KERNELS
// kb4: column pairs [P][J] -> time order, tiles of 64 frames x 32 pairs
__global__ void __launch_bounds__(256)
kb4_to_time(const BStream* __restrict__ streams, const BItem* __restrict__ items, int nitems, int* counter) {
  __shared__ float2 tile[64][33];
  __shared__ int slot;
  for (int guard = 0; guard < nitems + 1; ++guard) {
    const int it = fetch_item_cta(counter, &slot);
    if (it >= nitems) break;
    const BItem item = items[it];
    const BStream& st = streams[item.s];
    const int H = st.N / 2, J = st.J;
    const int ntp = (H + 31) / 32;
    const int p0 = (item.a % ntp) * 32, j0 = (item.a / ntp) * 64;
    for (int idx = threadIdx.x; idx < 32 * 64; idx += 256) {
      const int pp = idx / 64, jj = idx % 64;
      if (p0 + pp < H && j0 + jj < J) tile[jj][pp] = st.d2[(size_t)(p0 + pp) * J + j0 + jj];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 32 * 64; idx += 256) {
      const int jj = idx / 32, pp = idx % 32;
      if (p0 + pp < H && j0 + jj < J)
        reinterpret_cast<float2*>(st.x_out + (size_t)(j0 + jj) * st.N)[p0 + pp] = tile[jj][pp];
    }
    __syncthreads();
  }
}

#endif  // IPFB_BATCHED_HOST_KERNELS

}  // namespace ipfb
