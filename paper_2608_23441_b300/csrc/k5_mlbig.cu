// Maximum-likelihood inverse PFB with a time-domain prior (Sec. 4.2, Eq. chi squared) for
// columns longer than one CTA holds on chip.
//
// Per column n the conjugate gradient solves
//     (C_n^T C_n / sigma^2 + lam M_n) x_n = C_n^T d_n / sigma^2 + lam M_n p_n,
// as the single-CTA solve does, but the vectors b, x, r, p, q, z live in HBM in the
// column transform's residue layout (frame j = C m + r of pair p at v[(p C + r) S + m]),
// so that the Wiener preconditioner
//     z = F^dagger[ F r / (|W_n|^2 / sigma^2 + lam mbar_n) ]
// is the cluster transform K3 with its ML gain.  One CG iteration is
//     mlb_ap   x += alpha_prev p, p' = z + beta p, q = A p'    tiles with a stencil halo
//     k3       r -= alpha q (alpha from the tiles' p'.q), r.r,  listed pairs only;
//              z = M_W r, r.z                                    r.z by Parseval
//     mlb_ctl  stopping test, beta, alpha, the next list of active pairs
// (without a preconditioner mlb_xr forms alpha, r -= alpha q and r.r, and z = r).
// The step x += alpha p of an iteration is applied by the next iteration's mlb_ap,
// which reads that p anyway; a pair's last step is applied when the solution is
// written out.
// A pair leaves the list once both its columns have converged, so the work follows the
// columns still iterating.  p' goes to the other of two buffers: neighbouring tiles read
// the old p in their halos.  Each tile writes its partial sums to a slot of its own and a
// pair's slots are added in one fixed order (FP64), so every CTA of a pair derives the
// same alpha.  The tile kernels run persistent grids over (listed pair, tile) items.
#include "common.cuh"
#include "launch.h"

#include <mutex>

namespace ipfb {
namespace {
constexpr int kT = 256;                   // threads per CTA
constexpr int kTF = 2048;                 // frames per tile, at most
constexpr int kEPT = kTF / kT;            // items per thread, at most
constexpr int kSv = kTF + 2 * (15 + 7);   // tile + halo: RMAX <= 15, C <= 8 (float2)
constexpr int kW = kT / 32;

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }
int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// sum of K per-thread FP32 values over the CTA (FP32 within a warp, FP64 across warps);
// every thread receives the sums
template <int K>
__device__ __forceinline__ void cta_sum(float (&v)[K], double* red, double (&out)[K]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0) red[warp * K + k] = (double)v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kW; ++w) s += red[w * K + k];
    out[k] = s;
  }
  __syncthreads();
}

// FP64 sum over a warp in a fixed butterfly order (every lane receives it)
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// a pair's tile slots k0, k0 + 1 summed over its NT <= 32 tiles (one warp, fixed order)
__device__ __forceinline__ void pair_sums(const double* part, int p, int NT, int k0, double& s0, double& s1) {
  const int lane = threadIdx.x & 31;
  double a = 0.0, b = 0.0;
  if (lane < NT) {
    const double* q = part + ((size_t)p * NT + lane) * 8 + k0;
    a = __ldcg(q);
    b = __ldcg(q + 1);
  }
  s0 = warp_sum(a);
  s1 = warp_sum(b);
}

__device__ __forceinline__ size_t vidx(const MlbGeom& g, int p, int r, int m) {
  return ((size_t)p * g.C + r) * g.S + m;
}
// item i of tile t: residue i / TM, position t TM + i % TM, as an offset within the pair
__device__ __forceinline__ unsigned loc(const MlbGeom& g, int t, int i) {
  return (unsigned)((i >> g.logTM) * g.S + t * g.TM + (i & (g.TM - 1)));
}

// tile t of pair p with a halo of h positions: sv[r TMP + mm] = f(index of residue r,
// position t TM - h + mm (mod S)), mm < TMP = TM + 2h.  Every thread issues all its
// loads before the first shared-memory store, so each SM keeps enough bytes in flight
// to cover the HBM latency.
constexpr int kHv = (kSv + kT - 1) / kT;
template <class F>
__device__ __forceinline__ void load_halo(float2* sv, const MlbGeom& g, int p, int t, int h, F f) {
  const int TMP = g.TM + 2 * h, n = g.C * TMP, m0 = t * g.TM - h;
  const size_t base = vidx(g, p, 0, 0);
  float2 v[kHv];
#pragma unroll
  for (int k = 0; k < kHv; ++k) {
    const int i = threadIdx.x + k * kT;
    if (i < n) {
      const int r = i / TMP, mm = i - r * TMP;
      v[k] = f(base + (unsigned)(r * g.S + ((m0 + mm) & (g.S - 1))));
    }
  }
#pragma unroll
  for (int k = 0; k < kHv; ++k) {
    const int i = threadIdx.x + k * kT;
    if (i < n) sv[i] = v[k];
  }
}

// shared-memory offset of frame (r + s) relative to position m of residue r: residue
// (r + s) mod C, position m + floor((r + s) / C); the bias 32 (a multiple of C) keeps
// the shift a floor for negative r + s
__device__ __forceinline__ int nb_off(int r, int s, int m, int TMP, int h, int logC) {
  const int u = r + s + 32;
  return (u & ((1 << logC) - 1)) * TMP + h + m + (u >> logC) - (32 >> logC);
}

// sum_s a_s v[j + s] at residue r, position m of the tile (a includes 1/sigma^2)
template <int RMAX>
__device__ __forceinline__ float2 stencil(const float2* sv, int TMP, int h, int logC, int r, int m,
                                          const float2 (&a)[RMAX + 1]) {
  const float2 c = sv[r * TMP + h + m];
  float2 acc = make_float2(a[0].x * c.x, a[0].y * c.y);
#pragma unroll
  for (int s = 1; s <= RMAX; ++s) {
    const float2 lo = sv[nb_off(r, -s, m, TMP, h, logC)], hi = sv[nb_off(r, s, m, TMP, h, logC)];
    acc.x = fmaf(a[s].x, lo.x + hi.x, acc.x);
    acc.y = fmaf(a[s].y, lo.y + hi.y, acc.y);
  }
  return acc;
}

template <int RMAX>
__device__ __forceinline__ void load_coef(const MlbBufs& b, int p, float2 (&a)[RMAX + 1]) {
#pragma unroll
  for (int s = 0; s <= RMAX; ++s) a[s] = __ldg(b.acoef + (size_t)p * 16 + s);
}

// ---- setup ------------------------------------------------------------------------
// Tile: 32 pairs x 8C frames (8 positions of every residue).  Reads are rows of the
// time-order arrays; writes are runs of 8 positions of one residue.
__global__ void __launch_bounds__(kT)
k_mlb_transpose(const uint8_t* __restrict__ mask, const float* __restrict__ prior, const float* __restrict__ x0,
                float lam, MlbGeom g, MlbBufs b) {
  __shared__ float2 tp[64][33], tx[64][33];
  __shared__ uint16_t tm[64][33];
  const int P = g.N / 2, FJ = 8 * g.C;
  const int p0 = blockIdx.x * 32, j0 = blockIdx.y * FJ;
  for (int i = threadIdx.x; i < FJ * 32; i += kT) {
    const int jj = i >> 5, pp = i & 31, p = p0 + pp;
    if (p < P) {
      const size_t t = (size_t)(j0 + jj) * g.N + 2 * p;
      tm[jj][pp] = *reinterpret_cast<const uint16_t*>(mask + t);
      tp[jj][pp] = *reinterpret_cast<const float2*>(prior + t);
      tx[jj][pp] = x0 ? *reinterpret_cast<const float2*>(x0 + t) : make_float2(0.0f, 0.0f);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < FJ * 32; i += kT) {
    const int pp = i / FJ, rem = i - pp * FJ, r = rem >> 3, mi = rem & 7, p = p0 + pp;
    if (p >= P) continue;
    const int jj = g.C * mi + r;
    const size_t v = vidx(g, p, r, (j0 >> g.logC) + mi);
    const uint16_t mm = tm[jj][pp];
    const uint8_t bits = (uint8_t)(((mm & 0xFFu) ? 1 : 0) | ((mm >> 8) ? 2 : 0));
    const float2 pr = tp[jj][pp];
    b.mk[v] = bits;
    b.B[v] = make_float2((bits & 1) ? lam * pr.x : 0.0f, (bits & 2) ? lam * pr.y : 0.0f);
    b.X[v] = tx[jj][pp];
  }
}

// b = C^T d / sigma^2 + lam m prior with (C^T d)[j] = sum_q w_q d[j - q]; r0 = b - A x0.
// Slots: [0,1] mask counts, [4,5] r.r, [6,7] b.b.  Tile 0 of each pair stores the taps.
template <int RMAX>
__global__ void __launch_bounds__(kT, 2)
k_mlb_rhs(const float* __restrict__ window, MLParams mp, MlbGeom g, MlbBufs b) {
  __shared__ float2 sv[kSv];
  __shared__ double red[kW * 6];
  constexpr int NM = RMAX + 1;
  const int h = (RMAX + g.C - 1) >> g.logC, TMP = g.TM + 2 * h;
  const int P = g.N / 2, items = g.C << g.logTM;
  const bool zcopy = mp.precond == 1;
  for (int w = blockIdx.x; w < P * g.NT; w += gridDim.x) {
    const int p = w / g.NT, t = w - p * g.NT;
    float ta[NM], tb[NM];
#pragma unroll
    for (int q = 0; q < NM; ++q) {
      ta[q] = q < mp.ntap ? __ldg(window + (size_t)q * g.N + 2 * p) : 0.0f;
      tb[q] = q < mp.ntap ? __ldg(window + (size_t)q * g.N + 2 * p + 1) : 0.0f;
    }
    float2 a[NM];
#pragma unroll
    for (int s = 0; s < NM; ++s) {
      float sa = 0.0f, sb = 0.0f;
#pragma unroll
      for (int q = 0; q + s < NM; ++q) {
        sa = fmaf(ta[q], ta[q + s], sa);
        sb = fmaf(tb[q], tb[q + s], sb);
      }
      a[s] = make_float2(sa * mp.inv_s2, sb * mp.inv_s2);
    }
    if (t == 0 && threadIdx.x == 0) {
#pragma unroll
      for (int s = 0; s < 16; ++s) b.acoef[(size_t)p * 16 + s] = s < NM ? a[s < NM ? s : 0] : make_float2(0.0f, 0.0f);
    }
    float2 bt[kEPT];
    uint8_t mb[kEPT];
#pragma unroll
    for (int e = 0; e < kEPT; ++e) {
      const int i = threadIdx.x + e * kT;
      if (i < items) {
        const size_t v = vidx(g, p, 0, 0) + loc(g, t, i);
        bt[e] = b.B[v];  // lam m prior
        mb[e] = b.mk[v];
      }
    }
    load_halo(sv, g, p, t, h, [&](size_t i) { return b.Q[i]; });
    __syncthreads();
    float acc6[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};  // counts, r.r, b.b
#pragma unroll
    for (int e = 0; e < kEPT; ++e) {
      const int i = threadIdx.x + e * kT;
      if (i < items) {
        const int r = i >> g.logTM, m = i & (g.TM - 1);
        const size_t v = vidx(g, p, 0, 0) + loc(g, t, i);
        float2 c = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int q = 0; q < NM; ++q) {
          const float2 dv = sv[nb_off(r, -q, m, TMP, h, g.logC)];
          c.x = fmaf(ta[q], dv.x, c.x);
          c.y = fmaf(tb[q], dv.y, c.y);
        }
        const uint8_t bits = mb[e];
        bt[e] = make_float2(fmaf(c.x, mp.inv_s2, bt[e].x), fmaf(c.y, mp.inv_s2, bt[e].y));
        b.B[v] = bt[e];
        acc6[0] += (bits & 1) ? 1.0f : 0.0f;
        acc6[1] += (bits & 2) ? 1.0f : 0.0f;
        acc6[4] = fmaf(bt[e].x, bt[e].x, acc6[4]);
        acc6[5] = fmaf(bt[e].y, bt[e].y, acc6[5]);
      }
    }
    if (mp.use_x0) {
      __syncthreads();
      load_halo(sv, g, p, t, h, [&](size_t i) { return b.X[i]; });
      __syncthreads();
#pragma unroll
      for (int e = 0; e < kEPT; ++e) {
        const int i = threadIdx.x + e * kT;
        if (i < items) {
          const int r = i >> g.logTM, m = i & (g.TM - 1);
          const size_t v = vidx(g, p, 0, 0) + loc(g, t, i);
          const float2 xv = sv[r * TMP + h + m];
          const float2 ax = stencil<RMAX>(sv, TMP, h, g.logC, r, m, a);
          const uint8_t bits = mb[e];
          bt[e].x -= fmaf((bits & 1) ? mp.lam : 0.0f, xv.x, ax.x);
          bt[e].y -= fmaf((bits & 2) ? mp.lam : 0.0f, xv.y, ax.y);
        }
      }
    }
    float rr0 = 0.0f, rr1 = 0.0f;
#pragma unroll
    for (int e = 0; e < kEPT; ++e) {
      const int i = threadIdx.x + e * kT;
      if (i < items) {
        const size_t v = vidx(g, p, 0, 0) + loc(g, t, i);
        b.R[v] = bt[e];
        if (zcopy) b.Z[v] = bt[e];
        rr0 = fmaf(bt[e].x, bt[e].x, rr0);
        rr1 = fmaf(bt[e].y, bt[e].y, rr1);
      }
    }
    acc6[2] = acc6[4];
    acc6[3] = acc6[5];
    acc6[4] = rr0;
    acc6[5] = rr1;
    double s6[6];
    cta_sum<6>(acc6, red, s6);
    if (threadIdx.x == 0) {
      // slots: counts (0, 1), unused (2, 3), r.r (4, 5), b.b (6, 7)
      double* o = b.part + ((size_t)p * g.NT + t) * 8;
      o[0] = s6[0];
      o[1] = s6[1];
      o[2] = 0.0;
      o[3] = 0.0;
      o[4] = s6[4];
      o[5] = s6[5];
      o[6] = s6[2];
      o[7] = s6[3];
    }
  }
}

// one warp per pair: |b|, lam mbar; every pair listed; counters cleared
__global__ void __launch_bounds__(kT) k_mlb_init(MLParams mp, MlbGeom g, MlbBufs b) {
  const int P = g.N / 2, lane = threadIdx.x & 31;
  const int p = (blockIdx.x * kT + threadIdx.x) >> 5;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    b.ctl[0] = P;
    b.ctl[1] = 0;
    b.ctl[2] = 0;
  }
  if (p >= P) return;
  double c0, c1, q0, q1;
  pair_sums(b.part, p, g.NT, 0, c0, c1);
  pair_sums(b.part, p, g.NT, 6, q0, q1);
  if (lane == 0) {
    const double J = (double)g.C * (double)g.S;
    MlbPair s = {};
    s.bn[0] = q0 > 0.0 ? sqrtf((float)q0) : 1.0f;
    s.bn[1] = q1 > 0.0 ? sqrtf((float)q1) : 1.0f;
    s.act = 3;
    b.ps[p] = s;
    b.lam_m[2 * p] = mp.lam * (float)(c0 / J);
    b.lam_m[2 * p + 1] = mp.lam * (float)(c1 / J);
    b.list[p] = p;
  }
}

// ---- iteration ----------------------------------------------------------------------
// x += apend p (the previous iteration's step), p' = z + beta p (beta = 0: p' = z, the old
// p unread), q = A p'; slots [0,1] p'.q
template <int RMAX>
__global__ void __launch_bounds__(kT, RMAX <= 3 ? 4 : 2)
k_mlb_ap(const float2* __restrict__ Po, float2* __restrict__ Pn, MLParams mp, MlbGeom g, MlbBufs b) {
  __shared__ float2 sv[kSv];
  __shared__ double red[kW * 2];
  const int cnt = b.ctl[0];
  const int h = (RMAX + g.C - 1) >> g.logC, TMP = g.TM + 2 * h;
  const int items = g.C << g.logTM;
  for (int w = blockIdx.x; w < cnt * g.NT; w += gridDim.x) {
    const int li = w / g.NT, t = w - li * g.NT;
    const int p = __ldg(b.list + li);
    const float ba = b.ps[p].beta[0], bb = b.ps[p].beta[1];
    const float xa = b.ps[p].apend[0], xb = b.ps[p].apend[1];
    const bool rd = ba != 0.0f || bb != 0.0f, xs = xa != 0.0f || xb != 0.0f;
    float2 a[RMAX + 1];
    load_coef<RMAX>(b, p, a);
    uint8_t mb[kEPT];
#pragma unroll
    for (int e = 0; e < kEPT; ++e) {
      const int i = threadIdx.x + e * kT;
      if (i < items) mb[e] = b.mk[vidx(g, p, 0, 0) + loc(g, t, i)];
    }
    load_halo(sv, g, p, t, h, [&](size_t i) {
      const float2 z = b.Z[i];
      if (!rd) return z;
      const float2 po = Po[i];
      return make_float2(ba != 0.0f ? fmaf(ba, po.x, z.x) : z.x, bb != 0.0f ? fmaf(bb, po.y, z.y) : z.y);
    });
    __syncthreads();
    float acc[2] = {0.0f, 0.0f};
#pragma unroll
    for (int e = 0; e < kEPT; ++e) {
      const int i = threadIdx.x + e * kT;
      if (i < items) {
        const int r = i >> g.logTM, m = i & (g.TM - 1);
        const size_t v = vidx(g, p, 0, 0) + loc(g, t, i);
        const float2 pv = sv[r * TMP + h + m];
        const float2 ap = stencil<RMAX>(sv, TMP, h, g.logC, r, m, a);
        const uint8_t bits = mb[e];
        const float2 q = make_float2(fmaf((bits & 1) ? mp.lam : 0.0f, pv.x, ap.x),
                                     fmaf((bits & 2) ? mp.lam : 0.0f, pv.y, ap.y));
        Pn[v] = pv;
        b.Q[v] = q;
        if (xs) {
          // the previous iteration's step (its p is the old direction, just read through L2)
          const float2 po = Po[v];
          float2 x = b.X[v];
          x.x = fmaf(xa, po.x, x.x);
          x.y = fmaf(xb, po.y, x.y);
          b.X[v] = x;
        }
        acc[0] = fmaf(pv.x, q.x, acc[0]);
        acc[1] = fmaf(pv.y, q.y, acc[1]);
      }
    }
    double s[2];
    cta_sum<2>(acc, red, s);
    if (threadIdx.x == 0) {
      double* o = b.part + ((size_t)p * g.NT + t) * 8;
      o[0] = s[0];
      o[1] = s[1];
    }
  }
}

// float4 view of a pair's J frames (two pair-frames per access) and the offset of the
// e-th float4 this thread touches in tile t (-1 past the tile)
__device__ __forceinline__ float4* pair4(float2* v, const MlbGeom& g, int p) {
  return reinterpret_cast<float4*>(v + (size_t)p * g.C * g.S);
}
__device__ __forceinline__ int off4(const MlbGeom& g, int t, int e) {
  const int f = threadIdx.x + e * kT, half = g.TM >> 1;
  if (f >= (g.C << g.logTM) >> 1) return -1;
  const int r = f >> (g.logTM - 1);
  return r * (g.S >> 1) + t * half + (f & (half - 1));
}
constexpr int kE4 = kEPT / 2;  // float4 per thread per tile, at most

// without a preconditioner: alpha = r.r / p'.q per active column, r -= alpha q;
// slots [4,5] r.r (z is r itself)
__global__ void __launch_bounds__(kT, 4)
k_mlb_xr(MLParams mp, MlbGeom g, MlbBufs b) {
  __shared__ double red[kW * 2];
  __shared__ float al[2];
  const int cnt = b.ctl[0];
  for (int w = blockIdx.x; w < cnt * g.NT; w += gridDim.x) {
    const int li = w / g.NT, t = w - li * g.NT;
    const int p = __ldg(b.list + li);
    const float4* __restrict__ Q4 = pair4(b.Q, g, p);
    float4* __restrict__ R4 = pair4(b.R, g, p);
    int o[kE4];
    float4 q[kE4], rv[kE4];
#pragma unroll
    for (int e = 0; e < kE4; ++e) {
      o[e] = off4(g, t, e);
      if (o[e] >= 0) {
        q[e] = Q4[o[e]];
        rv[e] = R4[o[e]];
      }
    }
    if (threadIdx.x < 32) {
      double pq0, pq1;
      pair_sums(b.part, p, g.NT, 0, pq0, pq1);
      if (threadIdx.x == 0) {
        const MlbPair& s = b.ps[p];
        // ratios in FP32 (one rounding); the sums themselves are FP64
        al[0] = ((s.act & 1) && pq0 != 0.0) ? (float)s.rz[0] / (float)pq0 : 0.0f;
        al[1] = ((s.act & 2) && pq1 != 0.0) ? (float)s.rz[1] / (float)pq1 : 0.0f;
      }
    }
    __syncthreads();
    const float aa = al[0], ab = al[1];
    float acc[2] = {0.0f, 0.0f};
#pragma unroll
    for (int e = 0; e < kE4; ++e) {
      if (o[e] >= 0) {
        float4 r = rv[e];
        r.x = fmaf(-aa, q[e].x, r.x);
        r.y = fmaf(-ab, q[e].y, r.y);
        r.z = fmaf(-aa, q[e].z, r.z);
        r.w = fmaf(-ab, q[e].w, r.w);
        R4[o[e]] = r;
        acc[0] = fmaf(r.x, r.x, fmaf(r.z, r.z, acc[0]));
        acc[1] = fmaf(r.y, r.y, fmaf(r.w, r.w, acc[1]));
      }
    }
    double s[2];
    cta_sum<2>(acc, red, s);
    if (threadIdx.x == 0) {
      double* out = b.part + ((size_t)p * g.NT + t) * 8 + 4;
      out[0] = s[0];
      out[1] = s[1];
    }
  }
}

// One warp per listed pair: relative residuals, the stopping test, beta, iteration
// counts.  The last CTA to finish (a ticket) lists the pairs still active in ascending
// order, advances the iteration count and sets the loop condition.  When the iteration
// just run had no pair listed, nothing changes and the list stays empty.
__global__ void __launch_bounds__(kT)
k_mlb_ctl(int first, int set_cond, cudaGraphConditionalHandle h, MLParams mp, MlbGeom g, MlbBufs b) {
  __shared__ int s_last;
  __shared__ int s_scan[kT];
  const int P = g.N / 2, lane = threadIdx.x & 31;
  const int cnt0 = b.ctl[0];
  const int p = (blockIdx.x * kT + threadIdx.x) >> 5;
  if (cnt0 > 0 && p < P) {
    const int act0 = first ? 3 : b.ps[p].act;
    if (act0) {
      double rz0, rz1, rr0, rr1, pq0 = 0.0, pq1 = 0.0;
      if (mp.precond == 1 && !first) {
        // the fused update's per-CTA r.r, in CTA order
        const double* q = b.rrk + (size_t)p * g.C * 2;
        rr0 = warp_sum(lane < g.C ? __ldcg(q + 2 * lane) : 0.0);
        rr1 = warp_sum(lane < g.C ? __ldcg(q + 2 * lane + 1) : 0.0);
      } else {
        pair_sums(b.part, p, g.NT, 4, rr0, rr1);
      }
      if (mp.precond == 1) {
        // the preconditioner's per-CTA r.z, in CTA order
        const double* q = b.rzk + (size_t)p * g.C * 2;
        rz0 = warp_sum(lane < g.C ? __ldcg(q + 2 * lane) : 0.0);
        rz1 = warp_sum(lane < g.C ? __ldcg(q + 2 * lane + 1) : 0.0);
      } else {
        rz0 = rr0;
        rz1 = rr1;
      }
      if (!first) pair_sums(b.part, p, g.NT, 0, pq0, pq1);
      if (lane == 0) {
        MlbPair s = b.ps[p];
        const double rz[2] = {rz0, rz1}, rr[2] = {rr0, rr1}, pq[2] = {pq0, pq1};
        // the step this iteration took (the same alpha as the update kernels formed)
        // is applied to x by the next stencil pass, or when the solution is written
        if (!first) {
#pragma unroll
          for (int c = 0; c < 2; ++c)
            s.apend[c] = ((act0 & (1 << c)) && pq[c] != 0.0) ? (float)s.rz[c] / (float)pq[c] : 0.0f;
          s.pbuf = (b.ctl[1] + 1) & 1;
        }
        int nac = 0;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          if (!(act0 & (1 << c))) continue;
          if (!first) s.it[c] += 1;
          s.rel[c] = sqrtf((float)rr[c]) / s.bn[c];
          if (s.rel[c] > mp.tol) nac |= 1 << c;
          s.beta[c] = (!first && (nac & (1 << c)) && s.rz[c] != 0.0) ? (float)rz[c] / (float)s.rz[c] : 0.0f;
          if (first || (nac & (1 << c))) s.rz[c] = rz[c];
        }
        s.act = nac;
        b.ps[p] = s;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(b.ctl + 2, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  int total = 0;
  if (cnt0 > 0) {
    // contiguous chunks per thread, an exclusive scan of their counts, then the list
    // (P <= 8192 = 32 kT: a thread's flags fit one 32-bit mask, loaded all at once)
    const int per = (P + kT - 1) / kT, lo = threadIdx.x * per;
    unsigned bits = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const int q = lo + k;
      if (k < per && q < P && __ldcg(&b.ps[q].act) != 0) bits |= 1u << k;
    }
    const int n = __popc(bits);
    s_scan[threadIdx.x] = n;
    __syncthreads();
    for (int o = 1; o < kT; o <<= 1) {
      const int v = threadIdx.x >= o ? s_scan[threadIdx.x - o] : 0;
      __syncthreads();
      s_scan[threadIdx.x] += v;
      __syncthreads();
    }
    total = s_scan[kT - 1];
    int pos = s_scan[threadIdx.x] - n;
    for (; bits; bits &= bits - 1) b.list[pos++] = lo + __ffs(bits) - 1;
  }
  if (threadIdx.x == 0) {
    const int it = b.ctl[1] + ((first || cnt0 == 0) ? 0 : 1);
    const int count = (cnt0 == 0 || it >= mp.max_iter) ? 0 : total;
    b.ctl[0] = count;
    b.ctl[1] = it;
    b.ctl[2] = 0;
    if (set_cond) cudaGraphSetConditional(h, count > 0 ? 1u : 0u);
  }
}

// x = X + apend p (each pair's last step, p in Pv[pbuf]) written to Q; its true
// residual b - A x per tile: slots [6,7]
template <int RMAX>
__global__ void __launch_bounds__(kT, RMAX <= 3 ? 4 : 2) k_mlb_true_resid(MLParams mp, MlbGeom g, MlbBufs b) {
  __shared__ float2 sv[kSv];
  __shared__ double red[kW * 2];
  const int h = (RMAX + g.C - 1) >> g.logC, TMP = g.TM + 2 * h;
  const int P = g.N / 2, items = g.C << g.logTM;
  for (int w = blockIdx.x; w < P * g.NT; w += gridDim.x) {
    const int p = w / g.NT, t = w - p * g.NT;
    float2 a[RMAX + 1];
    load_coef<RMAX>(b, p, a);
    float2 bq[kEPT];
    uint8_t mb[kEPT];
#pragma unroll
    for (int e = 0; e < kEPT; ++e) {
      const int i = threadIdx.x + e * kT;
      if (i < items) {
        const size_t v = vidx(g, p, 0, 0) + loc(g, t, i);
        bq[e] = b.B[v];
        mb[e] = b.mk[v];
      }
    }
    const float xa = b.ps[p].apend[0], xb = b.ps[p].apend[1];
    const float2* __restrict__ Pl = (b.ps[p].pbuf & 1) ? b.Pv[1] : b.Pv[0];
    load_halo(sv, g, p, t, h, [&](size_t i) {
      float2 x = b.X[i];
      if (xa != 0.0f || xb != 0.0f) {
        const float2 pv = Pl[i];
        x.x = fmaf(xa, pv.x, x.x);
        x.y = fmaf(xb, pv.y, x.y);
      }
      return x;
    });
    __syncthreads();
    float acc[2] = {0.0f, 0.0f};
#pragma unroll
    for (int e = 0; e < kEPT; ++e) {
      const int i = threadIdx.x + e * kT;
      if (i < items) {
        const int r = i >> g.logTM, m = i & (g.TM - 1);
        const float2 xv = sv[r * TMP + h + m];
        b.Q[vidx(g, p, 0, 0) + loc(g, t, i)] = xv;
        const float2 ax = stencil<RMAX>(sv, TMP, h, g.logC, r, m, a);
        const uint8_t bits = mb[e];
        const float2 bv = bq[e];
        const float qx = bv.x - fmaf((bits & 1) ? mp.lam : 0.0f, xv.x, ax.x);
        const float qy = bv.y - fmaf((bits & 2) ? mp.lam : 0.0f, xv.y, ax.y);
        acc[0] = fmaf(qx, qx, acc[0]);
        acc[1] = fmaf(qy, qy, acc[1]);
      }
    }
    double s[2];
    cta_sum<2>(acc, red, s);
    if (threadIdx.x == 0) {
      double* o = b.part + ((size_t)p * g.NT + t) * 8 + 6;
      o[0] = s[0];
      o[1] = s[1];
    }
  }
}

// one warp per pair: iterations, recursive and true relative residuals
__global__ void __launch_bounds__(kT) k_mlb_report(MlbGeom g, MlbBufs b, int* __restrict__ iters,
                                                   float* __restrict__ resid) {
  const int P = g.N / 2, lane = threadIdx.x & 31;
  const int p = (blockIdx.x * kT + threadIdx.x) >> 5;
  if (p >= P) return;
  double q0, q1;
  pair_sums(b.part, p, g.NT, 6, q0, q1);
  if (lane == 0) {
    const MlbPair s = b.ps[p];
    iters[2 * p] = s.it[0];
    iters[2 * p + 1] = s.it[1];
    resid[2 * p] = s.rel[0];
    resid[2 * p + 1] = s.rel[1];
    resid[g.N + 2 * p] = sqrtf((float)q0) / s.bn[0];
    resid[g.N + 2 * p + 1] = sqrtf((float)q1) / s.bn[1];
  }
}

// CTAs of a persistent grid: the SM count times the CTAs resident per SM
int persistent_grid(const void* fn) {
  static std::mutex mu;
  static int nsm = 0;
  std::lock_guard<std::mutex> lk(mu);
  if (nsm == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      nsm = 148;
  }
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kT, 0) != cudaSuccess || occ < 1) occ = 1;
  return nsm * occ;
}

int warp_grid(int P) { return (P * 32 + kT - 1) / kT; }
}  // namespace

MlbGeom mlb_geom(int N, int C, int S) {
  MlbGeom g;
  g.N = N;
  g.C = C;
  g.S = S;
  g.logC = ilog2(C);
  const int J = C * S;
  const int TF = J < kTF ? J : kTF;
  g.TM = TF / C;
  g.logTM = ilog2(g.TM);
  g.NT = J / TF;
  return g;
}

size_t mlb_workspace(int N, int C, int S) {
  const MlbGeom g = mlb_geom(N, C, S);
  const size_t P = (size_t)N / 2, J = (size_t)C * S;
  return 7 * al256(P * J * sizeof(float2)) + al256(P * J) + al256(P * 16 * sizeof(float2)) +
         al256(P * g.NT * 8 * sizeof(double)) + 2 * al256(P * 16 * sizeof(double)) + al256(P * sizeof(MlbPair)) +
         al256((size_t)N * sizeof(float)) + al256(P * sizeof(int)) + al256(16 * sizeof(int));
}

MlbBufs mlb_carve(void* ws, int N, int C, int S) {
  const MlbGeom g = mlb_geom(N, C, S);
  const size_t P = (size_t)N / 2, J = (size_t)C * S, vec = al256(P * J * sizeof(float2));
  uint8_t* w = static_cast<uint8_t*>(ws);
  MlbBufs b;
  float2** vecs[7] = {&b.B, &b.X, &b.R, &b.Q, &b.Z, &b.Pv[0], &b.Pv[1]};
  for (int i = 0; i < 7; ++i) {
    *vecs[i] = reinterpret_cast<float2*>(w);
    w += vec;
  }
  b.mk = w;
  w += al256(P * J);
  b.acoef = reinterpret_cast<float2*>(w);
  w += al256(P * 16 * sizeof(float2));
  b.part = reinterpret_cast<double*>(w);
  w += al256(P * g.NT * 8 * sizeof(double));
  b.rzk = reinterpret_cast<double*>(w);
  w += al256(P * 16 * sizeof(double));
  b.rrk = reinterpret_cast<double*>(w);
  w += al256(P * 16 * sizeof(double));
  b.ps = reinterpret_cast<MlbPair*>(w);
  w += al256(P * sizeof(MlbPair));
  b.lam_m = reinterpret_cast<float*>(w);
  w += al256((size_t)N * sizeof(float));
  b.list = reinterpret_cast<int*>(w);
  w += al256(P * sizeof(int));
  b.ctl = reinterpret_cast<int*>(w);
  return b;
}

cudaError_t launch_mlb_transpose(const uint8_t* mask, const float* prior, const float* x0, float lam,
                                 const MlbGeom& g, const MlbBufs& b, cudaStream_t st) {
  dim3 grid((g.N / 2 + 31) / 32, (g.C * g.S) / (8 * g.C));
  k_mlb_transpose<<<grid, kT, 0, st>>>(mask, prior, x0, lam, g, b);
  return cudaGetLastError();
}

cudaError_t launch_mlb_rhs(const float* window, const MLParams& mp, const MlbGeom& g, const MlbBufs& b,
                           cudaStream_t st) {
  if (mp.ntap == 4) {
    k_mlb_rhs<3><<<persistent_grid((const void*)k_mlb_rhs<3>), kT, 0, st>>>(window, mp, g, b);
  } else {
    k_mlb_rhs<15><<<persistent_grid((const void*)k_mlb_rhs<15>), kT, 0, st>>>(window, mp, g, b);
  }
  return cudaGetLastError();
}

cudaError_t launch_mlb_init(const MLParams& mp, const MlbGeom& g, const MlbBufs& b, cudaStream_t st) {
  k_mlb_init<<<warp_grid(g.N / 2), kT, 0, st>>>(mp, g, b);
  return cudaGetLastError();
}

cudaError_t launch_mlb_ap(int src, const MLParams& mp, const MlbGeom& g, const MlbBufs& b, cudaStream_t st) {
  if (mp.ntap == 4) {
    k_mlb_ap<3><<<persistent_grid((const void*)k_mlb_ap<3>), kT, 0, st>>>(b.Pv[src], b.Pv[src ^ 1], mp, g, b);
  } else {
    k_mlb_ap<15><<<persistent_grid((const void*)k_mlb_ap<15>), kT, 0, st>>>(b.Pv[src], b.Pv[src ^ 1], mp, g, b);
  }
  return cudaGetLastError();
}

cudaError_t launch_mlb_xr(const MLParams& mp, const MlbGeom& g, const MlbBufs& b, cudaStream_t st) {
  k_mlb_xr<<<persistent_grid((const void*)k_mlb_xr), kT, 0, st>>>(mp, g, b);
  return cudaGetLastError();
}

cudaError_t launch_mlb_ctl(int first, int set_cond, cudaGraphConditionalHandle h, const MLParams& mp,
                           const MlbGeom& g, const MlbBufs& b, cudaStream_t st) {
  k_mlb_ctl<<<warp_grid(g.N / 2), kT, 0, st>>>(first, set_cond, h, mp, g, b);
  return cudaGetLastError();
}

cudaError_t launch_mlb_finish(const MLParams& mp, const MlbGeom& g, const MlbBufs& b, int* iters, float* resid,
                              cudaStream_t st) {
  if (mp.ntap == 4) {
    k_mlb_true_resid<3><<<persistent_grid((const void*)k_mlb_true_resid<3>), kT, 0, st>>>(mp, g, b);
  } else {
    k_mlb_true_resid<15><<<persistent_grid((const void*)k_mlb_true_resid<15>), kT, 0, st>>>(mp, g, b);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_mlb_report<<<warp_grid(g.N / 2), kT, 0, st>>>(g, b, iters, resid);
  return cudaGetLastError();
}
}  // namespace ipfb
