// Maximum-likelihood inverse PFB with a time-domain prior (Sec. 4.2, Eq. chi squared)
// by conjugate gradient, one CTA per column pair.
//
// Per column n the normal equations of Eq. chi squared in the circulant model are
//     (C_n^T C_n / sigma^2 + lam M_n) x_n = C_n^T d_n / sigma^2 + lam M_n p_n,
// (C x)[j] = sum_r w[r,n] x[(j + r) mod J].  C^T C is the circular stencil with taps
// a_s = sum_r w_r w_{r+s} (|s| < ntap), applied exactly in FP32 from registers.
// Both columns of a pair run their own CG (own alpha, beta, stopping test) in
// lockstep; vectors are FP32, every inner product is reduced across the CTA in
// FP64.  Optional Wiener preconditioner
//     z = F^dagger[ F r / (|W_n|^2/sigma^2 + lam mbar_n) ]
// through the same pair-packed J-point FFTs as the Wiener inverse.
#pragma once

#include "common.cuh"
#include "launch.h"

namespace ipfb {

constexpr int kMlMaxTaps = 16;

// Sum of K values over the CTA: FP32 within each warp (shuffles), then one warp
// adds the per-warp partials in FP64 and (optionally) derives the CG scalars; the
// results are broadcast through shared memory.  FP64 work is O(warps) per call,
// since FP64 throughput on this part is a small fraction of FP32.
//   part : [T/32][K] floats,  res : [K + 8] doubles (sums, then scalars)
template <int K, int T, class SCALARS>
__device__ __forceinline__ void block_sum_bcast(float (&v)[K], float* part, double* res, SCALARS scalars) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  constexpr int W = T / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) part[warp * K + k] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      acc[k] = lane < W ? (double)part[lane * K + k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) res[k] = acc[k];
      scalars(acc, res + K);
    }
  }
  __syncthreads();
}

// Per-column state of the flexible-CG solve (fcg_kernels.cuh); k5_ml_cg writes it too
// when it hands a Wiener-preconditioned solve over to the flexible-CG kernels.
struct FcgCol {
  double rz;    // r.z of the current search direction
  float bnorm;  // |b|
  float rel;    // |r| / |b| (recursive residual)
  float s;      // RMS of u = M_W r, the net input scale
  float lam_m;  // prior weight x mask mean of the column (Wiener preconditioner)
  int iters;
  int active;
  int slot;     // request slot of the current preconditioner application
  int pad;      // 1: the pair was finished in the on-chip CG kernel (hand-over)
};

struct NoScalars {
  template <class A>
  __device__ __forceinline__ void operator()(const A&, double*) const {}
};

// Wiener preconditioner on the pair held as r = (r_a, r_b) in smem (complex r_a + i r_b)
template <int J, int T, int NT>
__device__ __forceinline__ void wiener_precond_pair(float2* sm, const float* ta, const float* tb, int ntap,
                                                   float inv_s2, float lam_ma, float lam_mb) {
  constexpr int NMAX = NT > 0 ? NT : kMlMaxTaps;
  const int tid = threadIdx.x;
  block_fft<J, T, false, 8>(sm, tid, SPad{sm}, SPad{sm});
  __syncthreads();
  for (int k = tid; k <= J / 2; k += T) {
    const int km = (J - k) % J;
    const float2 e1 = twiddle<false>(k, J);
    float2 Wa = make_float2(0.0f, 0.0f), Wb = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int t = NMAX - 1; t >= 0; --t) {
      if (NT > 0 || t < ntap) {
        Wa = cmul(Wa, e1);
        Wa.x += ta[t];
        Wb = cmul(Wb, e1);
        Wb.x += tb[t];
      }
    }
    const float Pa = fmaf(Wa.x * Wa.x + Wa.y * Wa.y, inv_s2, lam_ma);
    const float Pb = fmaf(Wb.x * Wb.x + Wb.y * Wb.y, inv_s2, lam_mb);
    const float ga = Pa > 0.0f ? 1.0f / (Pa * (float)J) : 0.0f;
    const float gb = Pb > 0.0f ? 1.0f / (Pb * (float)J) : 0.0f;
    float2 zk = sm[pidx(k)], zm = sm[pidx(km)];
    // split, scale by the real gains, recombine (modes k and -k)
    const float2 A = cscale(cadd(zk, cconj(zm)), 0.5f);
    const float2 dd = csub(zk, cconj(zm));
    const float2 B = make_float2(0.5f * dd.y, -0.5f * dd.x);
    const float2 ya = cscale(A, ga), yb = cscale(B, gb);
    zk = cadd(ya, cmul_i(yb));
    zm = cadd(cconj(ya), cmul_i(cconj(yb)));
    sm[pidx(k)] = zk;
    if (km != k) sm[pidx(km)] = zm;
  }
  __syncthreads();
  block_fft<J, T, true, 8>(sm, tid, SPad{sm}, SPad{sm});
  __syncthreads();
}

// One CTA per column pair p (columns 2p, 2p+1).  Thread t owns frames
// [t*EPT, (t+1)*EPT) of both columns.  The search direction p and the solution x
// live in padded shared memory (the stencil reads its halo straight from there);
// the residual r and A p stay in registers.
//   d2: [P][J] pair-packed d;  x2: [P][J] pair-packed initial guess in, solution out
//   mask / prior: time order [J][N] (bytes / floats)
//   iters: [N]; resid: [2][N] (recursive relative residual, true relative residual)
template <int J, int T, int RMAX>
__device__ __forceinline__ void load_window(const float2* sm, int j0, float2 (&v)[J / T + 2 * RMAX]) {
  constexpr int EPT = J / T;
#pragma unroll
  for (int i = 0; i < EPT + 2 * RMAX; ++i) v[i] = sm[pidx((j0 + i - RMAX + J) & (J - 1))];
}

// A v on a window v[-RMAX .. EPT+RMAX): inv_s2 * sum_s a_s v[e+s] + lam m v
template <int EPT, int RMAX>
__device__ __forceinline__ float2 apply_A_at(const float2* v, const float2 (&a)[RMAX + 1], uint32_t mbits,
                                             float lam, int e) {
  const float2 c = v[e + RMAX];
  float2 acc = make_float2(a[0].x * c.x, a[0].y * c.y);
#pragma unroll
  for (int s = 1; s <= RMAX; ++s) {
    const float2 lo = v[e + RMAX - s], hi = v[e + RMAX + s];
    acc.x = fmaf(a[s].x, lo.x + hi.x, acc.x);
    acc.y = fmaf(a[s].y, lo.y + hi.y, acc.y);
  }
  const float ma = ((mbits >> e) & 1u) ? lam : 0.0f;
  const float mb = ((mbits >> (e + 16)) & 1u) ? lam : 0.0f;
  return make_float2(fmaf(ma, c.x, acc.x), fmaf(mb, c.y, acc.y));
}

// b = C^T d / sigma^2 + lam m prior for this thread's frames, (C^T d)[i] = sum_r w_r d[i - r]
template <int J, int T, int RMAX>
__device__ __forceinline__ void build_rhs(const float2* __restrict__ d2p, const uint8_t* __restrict__ mask,
                                          const float* __restrict__ prior, int N, int p, int j0, const float* ta,
                                          const float* tb, float inv_s2, float lam, uint32_t& mbits,
                                          float2 (&b)[J / T]) {
  constexpr int EPT = J / T;
  float2 d[EPT + RMAX];
#pragma unroll
  for (int i = 0; i < EPT + RMAX; ++i) d[i] = d2p[(j0 + i - RMAX + J) & (J - 1)];
  mbits = 0;
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const size_t t_idx = (size_t)(j0 + e) * N + 2 * p;
    const uint16_t mm = *reinterpret_cast<const uint16_t*>(mask + t_idx);
    if (mm & 0xFFu) mbits |= 1u << e;
    if (mm >> 8) mbits |= 1u << (e + 16);
    float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int r = 0; r <= RMAX; ++r) {
      acc.x = fmaf(ta[r], d[e + RMAX - r].x, acc.x);
      acc.y = fmaf(tb[r], d[e + RMAX - r].y, acc.y);
    }
    const float2 pr = *reinterpret_cast<const float2*>(prior + t_idx);
    const float ma = ((mbits >> e) & 1u) ? lam : 0.0f;
    const float mb = ((mbits >> (e + 16)) & 1u) ? lam : 0.0f;
    b[e] = make_float2(fmaf(ma, pr.x, acc.x * inv_s2), fmaf(mb, pr.y, acc.y * inv_s2));
  }
}

template <int J, int T, int RMAX, int PRE, int NT>
__global__ void __launch_bounds__(T, 1)
k5_ml_cg(const float2* __restrict__ d2, float2* __restrict__ x2, const uint8_t* __restrict__ mask,
         const float* __restrict__ prior, const float* __restrict__ window, int N, MLParams mp,
         int* __restrict__ iters, float* __restrict__ resid, FcgBufs ex, int ex_max_iter) {
  constexpr int EPT = J / T;
  constexpr int WIN = EPT + 2 * RMAX;
  static_assert(EPT >= 1 && EPT <= 16, "1..16 frames per thread");
  extern __shared__ float2 smem[];
  float2* sm_x = smem;                                  // [padded J] solution
  float2* sm_p = sm_x + padded_len(J);                  // [padded J] search direction
  double* res = reinterpret_cast<double*>(sm_p + padded_len(J));  // [8] sums + [16] CG scalars
  float* part = reinterpret_cast<float*>(res + 24);                 // [T/32][4] warp partials
  float2* sm_f = reinterpret_cast<float2*>(part + (T / 32) * 4);    // [padded J] FFT work (PRE == 1)

  const int tid = threadIdx.x;
  // Longest job first: the worst-conditioned sub-filters sit around column N/2
  // (pair N/4, App. A), so blocks are mapped to pairs by distance from it.
  const int P = N / 2, pc = P / 2, bi = blockIdx.x;
  const int p = (pc + ((bi & 1) ? -((bi + 1) >> 1) : (bi >> 1)) + P) % P;
  const int j0 = tid * EPT;
  const float2* d2p = d2 + (size_t)p * J;

  constexpr int NMAX = NT > 0 ? NT : kMlMaxTaps;
  float ta[NMAX], tb[NMAX];
#pragma unroll
  for (int t = 0; t < NMAX; ++t) {
    ta[t] = (t < mp.ntap) ? __ldg(window + (size_t)t * N + 2 * p) : 0.0f;
    tb[t] = (t < mp.ntap) ? __ldg(window + (size_t)t * N + 2 * p + 1) : 0.0f;
  }
  float2 a[RMAX + 1];
#pragma unroll
  for (int s = 0; s <= RMAX; ++s) {
    float sa = 0.0f, sb = 0.0f;
#pragma unroll
    for (int r = 0; r + s < NMAX; ++r) {
      sa = fmaf(ta[r], ta[r + s], sa);
      sb = fmaf(tb[r], tb[r + s], sb);
    }
    a[s] = make_float2(sa * mp.inv_s2, sb * mp.inv_s2);
  }

  uint32_t mbits;
  float2 r[EPT];
  build_rhs<J, T, RMAX>(d2p, mask, prior, N, p, j0, ta, tb, mp.inv_s2, mp.lam, mbits, r);
  // CG state shared through smem (written by one thread of warp 0):
  //   st[0..1] alpha, st[2..3] beta, st[4] active flags, st[5..6] |b|, st[7..8] r.z old
  //   st[9..10] relative residual, st[11..12] iterations
  double* st = res + 8;
  {
    float bn[4];
    float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      s0 = fmaf(r[e].x, r[e].x, s0);
      s1 = fmaf(r[e].y, r[e].y, s1);
    }
    bn[0] = s0;
    bn[1] = s1;
    bn[2] = (float)__popc(mbits & 0xFFFFu);
    bn[3] = (float)__popc(mbits >> 16);
    block_sum_bcast<4, T>(bn, part, res, [](const double* a, double* o) {
      (void)o;
    });
  }
  if (tid == 0) {
    st[5] = res[0] > 0.0 ? (double)sqrtf((float)res[0]) : 1.0;
    st[6] = res[1] > 0.0 ? (double)sqrtf((float)res[1]) : 1.0;
    st[11] = 0.0;
    st[12] = 0.0;
  }
  const float lam_ma = mp.lam * (float)(res[2] / (double)J);
  const float lam_mb = mp.lam * (float)(res[3] / (double)J);

  // x0 (and r0 = b - A x0)
#pragma unroll
  for (int e = 0; e < EPT; ++e)
    sm_x[pidx(j0 + e)] = mp.use_x0 ? x2[(size_t)p * J + j0 + e] : make_float2(0.0f, 0.0f);
  if (mp.use_x0) {
    __syncthreads();
    float2 v[WIN];
    load_window<J, T, RMAX>(sm_x, j0, v);
#pragma unroll
    for (int e = 0; e < EPT; ++e) r[e] = csub(r[e], apply_A_at<EPT, RMAX>(v, a, mbits, mp.lam, e));
  }

  float2 z[EPT];
  auto precondition = [&]() {
    if constexpr (PRE == 1) {
#pragma unroll
      for (int e = 0; e < EPT; ++e) sm_f[pidx(j0 + e)] = r[e];
      __syncthreads();
      wiener_precond_pair<J, T, NT>(sm_f, ta, tb, mp.ntap, mp.inv_s2, lam_ma, lam_mb);
#pragma unroll
      for (int e = 0; e < EPT; ++e) z[e] = sm_f[pidx(j0 + e)];
    } else {
#pragma unroll
      for (int e = 0; e < EPT; ++e) z[e] = r[e];
    }
  };
  // r.z and r.r of both columns; warp 0 derives the stopping test and beta
  auto rz_partials = [&](float (&q)[4]) {
    float s0 = 0.0f, s1 = 0.0f, q0 = 0.0f, q1 = 0.0f;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      s0 = fmaf(r[e].x, z[e].x, s0);
      s1 = fmaf(r[e].y, z[e].y, s1);
      q0 = fmaf(r[e].x, r[e].x, q0);
      q1 = fmaf(r[e].y, r[e].y, q1);
    }
    q[0] = s0; q[1] = s1; q[2] = q0; q[3] = q1;
  };
  const double tol = mp.tol;
  precondition();
#pragma unroll
  for (int e = 0; e < EPT; ++e) sm_p[pidx(j0 + e)] = z[e];
  {
    float q[4];
    rz_partials(q);
    block_sum_bcast<4, T>(q, part, res, [st, tol](const double* a, double* o) {
      (void)o;
      const double rel_a = (double)(sqrtf((float)a[2]) / (float)st[5]);
      const double rel_b = (double)(sqrtf((float)a[3]) / (float)st[6]);
      st[9] = rel_a;
      st[10] = rel_b;
      st[4] = (double)((rel_a > tol ? 1 : 0) | (rel_b > tol ? 2 : 0));
      st[7] = a[0];
      st[8] = a[1];
    });
  }
  int act = (int)st[4];

  for (int it = 0; it < mp.max_iter && act; ++it) {
    float2 pw[WIN];
    load_window<J, T, RMAX>(sm_p, j0, pw);
    {
      float q[2];
      float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const float2 ape = apply_A_at<EPT, RMAX>(pw, a, mbits, mp.lam, e);
        s0 = fmaf(pw[e + RMAX].x, ape.x, s0);
        s1 = fmaf(pw[e + RMAX].y, ape.y, s1);
      }
      q[0] = s0;
      q[1] = s1;
      block_sum_bcast<2, T>(q, part, res, [st](const double* pap, double* o) {
        (void)o;
        const int ac = (int)st[4];
        // ratios in FP32 (one rounding); the sums themselves were accumulated in FP64
        st[0] = ((ac & 1) && pap[0] != 0.0) ? (double)((float)st[7] / (float)pap[0]) : 0.0;
        st[1] = ((ac & 2) && pap[1] != 0.0) ? (double)((float)st[8] / (float)pap[1]) : 0.0;
        st[11] += (ac & 1) ? 1.0 : 0.0;
        st[12] += (ac & 2) ? 1.0 : 0.0;
      });
    }
    const float al_a = (float)st[0], al_b = (float)st[1];
    // A p is recomputed here (7 FMA per element) rather than held across the reduction
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const float2 ape = apply_A_at<EPT, RMAX>(pw, a, mbits, mp.lam, e);
      float2 xe = sm_x[pidx(j0 + e)];
      xe.x = fmaf(al_a, pw[e + RMAX].x, xe.x);
      xe.y = fmaf(al_b, pw[e + RMAX].y, xe.y);
      sm_x[pidx(j0 + e)] = xe;
      r[e].x = fmaf(-al_a, ape.x, r[e].x);
      r[e].y = fmaf(-al_b, ape.y, r[e].y);
    }
    precondition();
    {
      float q[4];
      rz_partials(q);
      block_sum_bcast<4, T>(q, part, res, [st, tol](const double* a4, double* o) {
        (void)o;
        const int ac = (int)st[4];
        int nac = 0;
        if (ac & 1) {
          st[9] = (double)(sqrtf((float)a4[2]) / (float)st[5]);
          if (st[9] > tol) nac |= 1;
        }
        if (ac & 2) {
          st[10] = (double)(sqrtf((float)a4[3]) / (float)st[6]);
          if (st[10] > tol) nac |= 2;
        }
        st[2] = ((nac & 1) && st[7] != 0.0) ? (double)((float)a4[0] / (float)st[7]) : 0.0;
        st[3] = ((nac & 2) && st[8] != 0.0) ? (double)((float)a4[1] / (float)st[8]) : 0.0;
        if (nac & 1) st[7] = a4[0];
        if (nac & 2) st[8] = a4[1];
        st[4] = (double)nac;
      });
    }
    act = (int)st[4];
    const float be_a = (float)st[2], be_b = (float)st[3];
    const bool na = act & 1, nb = act & 2;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      float2 pe = sm_p[pidx(j0 + e)];
      if (na) pe.x = fmaf(be_a, pe.x, z[e].x);
      if (nb) pe.y = fmaf(be_b, pe.y, z[e].y);
      sm_p[pidx(j0 + e)] = pe;
    }
    __syncthreads();  // publish sm_p before the next stencil
  }

  // Hand-over to the flexible-CG kernels (the learned solve runs its Wiener-only
  // iterations here, on chip).  A column stays active there if it has not converged
  // and has iterations left (ex_max_iter).  A pair with an active column hands over
  // x, r, the search direction p, z = M_W r of the last step and r.z, in their
  // lane-interleaved layout (element e of thread t at p J + e T + t), with the mask
  // bits and the per-column state; a pair with none is finished here (solution in
  // frame order, iterations and residuals written below) and marked done, so the
  // flexible-CG kernels skip it.
  const bool ex_done = ex.X && !((((int)st[4] & 1) && (int)st[11] < ex_max_iter) ||
                                 (((int)st[4] & 2) && (int)st[12] < ex_max_iter));
  if (ex.X && tid == 0 && ex_done) {
    FcgCol ca = {}, cb = {};
    ca.iters = (int)st[11];
    cb.iters = (int)st[12];
    ca.slot = cb.slot = -1;
    ca.pad = cb.pad = 1;
    ex.cs[2 * p] = ca;
    ex.cs[2 * p + 1] = cb;
  }
  if (ex.X && !ex_done) {
    const size_t vb = (size_t)p * J + tid;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      ex.X[vb + (size_t)e * T] = sm_x[pidx(j0 + e)];
      ex.R[vb + (size_t)e * T] = r[e];
      ex.P[vb + (size_t)e * T] = sm_p[pidx(j0 + e)];
      ex.Z[vb + (size_t)e * T] = z[e];
    }
    ex.mb[(size_t)p * T + tid] = mbits;
    if (tid == 0) {
      const int ac = (int)st[4];
      FcgCol ca = {}, cb = {};
      ca.rz = st[7];
      cb.rz = st[8];
      ca.bnorm = (float)st[5];
      cb.bnorm = (float)st[6];
      ca.rel = (float)st[9];
      cb.rel = (float)st[10];
      ca.s = cb.s = 1.0f;
      ca.lam_m = lam_ma;
      cb.lam_m = lam_mb;
      ca.iters = (int)st[11];
      cb.iters = (int)st[12];
      ca.active = ((ac & 1) && ca.iters < ex_max_iter) ? 1 : 0;
      cb.active = ((ac & 2) && cb.iters < ex_max_iter) ? 1 : 0;
      ca.slot = cb.slot = -1;
      ex.cs[2 * p] = ca;
      ex.cs[2 * p + 1] = cb;
    }
    return;
  }

  // true residual b - A x (FP32 operator, FP64 norms); write the solution
  __syncthreads();
  float2 b[EPT];
  uint32_t mb2;
  build_rhs<J, T, RMAX>(d2p, mask, prior, N, p, j0, ta, tb, mp.inv_s2, mp.lam, mb2, b);
  float2 xw[WIN];
  load_window<J, T, RMAX>(sm_x, j0, xw);
  {
    float q[2];
    float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const float2 qq = csub(b[e], apply_A_at<EPT, RMAX>(xw, a, mbits, mp.lam, e));
      s0 = fmaf(qq.x, qq.x, s0);
      s1 = fmaf(qq.y, qq.y, s1);
      x2[(size_t)p * J + j0 + e] = xw[e + RMAX];
    }
    q[0] = s0;
    q[1] = s1;
    block_sum_bcast<2, T>(q, part, res, NoScalars{});
  }
  if (tid == 0) {
    iters[2 * p] = (int)st[11];
    iters[2 * p + 1] = (int)st[12];
    resid[2 * p] = (float)st[9];
    resid[2 * p + 1] = (float)st[10];
    resid[N + 2 * p] = sqrtf((float)res[0]) / (float)st[5];
    resid[N + 2 * p + 1] = sqrtf((float)res[1]) / (float)st[6];
  }
}

#ifdef IPFB_ML_HOST_KERNELS
// time order [J][N] -> pair-packed [P][J] (initial guess)
__global__ void k_time_to_pairs(const float* __restrict__ x, float2* __restrict__ x2, int N, int J) {
  __shared__ float2 tile[32][33];
  const int H = N / 2;
  const int p0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) {
    const int jj = i / 32, pp = i % 32;
    if (p0 + pp < H && j0 + jj < J)
      tile[jj][pp] = reinterpret_cast<const float2*>(x + (size_t)(j0 + jj) * N)[p0 + pp];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) {
    const int pp = i / 32, jj = i % 32;
    if (p0 + pp < H && j0 + jj < J) x2[(size_t)(p0 + pp) * J + j0 + jj] = tile[jj][pp];
  }
}

#endif  // IPFB_ML_HOST_KERNELS

}  // namespace ipfb
