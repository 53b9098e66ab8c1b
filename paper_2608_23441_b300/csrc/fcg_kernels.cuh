// Flexible conjugate gradient (Notay 2000, Polak-Ribiere beta) for the ML solve of
// Sec. 4.2 (Eq. chi squared) with the learned preconditioner
//     z = u + lam mbar M_W(s g(u / s, m)),   u = M_W r (the Wiener preconditioner),
//     s = RMS(u), lam mbar = prior weight x the column's mask mean,
// g the convolutional net of net_kernels.cuh applied per column.  Because g is
// nonlinear the outer iteration is flexible CG:
//     alpha = r.z / p.Ap,  x += alpha p,  r -= alpha Ap,
//     beta = r_new.(z_new - z_old) / r_old.z_old,  p = z_new + beta p.
// One iteration is two launches: k5_fcg_step (one CTA per column pair: finish the
// previous preconditioner request, update p, x, r, test convergence, form u and the
// net input of the columns still active) and the net forward over the requests.
// Requests are compacted: a column that is still active takes the next free slot
// of the request buffer (atomic counter), so the net runs over active columns only.
// All vectors are FP32 column pairs (column 2p in .x, 2p+1 in .y).  Thread t of pair
// p works on frames t EPT .. t EPT + EPT - 1 (the stencil reads its neighbours in
// shared memory), so the iteration vectors X, R, P, Z, U are stored lane-interleaved:
// element e of thread t at p J + e T + t, which makes every warp access one contiguous
// run.  X enters (initial guess) and leaves (k5_fcg_finish) in frame order [P][J];
// the net's inputs and outputs stay in frame order [slot][J], moved as float4.
#pragma once

#include "ml_kernels.cuh"

namespace ipfb {

template <int NT, int RMAX>
__device__ __forceinline__ void load_taps_stencil(const float* __restrict__ window, int N, int p, int ntap,
                                                  float inv_s2, float (&ta)[NT > 0 ? NT : kMlMaxTaps],
                                                  float (&tb)[NT > 0 ? NT : kMlMaxTaps], float2 (&a)[RMAX + 1]) {
  constexpr int NMAX = NT > 0 ? NT : kMlMaxTaps;
#pragma unroll
  for (int t = 0; t < NMAX; ++t) {
    ta[t] = (t < ntap) ? __ldg(window + (size_t)t * N + 2 * p) : 0.0f;
    tb[t] = (t < ntap) ? __ldg(window + (size_t)t * N + 2 * p + 1) : 0.0f;
  }
#pragma unroll
  for (int s = 0; s <= RMAX; ++s) {
    float sa = 0.0f, sb = 0.0f;
#pragma unroll
    for (int r = 0; r + s < NMAX; ++r) {
      sa = fmaf(ta[r], ta[r + s], sa);
      sb = fmaf(tb[r], tb[r + s], sb);
    }
    a[s] = make_float2(sa * inv_s2, sb * inv_s2);
  }
}

template <int EPT>
__device__ __forceinline__ uint32_t load_mbits(const uint8_t* __restrict__ mask, int N, int p, int j0) {
  uint32_t mb = 0;
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const uint16_t mm = *reinterpret_cast<const uint16_t*>(mask + (size_t)(j0 + e) * N + 2 * p);
    if (mm & 0xFFu) mb |= 1u << e;
    if (mm >> 8) mb |= 1u << (e + 16);
  }
  return mb;
}

// u = M_W r for this CTA's pair (r in registers -> u in registers), RMS scales of u,
// request slots for the columns in `req` (bit 0: column 2p, bit 1: 2p + 1), and their
// net input rows
//   netin[slot][0][j] = u_j / s,  netin[slot][1][j] = m_j.
template <int J, int T, int NT>
__device__ __forceinline__ void fcg_request(const float2 (&r)[J / T], float2 (&u)[J / T], float2* sm_f, float* part,
                                            double* res, int* sflag, const float* ta, const float* tb, int ntap,
                                            float inv_s2, float lam_ma, float lam_mb, int req, uint32_t mbits,
                                            int* __restrict__ counter, float* __restrict__ netin, float& s_a,
                                            float& s_b, int& slot_a, int& slot_b) {
  constexpr int EPT = J / T;
  const int tid = threadIdx.x, j0 = tid * EPT;
#pragma unroll
  for (int e = 0; e < EPT; ++e) sm_f[pidx(j0 + e)] = r[e];
  __syncthreads();
  wiener_precond_pair<J, T, NT>(sm_f, ta, tb, ntap, inv_s2, lam_ma, lam_mb);
#pragma unroll
  for (int e = 0; e < EPT; ++e) u[e] = sm_f[pidx(j0 + e)];
  float q[2] = {0.0f, 0.0f};
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    q[0] = fmaf(u[e].x, u[e].x, q[0]);
    q[1] = fmaf(u[e].y, u[e].y, q[1]);
  }
  block_sum_bcast<2, T>(q, part, res, NoScalars{});
  s_a = res[0] > 0.0 ? sqrtf((float)(res[0] / (double)J)) : 1.0f;
  s_b = res[1] > 0.0 ? sqrtf((float)(res[1] / (double)J)) : 1.0f;
  if (tid == 0) {
    const int base = req ? atomicAdd(counter, __popc(req & 3)) : 0;
    sflag[0] = (req & 1) ? base : -1;
    sflag[1] = (req & 1) ? ((req & 2) ? base + 1 : -1) : ((req & 2) ? base : -1);
  }
  __syncthreads();
  slot_a = sflag[0];
  slot_b = sflag[1];
  const float ia = 1.0f / s_a, ib = 1.0f / s_b;
  static_assert(EPT % 4 == 0, "float4 rows");
  auto mk = [&](int bit) { return ((mbits >> bit) & 1u) ? 1.0f : 0.0f; };
#pragma unroll
  for (int q = 0; q < EPT / 4; ++q) {
    const int e = 4 * q;
    if (slot_a >= 0) {
      float4* row = reinterpret_cast<float4*>(netin + ((size_t)slot_a * 2) * J + j0);
      row[q] = make_float4(u[e].x * ia, u[e + 1].x * ia, u[e + 2].x * ia, u[e + 3].x * ia);
      row[J / 4 + q] = make_float4(mk(e), mk(e + 1), mk(e + 2), mk(e + 3));
    }
    if (slot_b >= 0) {
      float4* row = reinterpret_cast<float4*>(netin + ((size_t)slot_b * 2) * J + j0);
      row[q] = make_float4(u[e].y * ib, u[e + 1].y * ib, u[e + 2].y * ib, u[e + 3].y * ib);
      row[J / 4 + q] = make_float4(mk(e + 16), mk(e + 17), mk(e + 18), mk(e + 19));
    }
  }
}

template <int J, int T>
constexpr size_t fcg_smem_bytes() {
  return 2 * (size_t)padded_len(J) * sizeof(float2) + 8 * sizeof(double) + (size_t)(T / 32) * 4 * sizeof(float) +
         4 * sizeof(int);
}

// phase 0: r0 = b - A x0, first request, P = Z = 0.  phase 1: z0 from the net, p = z0.
// phase 2: z from the net, Polak-Ribiere beta, p update (with rz = 0 after phase 0,
// beta is 0 and phase 2 does what phase 1 does).  phase 3: resume from the state that
// k5_ml_cg handed over (search direction P and r.z already formed).  Phases 1 to 3
// then take one CG step and issue the next request for the columns still active.
template <int J, int T, int RMAX, int NT>
__device__ __forceinline__ void fcg_step_pair(int p, int phase, const float2* __restrict__ d2, float2* __restrict__ X,
                                              float2* __restrict__ R, float2* __restrict__ Pv,
                                              float2* __restrict__ Z, float2* __restrict__ U,
                                              const uint8_t* __restrict__ mask, const float* __restrict__ prior,
                                              const float* __restrict__ window, int N, const MLParams& mp,
                                              FcgCol* __restrict__ cs, const float* __restrict__ Y,
                                              float* __restrict__ netin, uint32_t* __restrict__ mbc,
                                              int* __restrict__ counter, float2* smem) {
  constexpr int EPT = J / T;
  constexpr int WIN = EPT + 2 * RMAX;
  constexpr int NMAX = NT > 0 ? NT : kMlMaxTaps;
  float2* sm_p = smem;
  float2* sm_f = sm_p + padded_len(J);
  double* res = reinterpret_cast<double*>(sm_f + padded_len(J));
  float* part = reinterpret_cast<float*>(res + 8);
  int* sflag = reinterpret_cast<int*>(part + (T / 32) * 4);

  const int tid = threadIdx.x, j0 = tid * EPT;
  const size_t vb = (size_t)p * J + tid;  // element e of this thread at vb + e T
  FcgCol sa = {}, sb = {};
  if (phase != 0) {
    sa = cs[2 * p];
    sb = cs[2 * p + 1];
    if (!sa.active && !sb.active) return;
  }
  float ta[NMAX], tb[NMAX];
  float2 a[RMAX + 1];
  load_taps_stencil<NT, RMAX>(window, N, p, mp.ntap, mp.inv_s2, ta, tb, a);

  uint32_t mbits;
  float2 r[EPT];
  if (phase == 0) {
    build_rhs<J, T, RMAX>(d2 + (size_t)p * J, mask, prior, N, p, j0, ta, tb, mp.inv_s2, mp.lam, mbits, r);
    mbc[(size_t)p * T + tid] = mbits;  // the mask bits of this thread's frames, for the later steps
    float q[4] = {0.0f, 0.0f, (float)__popc(mbits & 0xFFFFu), (float)__popc(mbits >> 16)};
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      q[0] = fmaf(r[e].x, r[e].x, q[0]);
      q[1] = fmaf(r[e].y, r[e].y, q[1]);
    }
    block_sum_bcast<4, T>(q, part, res, NoScalars{});
    sa.bnorm = res[0] > 0.0 ? sqrtf((float)res[0]) : 1.0f;
    sb.bnorm = res[1] > 0.0 ? sqrtf((float)res[1]) : 1.0f;
    sa.lam_m = mp.lam * (float)(res[2] / (double)J);
    sb.lam_m = mp.lam * (float)(res[3] / (double)J);
    if (mp.use_x0) {
      // the initial guess arrives in frame order: coalesced into shared memory, then
      // stored back lane-interleaved (every read of X precedes the barrier)
#pragma unroll
      for (int i = 0; i < EPT; ++i) sm_p[pidx(tid + i * T)] = X[(size_t)p * J + tid + i * T];
      __syncthreads();
#pragma unroll
      for (int e = 0; e < EPT; ++e) X[vb + (size_t)e * T] = sm_p[pidx(j0 + e)];
      float2 v[WIN];
      load_window<J, T, RMAX>(sm_p, j0, v);
#pragma unroll
      for (int e = 0; e < EPT; ++e) r[e] = csub(r[e], apply_A_at<EPT, RMAX>(v, a, mbits, mp.lam, e));
    } else {
#pragma unroll
      for (int e = 0; e < EPT; ++e) X[vb + (size_t)e * T] = make_float2(0.0f, 0.0f);
    }
    float q2[2] = {0.0f, 0.0f};
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      q2[0] = fmaf(r[e].x, r[e].x, q2[0]);
      q2[1] = fmaf(r[e].y, r[e].y, q2[1]);
    }
    block_sum_bcast<2, T>(q2, part, res, NoScalars{});
    sa.rel = sqrtf((float)res[0]) / sa.bnorm;
    sb.rel = sqrtf((float)res[1]) / sb.bnorm;
    sa.active = (sa.rel > mp.tol && mp.max_iter > 0) ? 1 : 0;
    sb.active = (sb.rel > mp.tol && mp.max_iter > 0) ? 1 : 0;
    sa.iters = sb.iters = 0;
    sa.rz = sb.rz = 0.0;
    sa.slot = sb.slot = -1;
    // P and Z start at zero, so that the first step after the net (rz = 0, beta = 0)
    // can run as phase 2 too: a graph loop body then repeats one fixed launch
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      R[vb + (size_t)e * T] = r[e];
      Pv[vb + (size_t)e * T] = make_float2(0.0f, 0.0f);
      Z[vb + (size_t)e * T] = make_float2(0.0f, 0.0f);
    }
  } else {
    mbits = mbc[(size_t)p * T + tid];
    const bool aa = sa.active, ab = sb.active;
    // columns whose preconditioner request went to the net this iteration
    const bool na = aa && sa.slot >= 0, nb = ab && sb.slot >= 0;
    float2 z[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) r[e] = R[vb + (size_t)e * T];
    if (phase == 3) {
#pragma unroll
      for (int e = 0; e < EPT; ++e) sm_p[pidx(j0 + e)] = Pv[vb + (size_t)e * T];
    } else {
#pragma unroll
      for (int e = 0; e < EPT; ++e) z[e] = U[vb + (size_t)e * T];
      if (na || nb) {
        // z = u + lam mbar M_W(s y) = M_W(r + lam mbar s y): the net's output enters
        // through the Wiener preconditioner weighted by the column's prior term, i.e.
        // mode k of it is scaled by rho(k) = lam mbar / (|W(k)|^2 / sigma^2 + lam mbar),
        // near 1 where the prior dominates (the near-null eigenvalues of App. A) and
        // near 0 where the Wiener step already resolves the mode, which is left as it is.
#pragma unroll
        for (int q = 0; q < EPT / 4; ++q) {
          const float4 va = na ? reinterpret_cast<const float4*>(Y + (size_t)sa.slot * J + j0)[q]
                               : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          const float4 vb4 = nb ? reinterpret_cast<const float4*>(Y + (size_t)sb.slot * J + j0)[q]
                                : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          const float ya[4] = {va.x, va.y, va.z, va.w}, yb[4] = {vb4.x, vb4.y, vb4.z, vb4.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) sm_f[pidx(j0 + 4 * q + i)] = make_float2(sa.s * ya[i], sb.s * yb[i]);
        }
        __syncthreads();
        wiener_precond_pair<J, T, NT>(sm_f, ta, tb, mp.ntap, mp.inv_s2, sa.lam_m, sb.lam_m);
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          const float2 c = sm_f[pidx(j0 + e)];
          if (na) z[e].x = fmaf(sa.lam_m, c.x, z[e].x);
          if (nb) z[e].y = fmaf(sb.lam_m, c.y, z[e].y);
        }
      }
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        if (!aa) z[e].x = 0.0f;
        if (!ab) z[e].y = 0.0f;
      }
      // r.z_new (and r.z_old for the Polak-Ribiere beta)
      float q[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      float2 zo[EPT];
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        zo[e] = phase == 2 ? Z[vb + (size_t)e * T] : make_float2(0.0f, 0.0f);
        q[0] = fmaf(r[e].x, z[e].x, q[0]);
        q[1] = fmaf(r[e].y, z[e].y, q[1]);
        q[2] = fmaf(r[e].x, zo[e].x, q[2]);
        q[3] = fmaf(r[e].y, zo[e].y, q[3]);
      }
      block_sum_bcast<4, T>(q, part, res, NoScalars{});
      float be_a = 0.0f, be_b = 0.0f;
      if (phase == 2) {
        be_a = (aa && sa.rz != 0.0) ? (float)((res[0] - res[2]) / sa.rz) : 0.0f;
        be_b = (ab && sb.rz != 0.0) ? (float)((res[1] - res[3]) / sb.rz) : 0.0f;
      }
      if (aa) sa.rz = res[0];
      if (ab) sb.rz = res[1];
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        float2 pe = phase == 2 ? Pv[vb + (size_t)e * T] : make_float2(0.0f, 0.0f);
        if (aa) pe.x = fmaf(be_a, pe.x, z[e].x);
        if (ab) pe.y = fmaf(be_b, pe.y, z[e].y);
        if (!aa) pe.x = 0.0f;
        if (!ab) pe.y = 0.0f;
        sm_p[pidx(j0 + e)] = pe;
        Pv[vb + (size_t)e * T] = pe;
        Z[vb + (size_t)e * T] = z[e];
      }
    }
    __syncthreads();
    float2 pw[WIN];
    load_window<J, T, RMAX>(sm_p, j0, pw);
    float q2[2] = {0.0f, 0.0f};
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const float2 ape = apply_A_at<EPT, RMAX>(pw, a, mbits, mp.lam, e);
      q2[0] = fmaf(pw[e + RMAX].x, ape.x, q2[0]);
      q2[1] = fmaf(pw[e + RMAX].y, ape.y, q2[1]);
    }
    block_sum_bcast<2, T>(q2, part, res, NoScalars{});
    const float al_a = (aa && res[0] != 0.0) ? (float)(sa.rz / res[0]) : 0.0f;
    const float al_b = (ab && res[1] != 0.0) ? (float)(sb.rz / res[1]) : 0.0f;
    float q3[2] = {0.0f, 0.0f};
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const float2 ape = apply_A_at<EPT, RMAX>(pw, a, mbits, mp.lam, e);
      float2 xe = X[vb + (size_t)e * T];
      xe.x = fmaf(al_a, pw[e + RMAX].x, xe.x);
      xe.y = fmaf(al_b, pw[e + RMAX].y, xe.y);
      X[vb + (size_t)e * T] = xe;
      r[e].x = fmaf(-al_a, ape.x, r[e].x);
      r[e].y = fmaf(-al_b, ape.y, r[e].y);
      R[vb + (size_t)e * T] = r[e];
      q3[0] = fmaf(r[e].x, r[e].x, q3[0]);
      q3[1] = fmaf(r[e].y, r[e].y, q3[1]);
    }
    block_sum_bcast<2, T>(q3, part, res, NoScalars{});
    if (aa) {
      sa.iters += 1;
      sa.rel = sqrtf((float)res[0]) / sa.bnorm;
      sa.active = (sa.rel > mp.tol && sa.iters < mp.max_iter) ? 1 : 0;
    }
    if (ab) {
      sb.iters += 1;
      sb.rel = sqrtf((float)res[1]) / sb.bnorm;
      sb.active = (sb.rel > mp.tol && sb.iters < mp.max_iter) ? 1 : 0;
    }
  }
  const int act = (sa.active ? 1 : 0) | (sb.active ? 2 : 0);
  // the net is asked only from a column's net_from-th preconditioner application on;
  // before that its z is the Wiener term alone
  const int req = (sa.active && sa.iters >= mp.net_from ? 1 : 0) | (sb.active && sb.iters >= mp.net_from ? 2 : 0);
  if (act) {
    float2 u[EPT];
    float s_a, s_b;
    int sl_a, sl_b;
    fcg_request<J, T, NT>(r, u, sm_f, part, res, sflag, ta, tb, mp.ntap, mp.inv_s2, sa.lam_m, sb.lam_m, req, mbits,
                          counter, netin, s_a, s_b, sl_a, sl_b);
#pragma unroll
    for (int e = 0; e < EPT; ++e) U[vb + (size_t)e * T] = u[e];
    sa.s = s_a;
    sb.s = s_b;
    sa.slot = sl_a;
    sb.slot = sl_b;
  } else {
    sa.slot = sb.slot = -1;
  }
  if (tid == 0) {
    cs[2 * p] = sa;
    cs[2 * p + 1] = sb;
  }
}

// One flexible-CG step over the column pairs.  A grid of G CTAs (one per SM) walks
// the pairs p = blockIdx.x + i G: every pair in phase 0, otherwise only the pairs with
// an active column (listed in shared memory first), so that a step near the end of a
// solve costs the few pairs still running rather than a launch wave per SM-full of
// finished ones.
template <int J, int T, int RMAX, int NT>
__global__ void __launch_bounds__(T, 1)
k5_fcg_step(int phase, const float2* __restrict__ d2, float2* __restrict__ X, float2* __restrict__ R,
            float2* __restrict__ Pv, float2* __restrict__ Z, float2* __restrict__ U, const uint8_t* __restrict__ mask,
            const float* __restrict__ prior, const float* __restrict__ window, int N, MLParams mp,
            FcgCol* __restrict__ cs, const float* __restrict__ Y, float* __restrict__ netin,
            uint32_t* __restrict__ mbc, int* __restrict__ counter) {
  extern __shared__ float2 smem[];
  __shared__ int plist[T];
  __shared__ int nlist;
  const int P = N / 2, G = gridDim.x;
  for (int base = blockIdx.x; base < P; base += G * T) {
    __syncthreads();  // the previous chunk's list and pairs are done
    if (threadIdx.x == 0) nlist = 0;
    __syncthreads();
    const int pp = base + threadIdx.x * G;
    if (pp < P && (phase == 0 || cs[2 * pp].active || cs[2 * pp + 1].active)) plist[atomicAdd(&nlist, 1)] = pp;
    __syncthreads();
    const int n = nlist;
    for (int k = 0; k < n; ++k) {
      __syncthreads();  // the previous pair's shared-memory readers are done
      fcg_step_pair<J, T, RMAX, NT>(plist[k], phase, d2, X, R, Pv, Z, U, mask, prior, window, N, mp, cs, Y, netin,
                                    mbc, counter, smem);
    }
  }
}

// True residual b - A x (FP32 operator, FP64 norms) and the per-column outputs.
template <int J, int T, int RMAX, int NT>
__global__ void __launch_bounds__(T, 1)
k5_fcg_finish(const float2* __restrict__ d2, float2* __restrict__ X, const uint8_t* __restrict__ mask,
              const float* __restrict__ prior, const float* __restrict__ window, int N, MLParams mp,
              const FcgCol* __restrict__ cs, int* __restrict__ iters, float* __restrict__ resid) {
  constexpr int EPT = J / T;
  constexpr int WIN = EPT + 2 * RMAX;
  constexpr int NMAX = NT > 0 ? NT : kMlMaxTaps;
  extern __shared__ float2 smem[];
  float2* sm_p = smem;
  double* res = reinterpret_cast<double*>(sm_p + 2 * padded_len(J));
  float* part = reinterpret_cast<float*>(res + 8);
  const int tid = threadIdx.x, p = blockIdx.x, j0 = tid * EPT;
  if (cs[2 * p].pad) return;  // finished in the on-chip CG kernel (solution and outputs written)
  float ta[NMAX], tb[NMAX];
  float2 a[RMAX + 1];
  load_taps_stencil<NT, RMAX>(window, N, p, mp.ntap, mp.inv_s2, ta, tb, a);
  uint32_t mbits;
  float2 b[EPT];
  build_rhs<J, T, RMAX>(d2 + (size_t)p * J, mask, prior, N, p, j0, ta, tb, mp.inv_s2, mp.lam, mbits, b);
#pragma unroll
  for (int e = 0; e < EPT; ++e) sm_p[pidx(j0 + e)] = X[(size_t)p * J + (size_t)e * T + tid];
  __syncthreads();
  // X back to frame order for the caller (every read of X precedes the barrier)
#pragma unroll
  for (int i = 0; i < EPT; ++i) X[(size_t)p * J + tid + i * T] = sm_p[pidx(tid + i * T)];
  float2 xw[WIN];
  load_window<J, T, RMAX>(sm_p, j0, xw);
  float q[2] = {0.0f, 0.0f};
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const float2 qq = csub(b[e], apply_A_at<EPT, RMAX>(xw, a, mbits, mp.lam, e));
    q[0] = fmaf(qq.x, qq.x, q[0]);
    q[1] = fmaf(qq.y, qq.y, q[1]);
  }
  block_sum_bcast<2, T>(q, part, res, NoScalars{});
  if (tid == 0) {
    const FcgCol sa = cs[2 * p], sb = cs[2 * p + 1];
    iters[2 * p] = sa.iters;
    iters[2 * p + 1] = sb.iters;
    resid[2 * p] = sa.rel;
    resid[2 * p + 1] = sb.rel;
    resid[N + 2 * p] = sqrtf((float)res[0]) / sa.bnorm;
    resid[N + 2 * p + 1] = sqrtf((float)res[1]) / sb.bnorm;
  }
}

// Training pairs for the net (one CTA per listed column pair i, pair index pl[i]):
//   e = x* - x_k,  r = A e,  u = M_W r,  s = RMS(u),
//   xin[2i + h] = (u / s, m),  target[2i + h] = (e - u) / s   (h = 0: column 2p, 1: 2p + 1),
// the target being what the net must add to u so that z = u + s g equals A^{-1} r = e.
template <int J, int T, int RMAX, int NT>
__global__ void __launch_bounds__(T, 1)
k5_net_pairs(const float2* __restrict__ xs, const float2* __restrict__ xk, const int* __restrict__ pl,
             const uint8_t* __restrict__ mask, const float* __restrict__ window, int N, MLParams mp,
             float* __restrict__ xin, float* __restrict__ target) {
  constexpr int EPT = J / T;
  constexpr int WIN = EPT + 2 * RMAX;
  constexpr int NMAX = NT > 0 ? NT : kMlMaxTaps;
  extern __shared__ float2 smem[];
  float2* sm_p = smem;
  float2* sm_f = sm_p + padded_len(J);
  double* res = reinterpret_cast<double*>(sm_f + padded_len(J));
  float* part = reinterpret_cast<float*>(res + 8);
  const int tid = threadIdx.x, i = blockIdx.x, p = pl[i], j0 = tid * EPT;
  float ta[NMAX], tb[NMAX];
  float2 a[RMAX + 1];
  load_taps_stencil<NT, RMAX>(window, N, p, mp.ntap, mp.inv_s2, ta, tb, a);
  const uint32_t mbits = load_mbits<EPT>(mask, N, p, j0);
  float2 e_[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    e_[e] = csub(xs[(size_t)p * J + j0 + e], xk[(size_t)p * J + j0 + e]);
    sm_p[pidx(j0 + e)] = e_[e];
  }
  float q[2] = {(float)__popc(mbits & 0xFFFFu), (float)__popc(mbits >> 16)};
  block_sum_bcast<2, T>(q, part, res, NoScalars{});
  const float lam_ma = mp.lam * (float)(res[0] / (double)J), lam_mb = mp.lam * (float)(res[1] / (double)J);
  float2 v[WIN];
  load_window<J, T, RMAX>(sm_p, j0, v);
#pragma unroll
  for (int e = 0; e < EPT; ++e) sm_f[pidx(j0 + e)] = apply_A_at<EPT, RMAX>(v, a, mbits, mp.lam, e);
  __syncthreads();
  wiener_precond_pair<J, T, NT>(sm_f, ta, tb, mp.ntap, mp.inv_s2, lam_ma, lam_mb);
  float2 u[EPT];
  float q2[2] = {0.0f, 0.0f};
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    u[e] = sm_f[pidx(j0 + e)];
    q2[0] = fmaf(u[e].x, u[e].x, q2[0]);
    q2[1] = fmaf(u[e].y, u[e].y, q2[1]);
  }
  block_sum_bcast<2, T>(q2, part, res, NoScalars{});
  const float sa = res[0] > 0.0 ? sqrtf((float)(res[0] / (double)J)) : 1.0f;
  const float sb = res[1] > 0.0 ? sqrtf((float)(res[1] / (double)J)) : 1.0f;
  const float ia = 1.0f / sa, ib = 1.0f / sb;
  const size_t ca = (size_t)(2 * i), cb = ca + 1;
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    xin[(ca * 2) * J + j0 + e] = u[e].x * ia;
    xin[(ca * 2 + 1) * J + j0 + e] = ((mbits >> e) & 1u) ? 1.0f : 0.0f;
    xin[(cb * 2) * J + j0 + e] = u[e].y * ib;
    xin[(cb * 2 + 1) * J + j0 + e] = ((mbits >> (e + 16)) & 1u) ? 1.0f : 0.0f;
    target[ca * J + j0 + e] = (e_[e].x - u[e].x) * ia;
    target[cb * J + j0 + e] = (e_[e].y - u[e].y) * ib;
  }
}

}  // namespace ipfb
