// Device helpers shared by the libipfb kernels: complex arithmetic, compile-time
// roots of unity, R-point DFTs held in registers, and Stockham radix passes over
// a padded shared-memory array.
//
// FFT conventions (Sec. 2.3, operator F): forward exp(-2 pi i n k / N),
// unnormalised; inverse exp(+2 pi i n k / N), unnormalised (callers fold 1/N
// into a gain or a pre-scale).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace ipfb {

// ----------------------------------------------------------------------------
// complex float2 arithmetic
// ----------------------------------------------------------------------------
// complex add / subtract on the paired FP32 pipe (add.rn.f32x2: both halves in one
// instruction, IEEE round-to-nearest as the scalar forms)
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  float2 r;
  asm("{\n .reg .b64 ta, tb, td;\n mov.b64 ta, {%2, %3};\n mov.b64 tb, {%4, %5};\n add.rn.f32x2 td, ta, tb;\n mov.b64 {%0, %1}, td;\n}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  float2 r;
  asm("{\n .reg .b64 ta, tb, td;\n mov.b64 ta, {%2, %3};\n mov.b64 tb, {%4, %5};\n sub.rn.f32x2 td, ta, tb;\n mov.b64 {%0, %1}, td;\n}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by +i
__device__ __forceinline__ float2 cmul_i(float2 a) { return make_float2(-a.y, a.x); }

// exp(s * 2 pi i * num / den) with s = -1 (forward) or +1 (inverse), 0 <= num < den.
// For a power-of-two den the argument 2 num / den is formed exactly (a multiply by
// an exact reciprocal), so sincospif sees an exact multiple of pi.
template <bool INV>
__device__ __forceinline__ float2 twiddle(int num, int den) {
  float s, c;
  const float x = ((den & (den - 1)) == 0) ? (float)num * (2.0f / (float)den) : __fdiv_rn(2.0f * (float)num, (float)den);
  sincospif(x, &s, &c);
  return make_float2(c, INV ? s : -s);
}

// exp(-+2 pi i t / L) for 0 <= t < L from two small tables built once per CTA:
//   hi[t >> LO] = exp(-+2 pi i (t >> LO) 2^LO / L),  lo[t & (2^LO - 1)] = exp(-+2 pi i (t & ..) / L)
// one complex multiply and two shared-memory reads per twiddle.
template <int LO>
struct Twid2 {
  const float2* hi;
  const float2* lo;
  __device__ __forceinline__ float2 operator()(int t) const {
    return cmul(hi[t >> LO], lo[t & ((1 << LO) - 1)]);
  }
};

// Fill the two tables for length L (power of two, > 2^LO) with T threads.
template <int LO, bool INV>
__device__ __forceinline__ void twid2_fill(float2* hi, float2* lo, int L, int tid, int T) {
  const int nhi = (L >> LO) > 0 ? (L >> LO) : 1;
  const int nlo = (1 << LO) < L ? (1 << LO) : L;
  for (int i = tid; i < nhi; i += T) hi[i] = twiddle<INV>((i << LO) % L, L);
  for (int i = tid; i < nlo; i += T) lo[i] = twiddle<INV>(i, L);
}

// ----------------------------------------------------------------------------
// compile-time roots of unity (Taylor series in double, evaluated by the compiler)
// ----------------------------------------------------------------------------
constexpr double kPi = 3.14159265358979323846264338327950288;

constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int i = 1; i < 40; ++i) {
    term *= -x * x / (double)((2 * i - 1) * (2 * i));
    sum += term;
  }
  return sum;
}
constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int i = 1; i < 40; ++i) {
    term *= -x * x / (double)((2 * i) * (2 * i + 1));
    sum += term;
  }
  return sum;
}
// cos and sin of 2 pi k / n, angle folded into [-pi, pi]
constexpr double root_cos(int k, int n) {
  int kk = ((k % n) + n) % n;
  if (2 * kk > n) kk -= n;
  return taylor_cos(2.0 * kPi * (double)kk / (double)n);
}
constexpr double root_sin(int k, int n) {
  int kk = ((k % n) + n) % n;
  if (2 * kk > n) kk -= n;
  return taylor_sin(2.0 * kPi * (double)kk / (double)n);
}

// a * W_R^K with W_R = exp(-+2 pi i / R); trivial angles specialised.
template <int K, int R, bool INV>
__device__ __forceinline__ float2 rot_const(float2 a) {
  constexpr int k = K % R;
  if constexpr (k == 0) {
    return a;
  } else if constexpr (4 * k == R) {  // -i (fwd) / +i (inv)
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
  } else if constexpr (2 * k == R) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (4 * k == 3 * R) {  // +i (fwd) / -i (inv)
    return INV ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
  } else if constexpr (8 * k == R) {
    constexpr float h = 0.70710678118654752440f;
    return INV ? make_float2((a.x - a.y) * h, (a.x + a.y) * h)
               : make_float2((a.x + a.y) * h, (a.y - a.x) * h);
  } else if constexpr (8 * k == 3 * R) {
    constexpr float h = 0.70710678118654752440f;
    return INV ? make_float2((-a.x - a.y) * h, (a.x - a.y) * h)
               : make_float2((a.y - a.x) * h, (-a.x - a.y) * h);
  } else {
    constexpr float c = (float)root_cos(K, R);
    constexpr float s = (float)root_sin(K, R);
    return cmul(a, make_float2(c, INV ? s : -s));
  }
}

// a * W_C^q for a runtime q in [0, C) (C a small power of two): the unrolled
// callers pass loop indices, which the compiler turns into constants.
template <int C, bool INV>
__device__ __forceinline__ float2 rotq(float2 a, int q) {
  float2 out = a;
#pragma unroll
  for (int k = 1; k < C; ++k) {
    if (q == k) {
      switch (k) {
        case 1: out = rot_const<1, C, INV>(a); break;
        case 2: out = rot_const<2 % C, C, INV>(a); break;
        case 3: out = rot_const<3 % C, C, INV>(a); break;
        case 4: out = rot_const<4 % C, C, INV>(a); break;
        case 5: out = rot_const<5 % C, C, INV>(a); break;
        case 6: out = rot_const<6 % C, C, INV>(a); break;
        case 7: out = rot_const<7 % C, C, INV>(a); break;
        default: break;
      }
    }
  }
  return out;
}

// ----------------------------------------------------------------------------
// R-point DFT in registers, natural order in and out: in-place radix-2
// decimation-in-frequency stages (block 2H: a + b, (a - b) W_{2H}^i), then the
// bit-reversal permutation as compile-time register swaps.  Peak register use is
// the R values plus one butterfly's temporaries.
// ----------------------------------------------------------------------------
template <int R, bool INV, int H, int P, int I>
__device__ __forceinline__ void dif_bf(float2* v) {
  const float2 a = v[P], b = v[P + H];
  v[P] = cadd(a, b);
  v[P + H] = rot_const<I * (R / (2 * H)), R, INV>(csub(a, b));
}
template <int R, bool INV, int H, int... Is>
__device__ __forceinline__ void dif_stage(float2* v, std::integer_sequence<int, Is...>) {
  (dif_bf<R, INV, H, (Is / H) * 2 * H + Is % H, Is % H>(v), ...);
}
__host__ __device__ constexpr int bitrev(int k, int R) {
  int r = 0;
  for (int m = R >> 1; m >= 1; m >>= 1, k >>= 1) r = (r << 1) | (k & 1);
  return r;
}
template <int R, int K>
__device__ __forceinline__ void bitrev_swap(float2* v) {
  constexpr int B = bitrev(K, R);
  if constexpr (K < B) {
    const float2 t = v[K];
    v[K] = v[B];
    v[B] = t;
  }
}
template <int R, int... Ks>
__device__ __forceinline__ void bitrev_all(float2* v, std::integer_sequence<int, Ks...>) {
  (bitrev_swap<R, Ks>(v), ...);
}
template <int R, bool INV, int H>
__device__ __forceinline__ void dif_stages(float2* v) {
  if constexpr (H >= 1) {
    dif_stage<R, INV, H>(v, std::make_integer_sequence<int, R / 2>{});
    dif_stages<R, INV, H / 2>(v);
  }
}

template <int R, bool INV>
struct DFT {
  __device__ __forceinline__ static void run(float2* v) {
    dif_stages<R, INV, R / 2>(v);
    bitrev_all<R>(v, std::make_integer_sequence<int, R>{});
  }
};
template <bool INV>
struct DFT<1, INV> {
  __device__ __forceinline__ static void run(float2*) {}
};

// w^r for r = 0..R-1 by a balanced product tree (rounding depth ~log2 R)
template <int R>
__device__ __forceinline__ void twiddle_powers(float2 w, float2* wr) {
  wr[0] = make_float2(1.0f, 0.0f);
  if (R > 1) wr[1] = w;
#pragma unroll
  for (int r = 2; r < R; ++r) wr[r] = cmul(wr[r / 2], wr[r - r / 2]);
}

// v[r] *= w^r for r = 1..R-1 without holding all R powers: w^(a + 4b) =
// w^a (a < 4, kept) times w^(4b) (advanced by one multiply per b).  The longest
// product chain is R/4 + 2 multiplies.
template <int R>
__device__ __forceinline__ void apply_twiddles(float2* v, float2 w) {
  if constexpr (R >= 2) v[1] = cmul(v[1], w);
  if constexpr (R >= 4) {
    const float2 w2 = cmul(w, w);
    const float2 w3 = cmul(w2, w);
    v[2] = cmul(v[2], w2);
    v[3] = cmul(v[3], w3);
    if constexpr (R > 4) {
      const float2 w4 = cmul(w2, w2);
      float2 wb = w4;
#pragma unroll
      for (int b = 1; b < R / 4; ++b) {
        v[4 * b] = cmul(v[4 * b], wb);
        v[4 * b + 1] = cmul(v[4 * b + 1], cmul(wb, w));
        v[4 * b + 2] = cmul(v[4 * b + 2], cmul(wb, w2));
        v[4 * b + 3] = cmul(v[4 * b + 3], cmul(wb, w3));
        if (b + 1 < R / 4) wb = cmul(wb, w4);
      }
    }
  }
}

// asynchronous 16-byte global -> shared copies (both addresses 16-byte aligned):
// issue, close the group, wait for all of this thread's groups
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// padded shared-memory index: one spare float2 after every 16, so that radix-16
// scatters (stride 16 elements) land in distinct banks.
__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> 4); }

// ----------------------------------------------------------------------------
// Addressing policies for the Stockham passes.  A pass loads element b + r*nb of
// its input and stores element j + r*Ns of its output (r < R); the policies turn
// that into a per-butterfly base plus a compile-time offset per r wherever the
// layout allows it.
//   SPad : the padded shared array (element i at pidx(i)); constant offsets when
//          nb % 16 == 0 (loads) and Ns % 16 == 0 or Ns == 1 with R % 16 == 0 (stores).
//   GMem : a plain array (global memory), element i at p[i].
//   FnLd / FnSt : arbitrary element functions (computed loads, scattered stores).
// ----------------------------------------------------------------------------
struct SPad {
  float2* p;
  template <int R, int NB>
  __device__ __forceinline__ int lbase(int b) const {
    if constexpr (NB % 16 == 0) return pidx(b);
    else return b;
  }
  template <int R, int NB>
  __device__ __forceinline__ float2 ld(int base, int r) const {
    if constexpr (NB % 16 == 0) return p[base + r * (NB + NB / 16)];
    else return p[pidx(base + r * NB)];
  }
  template <int R, int NS>
  __device__ __forceinline__ int sbase(int j) const {
    if constexpr ((NS == 1 && R % 16 == 0) || NS % 16 == 0) return pidx(j);
    else return j;
  }
  template <int R, int NS>
  __device__ __forceinline__ void st(int base, int r, float2 v) const {
    if constexpr (NS == 1 && R % 16 == 0) p[base + r + r / 16] = v;
    else if constexpr (NS % 16 == 0) p[base + r * (NS + NS / 16)] = v;
    else p[pidx(base + r * NS)] = v;
  }
};
struct GMem {
  float2* p;
  template <int R, int NB>
  __device__ __forceinline__ int lbase(int b) const { return b; }
  template <int R, int NB>
  __device__ __forceinline__ float2 ld(int base, int r) const { return p[base + r * NB]; }
  template <int R, int NS>
  __device__ __forceinline__ int sbase(int j) const { return j; }
  template <int R, int NS>
  __device__ __forceinline__ void st(int base, int r, float2 v) const { p[base + r * NS] = v; }
};
template <class F>
struct FnLd {
  F f;
  template <int R, int NB>
  __device__ __forceinline__ int lbase(int b) const { return b; }
  template <int R, int NB>
  __device__ __forceinline__ float2 ld(int base, int r) const { return f(base + r * NB); }
};
template <class F>
struct FnSt {
  F f;
  template <int R, int NS>
  __device__ __forceinline__ int sbase(int j) const { return j; }
  template <int R, int NS>
  __device__ __forceinline__ void st(int base, int r, float2 v) const { f(base + r * NS, v); }
};
template <class F>
__device__ __forceinline__ FnLd<F> fn_ld(F f) { return FnLd<F>{f}; }
template <class F>
__device__ __forceinline__ FnSt<F> fn_st(F f) { return FnSt<F>{f}; }

// ----------------------------------------------------------------------------
// One Stockham decimation-in-time radix-R pass of an S-point FFT (sub-size Ns ->
// Ns*R) executed by T threads (BPT butterflies per thread, b = tid + i*T).
// Butterfly b reads elements b + r*S/R, applies exp(-+2 pi i r k / (Ns R)) with
// k = b mod Ns, does an R-point DFT and writes (b/Ns)*Ns*R + k + r*Ns.
// A block barrier separates all loads from all stores (in-place safe).
// ----------------------------------------------------------------------------
template <int R, int BPT, int T, bool INV, int S, int Ns, class LD, class ST>
__device__ __forceinline__ void stockham_pass(int tid, const LD& ld, const ST& st) {
  constexpr int nb = S / R;
  float2 v[BPT][R];
#pragma unroll
  for (int i = 0; i < BPT; ++i) {
    const int b = tid + i * T;
    if (nb % T == 0 || b < nb) {
      const int lb = ld.template lbase<R, nb>(b);
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = ld.template ld<R, nb>(lb, r);
      if constexpr (Ns > 1) apply_twiddles<R>(v[i], twiddle<INV>(b % Ns, Ns * R));
      DFT<R, INV>::run(v[i]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < BPT; ++i) {
    const int b = tid + i * T;
    if (nb % T == 0 || b < nb) {
      const int j = (b / Ns) * Ns * R + b % Ns;
      const int sb = st.template sbase<R, Ns>(j);
#pragma unroll
      for (int r = 0; r < R; ++r) st.template st<R, Ns>(sb, r, v[i][r]);
    }
  }
}

// Radix choice for the pass that starts at sub-size Ns of an S-point transform:
// the remaining factor if it is <= MAXR (32 by default), otherwise 16 (or MAXR if smaller).
// A radix-32 pass is placed first (Ns == 1, where it needs no twiddles) when the
// size is 32 x 16^k, so that no pass holds 32 twiddles in registers.
__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v / 2); }
__host__ __device__ constexpr int next_radix(int S, int Ns, int MAXR = 32) {
  return (S / Ns) <= (MAXR < 16 ? MAXR : 16) ? (S / Ns)
         : (Ns == 1 && MAXR >= 32 && ilog2c(S) % 4 == 1) ? 32
         : (MAXR < 16 ? MAXR : 16);
}

// radix of the last pass of the plan chosen by next_radix for an S-point transform
__host__ __device__ constexpr int last_radix(int S, int MAXR = 32) {
  int Ns = 1;
  while (true) {
    const int R = next_radix(S, Ns, MAXR);
    if (Ns * R == S) return R;
    Ns *= R;
  }
}

// Full S-point FFT by T threads.  The first pass reads `first` (a policy), the
// last writes `last`, every intermediate pass works in place on the padded smem
// array sm.  Passes are separated by block barriers.
template <int S, int T, bool INV, int Ns, int MAXR, class LDF, class STL>
__device__ __forceinline__ void fft_passes(float2* sm, int tid, const LDF& first, const STL& last) {
  constexpr int R = next_radix(S, Ns, MAXR);
  constexpr int BPT = (S / R + T - 1) / T;
  constexpr bool is_first = (Ns == 1);
  constexpr bool is_last = (Ns * R == S);
  const SPad pad{sm};
  if constexpr (is_first && is_last) {
    stockham_pass<R, BPT, T, INV, S, Ns>(tid, first, last);
  } else if constexpr (is_first) {
    stockham_pass<R, BPT, T, INV, S, Ns>(tid, first, pad);
    __syncthreads();
    fft_passes<S, T, INV, Ns * R, MAXR>(sm, tid, first, last);
  } else if constexpr (is_last) {
    stockham_pass<R, BPT, T, INV, S, Ns>(tid, pad, last);
  } else {
    stockham_pass<R, BPT, T, INV, S, Ns>(tid, pad, pad);
    __syncthreads();
    fft_passes<S, T, INV, Ns * R, MAXR>(sm, tid, first, last);
  }
}

template <int S, int T, bool INV, int MAXR = 32, class LDF, class STL>
__device__ __forceinline__ void block_fft(float2* sm, int tid, const LDF& first, const STL& last) {
  fft_passes<S, T, INV, 1, MAXR>(sm, tid, first, last);
}

}  // namespace ipfb
