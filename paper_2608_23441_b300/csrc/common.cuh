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

namespace ipfb {

// ----------------------------------------------------------------------------
// complex float2 arithmetic
// ----------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by +i
__device__ __forceinline__ float2 cmul_i(float2 a) { return make_float2(-a.y, a.x); }

// exp(s * 2 pi i * num / den) with s = -1 (forward) or +1 (inverse), 0 <= num < den.
// sincospif keeps the argument an exact multiple of pi for power-of-two den.
template <bool INV>
__device__ __forceinline__ float2 twiddle(int num, int den) {
  float s, c;
  sincospif(__fdiv_rn(2.0f * (float)num, (float)den), &s, &c);
  return make_float2(c, INV ? s : -s);
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

// ----------------------------------------------------------------------------
// R-point DFT in registers, natural order in and out, radix-2 decimation in time
// ----------------------------------------------------------------------------
template <int K, int H, bool INV>
struct Combine {
  __device__ __forceinline__ static void run(float2* v, const float2* e, const float2* o) {
    float2 t = rot_const<K, 2 * H, INV>(o[K]);
    v[K] = cadd(e[K], t);
    v[K + H] = csub(e[K], t);
    Combine<K + 1, H, INV>::run(v, e, o);
  }
};
template <int H, bool INV>
struct Combine<H, H, INV> {
  __device__ __forceinline__ static void run(float2*, const float2*, const float2*) {}
};

template <int R, bool INV>
struct DFT {
  __device__ __forceinline__ static void run(float2* v) {
    float2 e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    DFT<R / 2, INV>::run(e);
    DFT<R / 2, INV>::run(o);
    Combine<0, R / 2, INV>::run(v, e, o);
  }
};
template <bool INV>
struct DFT<1, INV> {
  __device__ __forceinline__ static void run(float2*) {}
};
template <bool INV>
struct DFT<2, INV> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

// w^r for r = 0..R-1 by a balanced product tree (rounding depth ~log2 R)
template <int R>
__device__ __forceinline__ void twiddle_powers(float2 w, float2* wr) {
  wr[0] = make_float2(1.0f, 0.0f);
  if (R > 1) wr[1] = w;
#pragma unroll
  for (int r = 2; r < R; ++r) wr[r] = cmul(wr[r / 2], wr[r - r / 2]);
}

// padded shared-memory index: one spare float2 after every 16, so that radix-16
// scatters (stride 16 elements) land in distinct banks.
__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> 4); }

// ----------------------------------------------------------------------------
// One Stockham decimation-in-time radix-R pass of an S-point FFT (S = Ns*R*...)
// executed by T threads (BPT butterflies per thread, b = tid + i*T).
//   input element i  : ld(i)      output element i : st(i, v)
// Butterfly b reads elements b + r*S/R, applies exp(-+2 pi i r k / (Ns R)) with
// k = b mod Ns, does an R-point DFT and writes (b/Ns)*Ns*R + k + r*Ns.
// If INPLACE, a block barrier separates all loads from all stores.
// ----------------------------------------------------------------------------
template <int R, int BPT, int T, bool INV, bool INPLACE, class LD, class ST>
__device__ __forceinline__ void stockham_pass(int S, int Ns, int tid, LD ld, ST st) {
  const int nb = S / R;
  float2 v[BPT][R];
#pragma unroll
  for (int i = 0; i < BPT; ++i) {
    const int b = tid + i * T;
    if (b < nb) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = ld(b + r * nb);
      if (Ns > 1) {
        const int k = b % Ns;
        float2 wr[R];
        twiddle_powers<R>(twiddle<INV>(k, Ns * R), wr);
#pragma unroll
        for (int r = 1; r < R; ++r) v[i][r] = cmul(v[i][r], wr[r]);
      }
      DFT<R, INV>::run(v[i]);
    }
  }
  if (INPLACE) __syncthreads();
#pragma unroll
  for (int i = 0; i < BPT; ++i) {
    const int b = tid + i * T;
    if (b < nb) {
      const int k = b % Ns;
      const int j = (b / Ns) * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) st(j + r * Ns, v[i][r]);
    }
  }
}

// Radix choice for the pass that starts at sub-size Ns of an S-point transform:
// the remaining factor if it is <= 32, otherwise 16.
__host__ __device__ constexpr int next_radix(int S, int Ns) {
  return (S / Ns) <= 32 ? (S / Ns) : 16;
}

// Full S-point FFT by T threads.  The first pass reads ld_first, the last writes
// st_last, every intermediate pass works in place on the padded smem array sm.
// Callers must __syncthreads() before (if ld_first reads smem written by others)
// and after (if st_last writes smem read by others).
template <int S, int T, bool INV, int Ns, class LDF, class STL>
struct FFTPasses {
  __device__ __forceinline__ static void run(float2* sm, int tid, LDF ldf, STL stl) {
    constexpr int R = next_radix(S, Ns);
    constexpr int BPT = (S / R + T - 1) / T;
    constexpr bool first = (Ns == 1);
    constexpr bool last = (Ns * R == S);
    auto lds = [sm](int i) { return sm[pidx(i)]; };
    auto sts = [sm](int i, float2 v) { sm[pidx(i)] = v; };
    // every pass separates its loads from its stores by a barrier, so the first
    // pass may read, and the last pass may write, the same smem array
    if constexpr (first && last) {
      stockham_pass<R, BPT, T, INV, true>(S, Ns, tid, ldf, stl);
    } else if constexpr (first) {
      stockham_pass<R, BPT, T, INV, true>(S, Ns, tid, ldf, sts);
      __syncthreads();
      FFTPasses<S, T, INV, Ns * R, LDF, STL>::run(sm, tid, ldf, stl);
    } else if constexpr (last) {
      stockham_pass<R, BPT, T, INV, true>(S, Ns, tid, lds, stl);
    } else {
      stockham_pass<R, BPT, T, INV, true>(S, Ns, tid, lds, sts);
      __syncthreads();
      FFTPasses<S, T, INV, Ns * R, LDF, STL>::run(sm, tid, ldf, stl);
    }
  }
};

template <int S, int T, bool INV, class LDF, class STL>
__device__ __forceinline__ void block_fft(float2* sm, int tid, LDF ldf, STL stl) {
  FFTPasses<S, T, INV, 1, LDF, STL>::run(sm, tid, ldf, stl);
}

}  // namespace ipfb
