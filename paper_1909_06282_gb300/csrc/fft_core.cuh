// In-CTA FFT engine for the 2LPT pass kernels (sm_103a).
//
// A pencil of N complex points is owned by TPP = N / RMAX threads; thread t of
// the pencil holds RMAX values in registers.  The first and the last stage use
// the same radix R0, so the input of the first stage and the output of the last
// stage sit at the same element n = elem(t, j) = t + (j / R0) TPP + (j mod R0) N/R0
// (= t + j TPP when R0 = RMAX): prologue/epilogue code sees natural-order
// indices without an extra shared memory round trip.  Stages follow the Stockham autosort formulation (radix-R
// butterflies on inputs b + r N/R, twiddle W_{Ns R}^{r (b mod Ns)}, outputs at
// (b / Ns) Ns R + b mod Ns + r Ns) with one shared-memory exchange between
// consecutive stages.  Twiddles come from a table exp(-2 pi i m / N) computed in
// FP64 on the host and rounded once to FP32.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lpt2 {

// ---------------------------------------------------------------- complex ops
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 mul_i(float2 a) { return make_float2(-a.y, a.x); }    // i a
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }   // -i a

// ------------------------------------------------------------ radix schedules
// Radix sequences with the same radix first and last (so that stage-0 input and
// last-stage output share one element pattern); every radix divides RMAX.
template <int N> struct Cfg;
template <> struct Cfg<96>   { static constexpr int NS = 3, RMAX = 12; static __host__ __device__ constexpr int rad(int s) { return s == 1 ? 6 : 4; } };
template <> struct Cfg<192>  { static constexpr int NS = 3, RMAX = 12; static __host__ __device__ constexpr int rad(int s) { return s == 1 ? 12 : 4; } };
template <> struct Cfg<16>   { static constexpr int NS = 2, RMAX = 4;  static __host__ __device__ constexpr int rad(int s) { return 4; } };
template <> struct Cfg<32>   { static constexpr int NS = 3, RMAX = 4;  static __host__ __device__ constexpr int rad(int s) { return s == 1 ? 2 : 4; } };
template <> struct Cfg<64>   { static constexpr int NS = 2, RMAX = 8;  static __host__ __device__ constexpr int rad(int s) { return 8; } };
template <> struct Cfg<128>  { static constexpr int NS = 3, RMAX = 8;  static __host__ __device__ constexpr int rad(int s) { return s == 1 ? 2 : 8; } };
template <> struct Cfg<256>  { static constexpr int NS = 2, RMAX = 16; static __host__ __device__ constexpr int rad(int s) { return 16; } };
#ifndef LPT2_R512
#define LPT2_R512 16   // N = 512: radix 16-2-16 (16 values per thread) or 8-8-8 (8 values)
#endif
template <> struct Cfg<512>  { static constexpr int NS = 3, RMAX = LPT2_R512;
  static __host__ __device__ constexpr int rad(int s) { return LPT2_R512 == 8 ? 8 : (s == 1 ? 2 : 16); } };
template <> struct Cfg<1024> { static constexpr int NS = 3, RMAX = 16; static __host__ __device__ constexpr int rad(int s) { return s == 1 ? 4 : 16; } };

// element index held in register slot j by lane t (first-stage input = last-stage output)
template <int N> __host__ __device__ __forceinline__ constexpr int elem(int t, int j) {
  constexpr int R0 = Cfg<N>::rad(0), TPP = N / Cfg<N>::RMAX;
  return t + (j / R0) * TPP + (j % R0) * (N / R0);
}

// i mod N for i in [0, 2N) (periodic neighbour index)
template <int N> __host__ __device__ __forceinline__ constexpr int wrap_idx(int i) {
  return ((N & (N - 1)) == 0) ? (i & (N - 1)) : (i >= N ? i - N : i);
}

template <int N> __host__ __device__ constexpr int ns_before(int s) {
  int p = 1;
  for (int i = 0; i < s; ++i) p *= Cfg<N>::rad(i);
  return p;
}

// ------------------------------------------------------- in-register DFTs
// Forward: X[k] = sum_n x[n] exp(-2 pi i n k / R); INV flips the sign.
// Roots of unity of order 48 (covers R = 2, 3, 4, 6, 8, 12, 16): cos / sin of
// 2 pi j / 48, from cos(j * 7.5 deg) for j = 0..12.
__device__ __forceinline__ float2 root48(int j, bool inv) {
  // j in [0, 48); value exp(-+ 2 pi i j / 48)
  const float c[13] = {1.0f, 0.99144486137381038f, 0.96592582628906831f, 0.92387953251128674f,
                       0.86602540378443865f, 0.79335334029123517f, 0.70710678118654752f,
                       0.60876142900872066f, 0.5f, 0.38268343236508977f, 0.25881904510252074f,
                       0.13052619222005159f, 0.0f};
  float cs, sn;
  const int q = j % 12, quad = j / 12;
  const float cq = c[q], sq = c[12 - q];
  switch (quad) {
    case 0: cs = cq; sn = sq; break;
    case 1: cs = -sq; sn = cq; break;
    case 2: cs = -cq; sn = -sq; break;
    default: cs = sq; sn = -cq; break;
  }
  return make_float2(cs, inv ? sn : -sn);
}

template <int R, bool INV> struct Dft;

template <bool INV> struct Dft<1, INV> { static __device__ __forceinline__ void run(float2*) {} };

template <bool INV> struct Dft<3, INV> {
  static __device__ __forceinline__ void run(float2* v) {
    const float h = 0.86602540378443865f;   // sin(60 deg)
    const float2 a = v[0], s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    const float2 t = make_float2(a.x - 0.5f * s.x, a.y - 0.5f * s.y);
    const float2 u = INV ? cscale(mul_i(d), h) : cscale(mul_mi(d), h);
    v[0] = cadd(a, s);
    v[1] = cadd(t, u);
    v[2] = csub(t, u);
  }
};

template <bool INV> struct Dft<2, INV> {
  static __device__ __forceinline__ void run(float2* v) {
    const float2 a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  }
};

template <int R, bool INV> struct Dft {   // even R: split into even and odd halves
  static_assert(R % 2 == 0 && 48 % R == 0, "radix must be 2, 4, 6, 8, 12 or 16 here");
  static __device__ __forceinline__ void run(float2* v) {
    float2 e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) { e[i] = v[2 * i]; o[i] = v[2 * i + 1]; }
    Dft<R / 2, INV>::run(e);
    Dft<R / 2, INV>::run(o);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      const int j = k * (48 / R);   // exponent in units of 2 pi / 48
      float2 t;
      if (j == 0) t = o[k];
      else if (j == 12) t = INV ? mul_i(o[k]) : mul_mi(o[k]);
      else t = cmul(o[k], root48(j, INV));
      v[k] = cadd(e[k], t);
      v[k + R / 2] = csub(e[k], t);
    }
  }
};

// --------------------------------------------------------- shared accessors
// Z layout: one pencil per row of N + N/16 complex (one pad slot per 16).  The row is
// private to its pencil; when the pencil's threads lie in one warp (WARP), the exchange
// between stages needs only a warp barrier.
template <bool WARP = false> struct SmemRowT {
  float2* base;
  __device__ __forceinline__ void st(int n, float2 v) const { base[n + (n >> 4)] = v; }
  __device__ __forceinline__ float2 ld(int n) const { return base[n + (n >> 4)]; }
  __device__ __forceinline__ void sync() const {
    if (WARP) __syncwarp();
    else __syncthreads();
  }
  static __host__ __device__ constexpr int words(int n) { return n + n / 16; }
};
using SmemRow = SmemRowT<false>;
// z-pass pencils of N points lie in one warp when N / RMAX <= 32 threads hold one
template <int N> inline constexpr bool kRowWarp = (N / Cfg<N>::RMAX) <= 32;
// Column layout: W pencils interleaved, element (n, w) at n * W + w (a pencil spans warps).
template <int W> struct SmemCol {
  float2* base;   // already offset by w
  __device__ __forceinline__ void st(int n, float2 v) const { base[n * W] = v; }
  __device__ __forceinline__ float2 ld(int n) const { return base[n * W]; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// ------------------------------------------------------------ stage engine
// Runs all stages on v (in: x[t + r TPP], out: X[t + r TPP]).  Every thread of
// the CTA (of the warp, for a warp-private row layout) must call this the same number
// of times (it contains the layout's barriers).
template <int N, bool INV, int S, class SM>
__device__ __forceinline__ void fft_stages(float2 (&v)[Cfg<N>::RMAX], int t, const SM& sm,
                                           const float2* __restrict__ tw) {
  constexpr int RMAX = Cfg<N>::RMAX;
  constexpr int TPP = N / RMAX;
  constexpr int R = Cfg<N>::rad(S);
  constexpr int NS = ns_before<N>(S);
  constexpr int NB = RMAX / R;
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int b = t + q * TPP;
    if (S > 0) {
      const int j = b % NS;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = tw[(r * j) * (N / (NS * R))];
        if (INV) w.y = -w.y;
        v[q * R + r] = cmul(v[q * R + r], w);
      }
    }
    Dft<R, INV>::run(&v[q * R]);
  }
  if constexpr (S + 1 < Cfg<N>::NS) {
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int b = t + q * TPP;
      const int d = (b / NS) * NS * R + (b % NS);
#pragma unroll
      for (int r = 0; r < R; ++r) sm.st(d + r * NS, v[q * R + r]);
    }
    sm.sync();
    constexpr int R2 = Cfg<N>::rad(S + 1);
#pragma unroll
    for (int q = 0; q < RMAX / R2; ++q) {
      const int b = t + q * TPP;
#pragma unroll
      for (int r = 0; r < R2; ++r) v[q * R2 + r] = sm.ld(b + r * (N / R2));
    }
    sm.sync();
    fft_stages<N, INV, S + 1, SM>(v, t, sm, tw);
  }
}

template <int N, bool INV, class SM>
__device__ __forceinline__ void fft(float2 (&v)[Cfg<N>::RMAX], int t, const SM& sm,
                                    const float2* __restrict__ tw) {
  fft_stages<N, INV, 0, SM>(v, t, sm, tw);
}

// Copy the N-entry twiddle table to shared memory (all threads participate).
__device__ __forceinline__ void load_twiddles(float2* s_tw, const float2* __restrict__ g_tw, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) s_tw[i] = g_tw[i];
}

// ---------------------------------------------------------------- k helpers
__device__ __forceinline__ int mode_of(int i, int n) { return i < (n >> 1) ? i : i - n; }

}  // namespace lpt2
