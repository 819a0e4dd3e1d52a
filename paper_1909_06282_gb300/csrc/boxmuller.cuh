// Box-Muller transform of two Philox words, evaluated in float-float arithmetic so
// that the FP32 Gaussian is the correctly rounded value of
//   g_even = sqrt(-2 ln u0) cos(2 pi u1),   g_odd = sqrt(-2 ln u0) sin(2 pi u1),
// u_j = ((x_j >> 8) + 1) 2^-24, except where the float-float value (relative error
// below about 2^-44) falls within that distance of a rounding midpoint.
//
// A float-float number is an unevaluated sum h + l of two floats.  Sums and products
// use the error-free transforms of Dekker (1971) and Knuth (TAOCP vol. 2): two_sum,
// fast_two_sum and two_prod (the rounding error of a product from one FMA).  Every
// operation is written with the _rn intrinsics, which the compiler never contracts
// into FMAs, so each transform is exact as written.
//
//  ln u0  Table-driven logarithm after Tang (1990, ACM TOMS 16, "Table-driven
//         implementation of the logarithm function in IEEE floating-point arithmetic"):
//         u0 = 2^e f with f in [sqrt(1/2), sqrt(2)], c = a float near 1/F for the table
//         point F = 1 + j/128 nearest to f, t = f c - 1 (exact as a float-float,
//         |t| < 2^-7.5), ln u0 = e ln 2 - ln c + ln(1 + t), the last term by its Taylor
//         series (t and t^2/2 in float-float, t^3 (1/3 - t/4 + ...) in float).
//  sqrt   One Newton correction of the float square root with the exact residual.
//  sincos Quadrant and octant symmetry reduce 2 pi u1 exactly to phi in [0, pi/4];
//         phi = a_j + delta with a table point a_j = 2 pi j / 4096 and 0 <= delta <
//         2 pi / 4096; angle addition with the table's cos a_j, sin a_j (float-float)
//         and the Taylor series of cos delta, sin delta.
//
// The table (kBmTableLen float4, built in FP64 on the host by lpt2::bm_table):
//   [0, 513)          (cos a_j hi, lo, sin a_j hi, lo), a_j = 2 pi j / 4096, j = 0..512
//   [513, 604)        (c_j, -ln c_j hi, lo, 0), c_j = float(1 / (1 + j/128)), j = -37..53
//   604               (2 pi hi, lo, ln 2 hi, lo)
#pragma once
#include <stdint.h>

namespace lpt2 {

constexpr int kBmSinCos = 513;
constexpr int kBmLogLo = -37, kBmLogHi = 53;
constexpr int kBmLog0 = kBmSinCos;                           // entry of j = kBmLogLo
constexpr int kBmConst = kBmSinCos + (kBmLogHi - kBmLogLo + 1);
constexpr int kBmTableLen = kBmConst + 1;

// Fills the table on the host (FP64 values split into float pairs).
void bm_table(float4* t);

struct ffl {   // float-float value h + l
  float h, l;
};

__device__ __forceinline__ ffl ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ ffl ff_fast_two_sum(float a, float b) {   // |a| >= |b| or a = 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ffl ff_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ ffl ff_mul(ffl a, ffl b) {
  const ffl p = ff_two_prod(a.h, b.h);
  const float t = __fmaf_rn(a.h, b.l, __fmul_rn(a.l, b.h));
  return ff_fast_two_sum(p.h, __fadd_rn(p.l, t));
}
__device__ __forceinline__ ffl ff_add(ffl a, ffl b) {
  const ffl s = ff_two_sum(a.h, b.h);
  return ff_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ ffl ff_neg(ffl a) { return {-a.h, -a.l}; }

// ln(m 2^-24) for m in [1, 2^24], as a float-float.
__device__ __forceinline__ ffl bm_log_u(uint32_t m, const float4* tab) {
  const float fm = __uint2float_rn(m);                            // exact: m <= 2^24
  const int b = (int)((__float_as_uint(fm) >> 23) & 0xff) - 126;   // bit length of m, 1..25
  float f = __uint_as_float((__float_as_uint(fm) & 0x807fffffu) | 0x3f800000u);   // m / 2^(b-1)
  int e = b - 25;
  if (f > 1.41421353816986083984375f) {   // the float just below sqrt 2
    f = __fmul_rn(f, 0.5f);
    e += 1;
  }
  const int j = __float2int_rn(__fmul_rn(__fsub_rn(f, 1.0f), 128.0f));   // f - 1 is exact
  const float4 L = tab[kBmLog0 + (j - kBmLogLo)];                  // c, -ln c (hi, lo)
  const ffl pc = ff_two_prod(f, L.x);
  const ffl t = ff_two_sum(__fsub_rn(pc.h, 1.0f), pc.l);                 // pc.h - 1 is exact
  // ln(1 + t) = t - t^2/2 + t^3 (1/3 - t/4 + t^2/5 - t^3/6 + t^4/7)
  ffl t2 = ff_two_prod(t.h, t.h);
  t2.l = __fmaf_rn(__fmul_rn(2.0f, t.h), t.l, t2.l);
  float poly = __fmaf_rn(t.h, -1.0f / 7.0f, 1.0f / 6.0f);
  poly = __fmaf_rn(t.h, -poly, 0.2f);
  poly = __fmaf_rn(t.h, -poly, 0.25f);
  poly = __fmaf_rn(t.h, -poly, 1.0f / 3.0f);
  const float cube = __fmul_rn(__fmul_rn(t.h, t2.h), poly);
  ffl l1 = ff_two_sum(t.h, __fmul_rn(-0.5f, t2.h));
  l1 = ff_fast_two_sum(l1.h, __fadd_rn(l1.l, __fadd_rn(__fmaf_rn(-0.5f, t2.l, t.l), cube)));
  const float4 C = tab[kBmConst];                                  // 2 pi, ln 2
  ffl el = ff_two_prod((float)e, C.z);
  el.l = __fmaf_rn((float)e, C.w, el.l);
  return ff_add(ff_add(el, ffl{L.y, L.z}), l1);
}

// (cos, sin)(2 pi m 2^-24) for m in [1, 2^24], as float-floats.
__device__ __forceinline__ void bm_sincos_u(uint32_t m, const float4* tab, ffl& cs, ffl& sn) {
  m &= 0xffffffu;                          // 2^24 -> 0 (angle 2 pi)
  const uint32_t q = m >> 22;              // quadrant
  uint32_t r = m & 0x3fffffu;
  const bool swap = r > (1u << 21);        // second octant of the quadrant: pi/2 - phi
  if (swap) r = (1u << 22) - r;
  const uint32_t j = r >> 12, rem = r & 0xfffu;
  const float4 C = tab[kBmConst];
  const float x = __fmul_rn(__uint2float_rn(rem), 5.9604644775390625e-8f);   // rem 2^-24, exact
  ffl d = ff_two_prod(C.x, x);                                               // delta = 2 pi x
  d.l = __fmaf_rn(C.y, x, d.l);
  const float d2h = __fmul_rn(d.h, d.h);
  // sin delta = delta - delta^3/6 + delta^5/120
  const float s3 = __fmul_rn(__fmul_rn(d.h, d2h), __fmaf_rn(d2h, 1.0f / 120.0f, -1.0f / 6.0f));
  const ffl sd = ff_fast_two_sum(d.h, __fadd_rn(d.l, s3));
  // cos delta = 1 - delta^2/2 + delta^4/24
  ffl dd = ff_two_prod(d.h, d.h);
  dd.l = __fmaf_rn(__fmul_rn(2.0f, d.h), d.l, dd.l);
  ffl cd = ff_fast_two_sum(1.0f, __fmul_rn(-0.5f, dd.h));
  cd.l = __fadd_rn(cd.l, __fmaf_rn(__fmul_rn(dd.h, dd.h), 1.0f / 24.0f, __fmul_rn(-0.5f, dd.l)));
  const float4 T = tab[j];                                          // cos a_j, sin a_j
  const ffl ca{T.x, T.y}, sa{T.z, T.w};
  const ffl sphi = ff_add(ff_mul(sa, cd), ff_mul(ca, sd));
  const ffl cphi = ff_add(ff_mul(ca, cd), ff_neg(ff_mul(sa, sd)));
  const ffl c1 = swap ? sphi : cphi, s1 = swap ? cphi : sphi;   // angle of the quadrant
  switch (q) {
    case 0: cs = c1; sn = s1; break;
    case 1: cs = ff_neg(s1); sn = c1; break;
    case 2: cs = ff_neg(c1); sn = ff_neg(s1); break;
    default: cs = s1; sn = ff_neg(c1); break;
  }
}

// Copies the table from global to shared memory (all threads of the CTA take part; the
// caller synchronises before the first use).  The lookups of a warp hit random entries,
// which shared memory serves with far fewer transactions than the L1 cache.
__device__ __forceinline__ void bm_load_table(float4* s_tab, const float4* __restrict__ g_tab) {
  for (int i = threadIdx.x; i < kBmTableLen; i += blockDim.x) s_tab[i] = __ldg(g_tab + i);
}

// (g_even, g_odd) of the Box-Muller transform of Philox words x0, x1, rounded once to FP32;
// tab is the table in shared (or global) memory.
__device__ __forceinline__ float2 bm_pair(uint32_t x0, uint32_t x1, const float4* tab) {
  const ffl lu = bm_log_u((x0 >> 8) + 1u, tab);
  const float lh = __fmul_rn(-2.0f, lu.h), ll = __fmul_rn(-2.0f, lu.l);   // -2 ln u0 >= 0
  ffl r{0.0f, 0.0f};
  if (lh > 0.0f) {
    const float r0 = __fsqrt_rn(lh);
    const ffl sq = ff_two_prod(r0, r0);
    const float d = __fadd_rn(__fsub_rn(__fsub_rn(lh, sq.h), sq.l), ll);
    r = {r0, __fmul_rn(d, __fdiv_rn(0.5f, r0))};
  }
  ffl cs, sn;
  bm_sincos_u((x1 >> 8) + 1u, tab, cs, sn);
  const ffl ge = ff_mul(r, cs), go = ff_mul(r, sn);
  return make_float2(ge.h, go.h);   // ff_mul normalises: h is the rounded sum
}

}  // namespace lpt2
