// Pass kernels of the 2LPT pipeline, templated on the grid side N.
//
// Spectral arrays are half spectra float2[N][N][N/2] (kx, ky, kz; kz fastest,
// the kz = N/2 plane dropped because the method zeroes every Nyquist plane).
// A 3-D transform is three passes: z (contiguous pencils, real <-> half
// complex, two real rows packed as one complex pencil), y and x (strided
// pencils, W consecutive kz handled per CTA so every load/store is a 128-byte
// row segment).  The k-space multiplications of the method are fused into the
// x pass, which sees full (kx, ky, kz) and runs the forward transform, the
// multiplier and the first inverse transform back to back in registers.
#pragma once
#include <algorithm>

#include "fft_core.cuh"
#include "passes.h"
#include "philox.cuh"
#include "tma.cuh"

namespace lpt2 {

#ifndef LPT2_ZTHREADS
#define LPT2_ZTHREADS 256   // threads per z-pass CTA (pencil pairs per CTA = this / threads per pencil)
#endif
#ifndef LPT2_Z_MINB
#define LPT2_Z_MINB (LPT2_ZTHREADS >= 512 ? 1 : 512 / LPT2_ZTHREADS)   // resident z-pass CTAs per SM asked: 128-register cap
#endif
#ifndef LPT2_WSMALL
#define LPT2_WSMALL 16  // pencils per y/x CTA for 32 <= N <= 256
#endif
#ifndef LPT2_W512
#define LPT2_W512 8     // pencils per y/x CTA at N = 512 (measured: 8 beats 16 and 32)
#endif

template <int N> struct PassCfg {
  static constexpr int RMAX = Cfg<N>::RMAX;
  static constexpr int TPP = N / RMAX;
  static constexpr int H = N / 2;
  static constexpr int ZP = (LPT2_ZTHREADS / TPP) < 1 ? 1 : (LPT2_ZTHREADS / TPP);   // pencil pairs per z CTA
  static constexpr int ZT = ZP * TPP;                                 // z CTA threads
  static constexpr int W = (N <= 16) ? 8 : (N >= 1024 ? 8 : (N == 512 ? LPT2_W512 : LPT2_WSMALL));   // pencils per y/x CTA
  static constexpr int XT = TPP * W;                                  // y/x CTA threads
  static constexpr int ZSMEM = (N + ZP * SmemRow::words(N)) * 8;
  static constexpr int XSMEM = (N + N * W) * 8;
  // resident x-pass CTAs per SM asked of the compiler: caps a thread at 128 registers for
  // every CTA size (at 256 threads the multi-output modes would otherwise take 184 and
  // halve the warps per SM)
  static constexpr int XMINB = XT >= 512 ? 1 : 512 / XT;
};

// y passes: their own pencils per CTA (the y tile rows are 2 KB apart, the x tile rows a
// whole (ky, kz) plane apart, and the two passes hold different working sets).  WY = 0 is
// the build default; the launcher also has WY = 8 and 16 compiled, which a plan's tile
// schedule (Geo::ytile) selects per grid-size group.
#ifndef LPT2_WY512
#define LPT2_WY512 LPT2_W512
#endif
template <int N, int WY = 0> struct YCfg {
  static constexpr int RMAX = Cfg<N>::RMAX;
  static constexpr int TPP = N / RMAX;
  static constexpr int H = N / 2;
  static constexpr int W = WY ? WY : (N == 512 ? LPT2_WY512 : PassCfg<N>::W);
  static constexpr int XT = TPP * W;
  static constexpr int XSMEM = (N + N * W) * 8;
  static_assert(H % W == 0, "a CTA's kz block must tile the half spectrum");
};

// (i k)^m v for m = 0, 1, 2
__device__ __forceinline__ float2 deriv(float2 v, float k, int m) {
  if (m == 0) return v;
  if (m == 1) return cscale(mul_i(v), k);
  return cscale(v, -k * k);
}

// conj((i k)^m) v for m = 0, 1, 2 (the transpose of deriv)
__device__ __forceinline__ float2 dconj(float2 v, float k, int m) {
  if (m == 0) return v;
  if (m == 1) return cscale(mul_mi(v), k);
  return cscale(v, -k * k);
}
// v + conj((i k)^m) u with every product and sum rounded on its own (the _rn intrinsics are
// never contracted), so that the kernels that accumulate the x-order groups of the adjoint
// (global-load and bulk-tensor tile paths) give the same bits
__device__ __forceinline__ float2 acc_dconj(float2 v, float2 u, float k, int m) {
  float2 w = u;
  if (m == 1) {
    w = make_float2(__fmul_rn(u.y, k), __fmul_rn(-u.x, k));
  } else if (m == 2) {
    const float kk = -__fmul_rn(k, k);
    w = make_float2(__fmul_rn(u.x, kk), __fmul_rn(u.y, kk));
  }
  return make_float2(__fadd_rn(v.x, w.x), __fadd_rn(v.y, w.y));
}

// ===================================================================== z pass
// Thread layout: tid = p * TPP + t (pencil pair p, lane t within the pencil).

template <int N, class SM>
__device__ __forceinline__ void z_store_pair(const float2 (&v)[Cfg<N>::RMAX], int t, const SM& sm,
                                             float2* __restrict__ outa, float2* __restrict__ outb) {
  // v holds Z = FFT(fa + i fb) at n = elem(t, r). Split into the two real spectra;
  // outputs k = t + r TPP, r < RMAX/2, cover [0, N/2) once.
  constexpr int RMAX = Cfg<N>::RMAX, TPP = N / RMAX, H = N / 2;
#pragma unroll
  for (int r = 0; r < RMAX; ++r) sm.st(elem<N>(t, r), v[r]);
  sm.sync();
#pragma unroll
  for (int r = 0; r < RMAX / 2; ++r) {
    const int k = t + r * TPP;                      // < H
    const float2 zk = sm.ld(k);
    const float2 zm = cconj(sm.ld(k == 0 ? 0 : N - k));
    outa[k] = cscale(cadd(zk, zm), 0.5f);
    outb[k] = cscale(mul_mi(csub(zk, zm)), 0.5f);
  }
  (void)H;
}

// As z_store_pair, each output multiplied by conj((i k_z)^m) (transpose of a z derivative).
template <int N, class SM>
__device__ __forceinline__ void z_store_pair_d(const float2 (&v)[Cfg<N>::RMAX], int t, const SM& sm,
                                               float2* __restrict__ outa, float2* __restrict__ outb,
                                               float kf, int ma, int mb) {
  constexpr int RMAX = Cfg<N>::RMAX, TPP = N / RMAX;
#pragma unroll
  for (int r = 0; r < RMAX; ++r) sm.st(elem<N>(t, r), v[r]);
  sm.sync();
#pragma unroll
  for (int r = 0; r < RMAX / 2; ++r) {
    const int k = t + r * TPP;
    const float2 zk = sm.ld(k);
    const float2 zm = cconj(sm.ld(k == 0 ? 0 : N - k));
    const float kz = kf * (float)k;
    outa[k] = dconj(cscale(cadd(zk, zm), 0.5f), kz, ma);
    outb[k] = dconj(cscale(mul_mi(csub(zk, zm)), 0.5f), kz, mb);
  }
}

// Z value at element n of the Hermitian extension of two half-spectrum rows,
// each multiplied by (i k_z)^m first: Z = A + i B.
template <int N>
__device__ __forceinline__ float2 z_assemble(const float2* __restrict__ ra, const float2* __restrict__ rb,
                                             int n, float kf, int ma, int mb) {
  constexpr int H = N / 2;
  if (n == H) return make_float2(0.f, 0.f);
  const bool lo = n < H;
  const int m = lo ? n : N - n;
  const float kz = kf * (float)m;
  float2 A = deriv(__ldg(ra + m), kz, ma);
  float2 B = deriv(__ldg(rb + m), kz, mb);
  if (!lo) { A = cconj(A); B = cconj(B); }
  return make_float2(A.x - B.y, A.y + B.x);
}

// shared memory of the forward z pass: twiddles and exchange rows, then (noise source)
// the Box-Muller table at a 16-byte boundary
template <int N> constexpr int zr2c_tab_off() { return (PassCfg<N>::ZSMEM + 15) / 16 * 16; }
template <int N, int SRC> constexpr int zr2c_smem() {
  return SRC == Z_NOISE ? zr2c_tab_off<N>() + kBmTableLen * 16 : PassCfg<N>::ZSMEM;
}

#ifndef LPT2_ZNOISE_MINB
#define LPT2_ZNOISE_MINB 3   // resident noise-pass CTAs per SM asked: 80 registers (it is issue bound)
#endif
template <int N, int SRC>
__global__ void __launch_bounds__(PassCfg<N>::ZT, SRC == Z_NOISE ? LPT2_ZNOISE_MINB : LPT2_Z_MINB)
    k_z_r2c(ZR2CArgs a) {
  using C = PassCfg<N>;
  extern __shared__ __align__(16) float2 smem[];
  float2* s_tw = smem;
  float4* s_bm = reinterpret_cast<float4*>(reinterpret_cast<char*>(smem) + zr2c_tab_off<N>());
  load_twiddles(s_tw, a.tw, N);
  if (SRC == Z_NOISE) {
    bm_load_table(s_bm, a.bm);
    __syncthreads();
  }
  const int p = threadIdx.x / C::TPP, t = threadIdx.x % C::TPP;
  const SmemRowT<kRowWarp<N>> sm{smem + N + p * SmemRow::words(N)};
  const int pair = blockIdx.x * C::ZP + p;
  const int rowa = 2 * pair, rowb = rowa + 1;
  const size_t n3 = (size_t)N * N * N;                 // instance blockIdx.z of the batch
  if (SRC != Z_NOISE) a.in += blockIdx.z * n3;
  a.out += blockIdx.z * (n3 / 2);
  if (SRC == Z_NOISE && a.seeds) {
    const uint64_t sd = a.seeds[a.g.inst0 + blockIdx.z];
    a.seed_lo = (uint32_t)sd;
    a.seed_hi = (uint32_t)(sd >> 32);
  }
  float2 v[C::RMAX];
#pragma unroll
  for (int r = 0; r < C::RMAX; ++r) {
    const int n = elem<N>(t, r);
    float fa, fb;
    if (SRC == Z_NOISE) {   // rows (x, y) and (x, y+1), y even: one Box-Muller pair per z
      const float2 g2 = philox_gauss2((uint64_t)rowa * N + n, a.seed_lo, a.seed_hi, s_bm);
      fa = g2.x;
      fb = g2.y;
    } else {
      fa = __ldg(a.in + (size_t)rowa * N + n);
      fb = __ldg(a.in + (size_t)rowb * N + n);
      if (SRC == Z_DENSITY) { fa -= 1.0f; fb -= 1.0f; }
    }
    v[r] = make_float2(fa, fb);
  }
  __syncthreads();   // twiddles visible
  fft<N, false>(v, t, sm, s_tw);
  z_store_pair<N>(v, t, sm, a.out + (size_t)rowa * C::H, a.out + (size_t)rowb * C::H);
}

template <int N>
__global__ void __launch_bounds__(PassCfg<N>::ZT, LPT2_Z_MINB) k_z_c2r(ZC2RArgs a) {
  using C = PassCfg<N>;
  extern __shared__ float2 smem[];
  float2* s_tw = smem;
  load_twiddles(s_tw, a.tw, N);
  const int p = threadIdx.x / C::TPP, t = threadIdx.x % C::TPP;
  const SmemRowT<kRowWarp<N>> sm{smem + N + p * SmemRow::words(N)};
  const int pair = blockIdx.x * C::ZP + p;
  const int rowa = 2 * pair, rowb = rowa + 1;
  const size_t n3 = (size_t)N * N * N;                 // instance blockIdx.z of the batch
  a.in += blockIdx.z * (n3 / 2);
  a.out += blockIdx.z * n3;
  if (a.add_in) a.add_in += blockIdx.z * n3;
  const float2* ra = a.in + (size_t)rowa * C::H;
  const float2* rb = a.in + (size_t)rowb * C::H;
  float2 v[C::RMAX];
#pragma unroll
  for (int r = 0; r < C::RMAX; ++r) v[r] = z_assemble<N>(ra, rb, elem<N>(t, r), 0.f, 0, 0);
  __syncthreads();
  fft<N, true>(v, t, sm, s_tw);
#pragma unroll
  for (int r = 0; r < C::RMAX; ++r) {
    const int n = elem<N>(t, r);
    const size_t ea = (size_t)rowa * N + n, eb = (size_t)rowb * N + n;
    a.out[ea] = a.add_in ? v[r].x + __ldg(a.add_in + ea) : v[r].x;
    a.out[eb] = a.add_in ? v[r].y + __ldg(a.add_in + eb) : v[r].y;
  }
}

// Six phi_ij -> S = sum_{i<j} (phi_ii phi_jj - phi_ij^2)  (Eq. second-ini) -> forward z.
//
// A CTA owns ROWS = 2 ZP consecutive real rows (x, y) of every field.  The rows of
// one field are contiguous in the half-spectrum layout, so each field's tile is one
// bulk copy into a ring of STAGES shared-memory buffers: the copy of field f +
// STAGES is in flight while field f is transformed.  Rows 2p and 2p + 1 of a field
// are packed as one complex pencil (Z = A + i B), so its inverse transform gives the
// field on both rows; the source term accumulates per row in registers:
//   S = phi_xx phi_yy + (phi_xx + phi_yy) phi_zz - phi_xy^2 - phi_xz^2 - phi_yz^2.
#ifndef LPT2_ZS_STAGES
#define LPT2_ZS_STAGES 2
#endif

template <int N> struct ZSrcCfg {
  using C = PassCfg<N>;
  static constexpr int STAGES = LPT2_ZS_STAGES;
  static constexpr int ROWS = 2 * C::ZP;                     // real rows per CTA
  static constexpr int STAGE_F2 = ROWS * C::H;               // one field's tile (float2)
  static constexpr unsigned STAGE_BYTES = STAGE_F2 * 8u;
  static constexpr int BAR_OFF = STAGES * STAGE_BYTES;       // mbarriers after the ring
  static constexpr int SMEM = BAR_OFF + 64 + C::ZSMEM;       // + twiddles and exchange rows
  static_assert(STAGES >= 1 && STAGES <= 6 && STAGES * 8 <= 64, "stage count");
  static_assert(STAGE_BYTES % 16 == 0 && (C::H * 8) % 16 == 0, "bulk copies need 16-byte multiples");
};

// Z value at element n of the Hermitian extension of half rows ra, rb (shared
// memory), both multiplied by (i k_z)^m first: Z = A + i B.
template <int N>
__device__ __forceinline__ float2 z_assemble_smem(const float2* ra, const float2* rb, int n, float kf, int m) {
  constexpr int H = N / 2;
  if (n == H) return make_float2(0.f, 0.f);
  const bool lo = n < H;
  const int j = lo ? n : N - n;
  const float kz = kf * (float)j;
  float2 A = deriv(ra[j], kz, m);
  float2 B = deriv(rb[j], kz, m);
  if (!lo) { A = cconj(A); B = cconj(B); }
  return make_float2(A.x - B.y, A.y + B.x);
}

template <int N>
__global__ void __launch_bounds__(PassCfg<N>::ZT, LPT2_Z_MINB) k_z_source(ZSourceArgs a) {
  using C = PassCfg<N>;
  using Q = ZSrcCfg<N>;
  extern __shared__ __align__(128) unsigned char zs_raw[];
  float2* ring = reinterpret_cast<float2*>(zs_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(zs_raw + Q::BAR_OFF);
  float2* s_tw = reinterpret_cast<float2*>(zs_raw + Q::BAR_OFF + 64);
  __shared__ int s_fail;
  const int p = threadIdx.x / C::TPP, t = threadIdx.x % C::TPP;
  const SmemRowT<kRowWarp<N>> sm{s_tw + N + p * SmemRow::words(N)};
  const size_t zoff = blockIdx.z * ((size_t)N * N * N / 2);   // instance blockIdx.z
  const size_t tile = (size_t)blockIdx.x * Q::STAGE_F2;        // first float2 of the tile in a field
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < Q::STAGES; ++s) mbar_init(&bar[s], 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int f = 0; f < Q::STAGES; ++f) {
      mbar_expect_tx(&bar[f], Q::STAGE_BYTES);
      bulk_load(ring + f * Q::STAGE_F2, a.in[f] + zoff + tile, Q::STAGE_BYTES, &bar[f]);
    }
  }
  load_twiddles(s_tw, a.tw, N);
  // field f of the ring into v, then the copy of field f + STAGES; false if a wait ran out
  // (the CTA has then drained its copies and reported, and must return)
  auto fetch = [&](int f, float2 (&v)[C::RMAX]) -> bool {
    const int s = f % Q::STAGES;
    const bool ok = mbar_wait(&bar[s], (f / Q::STAGES) & 1, a.g.wait);
    if (!ok) s_fail = 1;
    const float2* ra = ring + s * Q::STAGE_F2 + (2 * p) * C::H;
    const int m = a.ord[f];
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r)
      v[r] = ok ? z_assemble_smem<N>(ra, ra + C::H, elem<N>(t, r), a.g.kf, m) : make_float2(0.f, 0.f);
    __syncthreads();   // stage s consumed by every thread (and, at f = 0, twiddles visible)
    if (s_fail) {      // a copy never landed: wait (bounded) for the copies in flight, report
      if (threadIdx.x == 0) {
        for (int g = f; g < 6 && g < f + Q::STAGES; ++g) mbar_wait(&bar[g % Q::STAGES], (g / Q::STAGES) & 1);
        report_device_error(a.g.err, LPT2_DEV_ETIMEOUT_ZSOURCE);
      }
      return false;
    }
    if (threadIdx.x == 0 && f + Q::STAGES < 6) {
      mbar_expect_tx(&bar[s], Q::STAGE_BYTES);
      bulk_load(ring + s * Q::STAGE_F2, a.in[f + Q::STAGES] + zoff + tile, Q::STAGE_BYTES, &bar[s]);
    }
    return true;
  };
  float S0[C::RMAX], S1[C::RMAX], T0[C::RMAX], T1[C::RMAX];
#pragma unroll
  for (int f = 0; f < 3; ++f) {   // phi_xx, phi_yy, phi_zz
    float2 v[C::RMAX];
    if (!fetch(f, v)) return;
    fft<N, true>(v, t, sm, s_tw);
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) {
      const float e = v[r].x, g = v[r].y;   // rows 2p and 2p + 1
      if (f == 0) {
        S0[r] = e;
        S1[r] = g;
      } else if (f == 1) {
        T0[r] = S0[r] + e;
        T1[r] = S1[r] + g;
        S0[r] *= e;
        S1[r] *= g;
      } else {
        S0[r] = fmaf(T0[r], e, S0[r]);
        S1[r] = fmaf(T1[r], g, S1[r]);
      }
    }
  }
  // phi_xy, phi_xz, phi_yz: one loop body (three unrolled copies of the transform push the
  // kernel out of the instruction cache)
#pragma unroll 1
  for (int f = 3; f < 6; ++f) {
    float2 v[C::RMAX];
    if (!fetch(f, v)) return;
    fft<N, true>(v, t, sm, s_tw);
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) {
      S0[r] = fmaf(-v[r].x, v[r].x, S0[r]);
      S1[r] = fmaf(-v[r].y, v[r].y, S1[r]);
    }
  }
  float2 v[C::RMAX];
#pragma unroll
  for (int r = 0; r < C::RMAX; ++r) v[r] = make_float2(S0[r], S1[r]);
  fft<N, false>(v, t, sm, s_tw);
  float2* out = a.out + zoff + tile + (size_t)(2 * p) * C::H;
  z_store_pair<N>(v, t, sm, out, out + C::H);
}

// Periodic CIC deposit of one particle with 16-byte vector atomics where the two
// z cells of a corner row fall in one aligned group of four floats (sm_90+),
// two scalar atomics otherwise: 4 to 8 atomic instructions per particle.
template <int N>
__device__ __forceinline__ void add_zpair(float* __restrict__ rho, size_t b, int iz, int jz, float w0, float w1) {
  const int q = iz & 3;
  if (q != 3 && iz + 1 < N) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q == 0) { v.x = w0; v.y = w1; }
    else if (q == 1) { v.y = w0; v.z = w1; }
    else { v.z = w0; v.w = w1; }
    atomicAdd(reinterpret_cast<float4*>(rho + b + (iz - q)), v);
  } else {
    atomicAdd(rho + b + iz, w0);
    atomicAdd(rho + b + jz, w1);
  }
}

template <int N>
__device__ __forceinline__ void cic_deposit_vec(float* __restrict__ rho, float ux, float uy, float uz) {
  const float fx = floorf(ux), fy = floorf(uy), fz = floorf(uz);
  const float dx = ux - fx, dy = uy - fy, dz = uz - fz;
  const int ix = wrap_idx<N>((int)fx), iy = wrap_idx<N>((int)fy), iz = wrap_idx<N>((int)fz);
  const int jx = wrap_idx<N>(ix + 1), jy = wrap_idx<N>(iy + 1), jz = wrap_idx<N>(iz + 1);
  const float wx0 = 1.f - dx, wy0 = 1.f - dy, wz0 = 1.f - dz;
  float w;
  w = wx0 * wy0; add_zpair<N>(rho, ((size_t)ix * N + iy) * N, iz, jz, w * wz0, w * dz);
  w = wx0 * dy;  add_zpair<N>(rho, ((size_t)ix * N + jy) * N, iz, jz, w * wz0, w * dz);
  w = dx * wy0;  add_zpair<N>(rho, ((size_t)jx * N + iy) * N, iz, jz, w * wz0, w * dz);
  w = dx * dy;   add_zpair<N>(rho, ((size_t)jx * N + jy) * N, iz, jz, w * wz0, w * dz);
}

// wrap grid coordinate into [0, N); a value that is not finite, or a rounding stray of a
// coordinate far outside the box, goes to 0, so every cell index derived from the result
// lies in the grid whatever the input
template <int N>
__device__ __forceinline__ float wrapN(float u) {
  u = u - (float)N * floorf(u * (1.0f / N));
  u = (u >= (float)N) ? u - (float)N : u;
  return (u >= 0.0f && u < (float)N) ? u : 0.0f;
}

// Psi inputs (z order 1 -> Psi_z, 0 -> Psi_y, 0 -> Psi_x) -> particle positions
// x = q + Psi (Eq. position), periodic.  The tile and copy ring are those of
// k_z_source: a CTA owns ROWS consecutive rows of every input, one bulk copy per
// input tile, rows 2p and 2p + 1 of a field packed as one complex pencil.  The
// three components are independent, so nothing is carried from one input to the
// next except, when SPLIT (separate Psi1 / Psi2 inputs), the Psi1 part of the
// current component.
template <int N, bool SPLIT>
__global__ void __launch_bounds__(PassCfg<N>::ZT, LPT2_Z_MINB) k_z_final(ZFinalArgs a) {
  using C = PassCfg<N>;
  using Q = ZSrcCfg<N>;
  constexpr int NQ = SPLIT ? 6 : 3;   // input tiles: (Psi1, Psi2) per component, or the totals
  extern __shared__ __align__(128) unsigned char zs_raw[];
  float2* ring = reinterpret_cast<float2*>(zs_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(zs_raw + Q::BAR_OFF);
  float2* s_tw = reinterpret_cast<float2*>(zs_raw + Q::BAR_OFF + 64);
  __shared__ int s_fail;
  const int p = threadIdx.x / C::TPP, t = threadIdx.x % C::TPP;
  const SmemRowT<kRowWarp<N>> sm{s_tw + N + p * SmemRow::words(N)};
  const size_t n3 = (size_t)N * N * N;
  const size_t zs = blockIdx.z * (n3 / 2), zr = blockIdx.z * n3;   // instance blockIdx.z
  const size_t tile = (size_t)blockIdx.x * Q::STAGE_F2;
  const int row = blockIdx.x * Q::ROWS + 2 * p;                    // rows `row`, `row` + 1
  auto input = [&](int q) -> const float2* {
    return (SPLIT ? ((q & 1) ? a.b[q >> 1] : a.a[q >> 1]) : a.a[q]) + zs + tile;
  };
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int st = 0; st < Q::STAGES; ++st) mbar_init(&bar[st], 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < Q::STAGES && q < NQ; ++q) {
      mbar_expect_tx(&bar[q], Q::STAGE_BYTES);
      bulk_load(ring + q * Q::STAGE_F2, input(q), Q::STAGE_BYTES, &bar[q]);
    }
  }
  load_twiddles(s_tw, a.tw, N);
  float2 keep[C::RMAX];
#pragma unroll 1
  for (int q = 0; q < NQ; ++q) {
    const int st = q % Q::STAGES;
    const int c = SPLIT ? (q >> 1) : q;   // 0: Psi_z, 1: Psi_y, 2: Psi_x
    const bool ok = mbar_wait(&bar[st], (q / Q::STAGES) & 1, a.g.wait);
    if (!ok) s_fail = 1;
    float2 v[C::RMAX];
    const float2* ra = ring + st * Q::STAGE_F2 + (2 * p) * C::H;
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r)
      v[r] = ok ? z_assemble_smem<N>(ra, ra + C::H, elem<N>(t, r), a.g.kf, c == 0 ? 1 : 0) : make_float2(0.f, 0.f);
    __syncthreads();   // stage consumed by every thread (and, at q = 0, twiddles visible)
    if (s_fail) {
      if (threadIdx.x == 0) {
        for (int g = q; g < NQ && g < q + Q::STAGES; ++g) mbar_wait(&bar[g % Q::STAGES], (g / Q::STAGES) & 1);
        report_device_error(a.g.err, LPT2_DEV_ETIMEOUT_ZFINAL);
      }
      return;
    }
    if (threadIdx.x == 0 && q + Q::STAGES < NQ) {
      mbar_expect_tx(&bar[st], Q::STAGE_BYTES);
      bulk_load(ring + st * Q::STAGE_F2, input(q + Q::STAGES), Q::STAGE_BYTES, &bar[st]);
    }
    fft<N, true>(v, t, sm, s_tw);
    const int d = 2 - c;                  // output component: x 0, y 1, z 2
    if (SPLIT) {
      float* outp = (q & 1) ? a.psi2 : a.psi1;
      if (outp) {
        outp += 3 * zr + d * n3;
#pragma unroll
        for (int r = 0; r < C::RMAX; ++r) {
          const int iz = elem<N>(t, r);
          outp[(size_t)row * N + iz] = v[r].x;
          outp[(size_t)(row + 1) * N + iz] = v[r].y;
        }
      }
      if (!(q & 1)) {
#pragma unroll
        for (int r = 0; r < C::RMAX; ++r) keep[r] = v[r];
        continue;
      }
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) v[r] = cadd(v[r], keep[r]);
    }
    if (a.pos) {
      float* pos = a.pos + 3 * zr + d * n3;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int R = row + h;
        const float q0 = (d == 0) ? (float)(R / N) : (float)(R % N);   // Lagrangian x or y
#pragma unroll
        for (int r = 0; r < C::RMAX; ++r) {
          const int iz = elem<N>(t, r);
          const float psi = h ? v[r].y : v[r].x;
          const float u = wrapN<N>((d == 2 ? (float)iz : q0) + psi * a.g.inv_cell);
          pos[(size_t)R * N + iz] = u * a.g.cell;
        }
      }
    }
  }
}

// Transpose of the CIC deposit + positions + inverse z of k_z_final: gathers
// dL/drho at the 8 cells of each particle into dL/dx (= dL/dPsi), then forward
// z transforms with conj z-derivatives: (g_x, g_y) of each row, g_z of both rows.
template <int N>
__device__ __forceinline__ void cic_gather_grad(const float* __restrict__ g, const float* __restrict__ pos,
                                                size_t e, size_t n3, float inv_cell, float& gx, float& gy,
                                                float& gz) {
  const float ux = wrapN<N>(__ldg(pos + e) * inv_cell);
  const float uy = wrapN<N>(__ldg(pos + n3 + e) * inv_cell);
  const float uz = wrapN<N>(__ldg(pos + 2 * n3 + e) * inv_cell);
  const float fx = floorf(ux), fy = floorf(uy), fz = floorf(uz);
  const float dx = ux - fx, dy = uy - fy, dz = uz - fz;
  const int ix = wrap_idx<N>((int)fx), iy = wrap_idx<N>((int)fy), iz = wrap_idx<N>((int)fz);
  const int jx = wrap_idx<N>(ix + 1), jy = wrap_idx<N>(iy + 1), jz = wrap_idx<N>(iz + 1);
  const float wx[2] = {1.f - dx, dx}, wy[2] = {1.f - dy, dy}, wz[2] = {1.f - dz, dz};
  const int cx[2] = {ix, jx}, cy[2] = {iy, jy}, cz[2] = {iz, jz};
  float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
  for (int ox = 0; ox < 2; ++ox)
#pragma unroll
    for (int oy = 0; oy < 2; ++oy)
#pragma unroll
      for (int oz = 0; oz < 2; ++oz) {
        const float gc = __ldg(g + ((size_t)cx[ox] * N + cy[oy]) * N + cz[oz]);
        const float sx = ox ? 1.f : -1.f, sy = oy ? 1.f : -1.f, sz = oz ? 1.f : -1.f;
        ax = fmaf(gc * sx, wy[oy] * wz[oz], ax);
        ay = fmaf(gc * sy, wx[ox] * wz[oz], ay);
        az = fmaf(gc * sz, wx[ox] * wy[oy], az);
      }
  gx = ax * inv_cell;
  gy = ay * inv_cell;
  gz = az * inv_cell;
}

// Transpose of k_z_source.  g_S = dL/dS is given in real space (the inverse z of h_S,
// one z_c2r pass); the six phi_ij are recomputed (inverse z) and
//   dL/dphi_ii = g_S (Tr - phi_ii),  Tr = phi_xx + phi_yy + phi_zz,   dL/dphi_ij = -2 g_S phi_ij,
// each transformed forward with conj z-derivatives.  Tiles and copy ring as k_z_source
// (rows 2p, 2p + 1 of one field per complex pencil); the diagonal fields are read twice,
// first for Tr (kept in registers for both rows), then for their cotangents.
template <int N>
__global__ void __launch_bounds__(PassCfg<N>::ZT, LPT2_Z_MINB) k_z_adj_source(ZAdjSourceArgs a) {
  using C = PassCfg<N>;
  using Q = ZSrcCfg<N>;
  constexpr int NQ = 9;                         // xx, yy, zz (trace), then xx .. yz (cotangents)
  extern __shared__ __align__(128) unsigned char zs_raw[];
  float2* ring = reinterpret_cast<float2*>(zs_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(zs_raw + Q::BAR_OFF);
  float2* s_tw = reinterpret_cast<float2*>(zs_raw + Q::BAR_OFF + 64);
  __shared__ int s_fail;
  const int p = threadIdx.x / C::TPP, t = threadIdx.x % C::TPP;
  const SmemRowT<kRowWarp<N>> sm{s_tw + N + p * SmemRow::words(N)};
  const size_t n3 = (size_t)N * N * N;
  const size_t zs = blockIdx.z * (n3 / 2), zr = blockIdx.z * n3;   // instance blockIdx.z
  const size_t tile = (size_t)blockIdx.x * Q::STAGE_F2;
  const int row = blockIdx.x * Q::ROWS + 2 * p;                    // rows `row`, `row` + 1
  const float kf = a.g.kf;
  auto field = [](int q) { return q < 3 ? q : q - 3; };
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int st = 0; st < Q::STAGES; ++st) mbar_init(&bar[st], 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < Q::STAGES; ++q) {
      mbar_expect_tx(&bar[q], Q::STAGE_BYTES);
      bulk_load(ring + q * Q::STAGE_F2, a.in[field(q)] + zs + tile, Q::STAGE_BYTES, &bar[q]);
    }
  }
  load_twiddles(s_tw, a.tw, N);
  // Stage q of the ring into v (z_assemble with the field's z-derivative order), then the
  // copy of stage q + STAGES; false if a wait ran out (the CTA has then drained its copies
  // and reported, and must return).
  auto fetch = [&](int q, float2 (&v)[C::RMAX]) -> bool {
    const int st = q % Q::STAGES;
    const bool ok = mbar_wait(&bar[st], (q / Q::STAGES) & 1, a.g.wait);
    if (!ok) s_fail = 1;
    const float2* ra = ring + st * Q::STAGE_F2 + (2 * p) * C::H;
    const int m = a.ord[field(q)];
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r)
      v[r] = ok ? z_assemble_smem<N>(ra, ra + C::H, elem<N>(t, r), kf, m) : make_float2(0.f, 0.f);
    __syncthreads();   // stage consumed by every thread (and, at q = 0, twiddles visible)
    if (s_fail) {
      if (threadIdx.x == 0) {
        for (int g = q; g < NQ && g < q + Q::STAGES; ++g) mbar_wait(&bar[g % Q::STAGES], (g / Q::STAGES) & 1);
        report_device_error(a.g.err, LPT2_DEV_ETIMEOUT_ZADJSOURCE);
      }
      return false;
    }
    if (threadIdx.x == 0 && q + Q::STAGES < NQ) {
      mbar_expect_tx(&bar[st], Q::STAGE_BYTES);
      bulk_load(ring + st * Q::STAGE_F2, a.in[field(q + Q::STAGES)] + zs + tile, Q::STAGE_BYTES, &bar[st]);
    }
    return true;
  };
  // trace of the Hessian for both rows (fields xx, yy, zz)
  float T0[C::RMAX], T1[C::RMAX];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    float2 v[C::RMAX];
    if (!fetch(q, v)) return;
    fft<N, true>(v, t, sm, s_tw);
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) {
      T0[r] = q == 0 ? v[r].x : T0[r] + v[r].x;
      T1[r] = q == 0 ? v[r].y : T1[r] + v[r].y;
    }
  }
  // the six cotangents: one loop body (not unrolled: nine copies of the two transforms
  // overflow the instruction cache)
  const float* g0 = a.gs + zr + (size_t)row * N;
#pragma unroll 1
  for (int q = 3; q < NQ; ++q) {
    float2 v[C::RMAX];
    if (!fetch(q, v)) return;
    const int f = q - 3;
    fft<N, true>(v, t, sm, s_tw);
    if (f < 3) {
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) {
        const int iz = elem<N>(t, r);
        const float ga = __ldg(g0 + iz), gb = __ldg(g0 + N + iz);
        v[r] = make_float2(ga * (T0[r] - v[r].x), gb * (T1[r] - v[r].y));
      }
    } else {
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) {
        const int iz = elem<N>(t, r);
        const float ga = __ldg(g0 + iz), gb = __ldg(g0 + N + iz);
        v[r] = make_float2(-2.f * ga * v[r].x, -2.f * gb * v[r].y);
      }
    }
    fft<N, false>(v, t, sm, s_tw);
    float2* out = a.out[f] + zs + tile + (size_t)(2 * p) * C::H;
    z_store_pair_d<N>(v, t, sm, out, out + C::H, kf, a.ord[f], a.ord[f]);
    sm.sync();   // the row's reads above are done before the next transform reuses it
  }
}

// Field-pair form of k_z_adj_source, for grids whose pencil is one warp (N / RMAX = 32,
// N = 512).  A warp owns one real row; its six phi_ij arrive as three complex pencils
// (xx + i yy, zz + i xy, xz + i yz).  After the first two inverse transforms the row holds
// A = phi_xx, B = phi_yy, C = phi_zz, D = phi_xy, which give four of the cotangents,
//   g_xx = g_S (B + C),  g_yy = g_S (A + C),  g_zz = g_S (A + B),  g_xy = -2 g_S D
// (g_ii = g_S (Tr - phi_ii)), transformed forward two at a time (g_xx + i g_yy,
// g_zz + i g_xy) and split into their half spectra; the third pencil gives g_xz, g_yz.
// Per row: three inverse and three forward transforms, each phi_ij and g_S read once (the
// paired-row form transforms 7.5 pencils per row and reads the diagonal fields twice).
// Tiles as in the field-pair layout: a ring stage holds the two fields of a pencil for the
// CTA's eight rows, each row in its warp's padded region, used in place as the exchange row.
#ifndef LPT2_ZADJ_FIELD_PAIRS
#define LPT2_ZADJ_FIELD_PAIRS 1
#endif
template <int N> struct ZAdjFpCfg {
  static constexpr int RMAX = Cfg<N>::RMAX, TPP = N / RMAX, H = N / 2;
  static constexpr int ROWS = 8;                               // rows (warps) per CTA
  static constexpr int THREADS = ROWS * 32;
  static constexpr int ROWW = SmemRow::words(N);               // float2 per warp region
  static constexpr int STAGE_F2 = ROWS * ROWW;
  static constexpr unsigned STAGE_BYTES = ROWS * 2 * H * 8u;   // bytes landing per stage
  static constexpr int BAR_OFF = (N + 2 * STAGE_F2) * 8;       // twiddles, two stages, barriers
  static constexpr int SMEM = BAR_OFF + 64;
  static constexpr bool OK = TPP == 32;
  static_assert(!OK || ((ROWW * 8) % 16 == 0 && (H * 8) % 16 == 0), "bulk copies need 16-byte alignment");
};
template <int N> constexpr bool zadj_field_pairs() { return LPT2_ZADJ_FIELD_PAIRS && ZAdjFpCfg<N>::OK; }

template <int N>
__global__ void __launch_bounds__(ZAdjFpCfg<N>::THREADS, 2) k_z_adj_source_fp(ZAdjSourceArgs a) {
  using Q = ZAdjFpCfg<N>;
  constexpr int RMAX = Q::RMAX, H = Q::H;
  extern __shared__ __align__(128) unsigned char za_raw[];
  float2* s_tw = reinterpret_cast<float2*>(za_raw);
  float2* ring = s_tw + N;
  uint64_t* bar = reinterpret_cast<uint64_t*>(za_raw + Q::BAR_OFF);
  __shared__ int s_fail;
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  const size_t n3 = (size_t)N * N * N;
  const size_t zs = blockIdx.z * (n3 / 2), zr = blockIdx.z * n3;   // instance blockIdx.z
  const size_t row0 = (size_t)blockIdx.x * Q::ROWS, row = row0 + warp;
  const float kf = a.g.kf;
  auto issue = [&](int k) {   // pencil k's two fields -> stage k & 1
    float2* st = ring + (k & 1) * Q::STAGE_F2;
    mbar_expect_tx(&bar[k & 1], Q::STAGE_BYTES);
    for (int r = 0; r < Q::ROWS; ++r) {
      bulk_load(st + r * Q::ROWW, a.in[2 * k] + zs + (row0 + r) * H, H * 8u, &bar[k & 1]);
      bulk_load(st + r * Q::ROWW + H, a.in[2 * k + 1] + zs + (row0 + r) * H, H * 8u, &bar[k & 1]);
    }
  };
  if (threadIdx.x == 0) {
    s_fail = 0;
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
    issue(0);
    issue(1);
  }
  const float* gsr = a.gs + zr + row * N;   // g_S of this row (read where used: registers are short)
  load_twiddles(s_tw, a.tw, N);
  __syncthreads();
  // pencil k of this warp's row into v (Hermitian extension of both fields with their z
  // derivative orders, Z = A + i B); false if a wait ran out (drained and reported)
  auto fetch = [&](int k, float2 (&v)[RMAX]) -> bool {
    const bool ok = mbar_wait(&bar[k & 1], (k >> 1) & 1, a.g.wait);
    if (!ok) s_fail = 1;
    __syncthreads();
    if (s_fail) {
      if (threadIdx.x == 0) {
        for (int g = k; g < (k == 0 ? 2 : 3); ++g) mbar_wait(&bar[g & 1], (g >> 1) & 1);
        report_device_error(a.g.err, LPT2_DEV_ETIMEOUT_ZADJSOURCE);
      }
      return false;
    }
    const float2* reg = ring + (k & 1) * Q::STAGE_F2 + warp * Q::ROWW;
    const int ma = a.ord[2 * k], mb = a.ord[2 * k + 1];
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      const int n = elem<N>(t, r);
      if (n == H) {
        v[r] = make_float2(0.f, 0.f);
      } else {
        const bool lo = n < H;
        const int j = lo ? n : N - n;
        const float kz = kf * (float)j;
        float2 A = deriv(reg[j], kz, ma), B = deriv(reg[H + j], kz, mb);
        if (!lo) { A = cconj(A); B = cconj(B); }
        v[r] = make_float2(A.x - B.y, A.y + B.x);
      }
    }
    __syncwarp();   // the row is read before the transform's exchanges overwrite it
    return true;
  };
  const SmemRowT<true> sm0{ring + warp * Q::ROWW}, sm1{ring + Q::STAGE_F2 + warp * Q::ROWW};
  // pencil 0: phi_xx + i phi_yy
  float2 ab[RMAX];
  if (!fetch(0, ab)) return;
  fft<N, true>(ab, t, sm0, s_tw);
  __syncthreads();   // stage 0 free in every warp: the third pencil goes there
  if (threadIdx.x == 0) {
    fence_proxy_async_smem();
    issue(2);
  }
  // pencil 1: phi_zz + i phi_xy; the cotangents of the diagonals and of xy
  float2 v[RMAX], q[RMAX];
  if (!fetch(1, v)) return;
  fft<N, true>(v, t, sm1, s_tw);
#pragma unroll
  for (int r = 0; r < RMAX; ++r) {
    const float A = ab[r].x, B = ab[r].y, Cz = v[r].x, D = v[r].y, g = __ldg(gsr + elem<N>(t, r));
    q[r] = make_float2(g * (A + B), -2.f * g * D);    // g_zz + i g_xy
    v[r] = make_float2(g * (B + Cz), g * (A + Cz));   // g_xx + i g_yy
  }
  fft<N, false>(v, t, sm1, s_tw);
  z_store_pair_d<N>(v, t, sm1, a.out[0] + zs + row * H, a.out[1] + zs + row * H, kf, a.ord[0], a.ord[1]);
  sm1.sync();
  fft<N, false>(q, t, sm1, s_tw);
  z_store_pair_d<N>(q, t, sm1, a.out[2] + zs + row * H, a.out[3] + zs + row * H, kf, a.ord[2], a.ord[3]);
  // pencil 2: phi_xz + i phi_yz
  if (!fetch(2, v)) return;
  fft<N, true>(v, t, sm0, s_tw);
#pragma unroll
  for (int r = 0; r < RMAX; ++r) {
    const float g = -2.f * __ldg(gsr + elem<N>(t, r));
    v[r] = make_float2(g * v[r].x, g * v[r].y);
  }
  fft<N, false>(v, t, sm0, s_tw);
  z_store_pair_d<N>(v, t, sm0, a.out[4] + zs + row * H, a.out[5] + zs + row * H, kf, a.ord[4], a.ord[5]);
}

// ===================================================================== y pass
// CTA = (kz block of W, fixed x). Thread tid = t * W + w.
// KIND: Y_MULTI  each output = transform of (i k_y)^ord times its input; the input
//                tile is re-read (an L2 hit after the first) for every output so no
//                input copy stays in registers;
//       Y_SUM    out[dst[i]] += conj((i k_y)^ord[i]) forward-transform(in[i]);
//       Y_ONE    one input, one output, no derivative (forward or inverse).
enum YKind { Y_MULTI = 0, Y_SUM = 1, Y_ONE = 2 };

template <int N, int KIND, int WY>
__global__ void __launch_bounds__(YCfg<N, WY>::XT) k_y(YArgs a) {
  using C = YCfg<N, WY>;
  extern __shared__ float2 smem[];
  float2* s_tw = smem;
  load_twiddles(s_tw, a.tw, N);
  const int w = threadIdx.x % C::W, t = threadIdx.x / C::W;
  const SmemCol<C::W> sm{smem + N + w};
  const int kz = blockIdx.x * C::W + w;
  const int x = blockIdx.y;
  const size_t base = blockIdx.z * ((size_t)N * N * C::H) + (size_t)x * N * C::H + kz;   // + y * H
  __syncthreads();
  if (KIND == Y_SUM) {
    for (int o = 0; o < a.job.n_out; ++o) {
      float2 acc[C::RMAX];
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) acc[r] = make_float2(0.f, 0.f);
      for (int i = 0; i < a.job.n_in; ++i) {
        if (a.job.dst[i] != o) continue;
        float2 v[C::RMAX];
#pragma unroll
        for (int r = 0; r < C::RMAX; ++r) v[r] = a.job.in[i][base + (size_t)(elem<N>(t, r)) * C::H];
        fft<N, false>(v, t, sm, s_tw);
        const int zo = a.job.zord[i];
#pragma unroll
        for (int r = 0; r < C::RMAX; ++r) {
          const int n = elem<N>(t, r);
          const float2 u = dconj(v[r], a.g.kf * (float)mode_of(n, N), a.job.ord[i]);
          acc[r] = cadd(acc[r], zo ? dconj(u, a.g.kf * (float)kz, zo) : u);
        }
      }
      float2* dst = a.job.out[o];
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) dst[base + (size_t)(elem<N>(t, r)) * C::H] = acc[r];
    }
    return;
  }
  if (KIND == Y_ONE) {
    float2 v[C::RMAX];
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) v[r] = a.job.in[0][base + (size_t)(elem<N>(t, r)) * C::H];
    if (a.inverse) fft<N, true>(v, t, sm, s_tw);
    else fft<N, false>(v, t, sm, s_tw);
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) a.job.out[0][base + (size_t)(elem<N>(t, r)) * C::H] = v[r];
    return;
  }
  for (int o = 0; o < a.job.n_out; ++o) {
    const float2* src = a.job.in[a.job.src[o]];
    const int m = a.job.ord[o];
    float2 v[C::RMAX];
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) {
      const int n = elem<N>(t, r);
      const float2 u = src[base + (size_t)n * C::H];
      v[r] = (m != 0 && n == C::H) ? make_float2(0.f, 0.f) : deriv(u, a.g.kf * (float)mode_of(n, N), m);
    }
    if (a.inverse) fft<N, true>(v, t, sm, s_tw);
    else fft<N, false>(v, t, sm, s_tw);
    float2* dst = a.job.out[o];
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) dst[base + (size_t)(elem<N>(t, r)) * C::H] = v[r];
  }
}

// ===================================================================== x pass
// Exact integer P(k) shell of mode (mx, my, mz): b = floor(2 ns |n| / N) for
// 0 < |n| < N/2, else -1.  A float estimate is corrected by exact 64-bit integer
// comparisons (b N)^2 <= 4 ns^2 |n|^2 < ((b+1) N)^2; no 64-bit int/float conversion.
template <int N>
__device__ __forceinline__ int shell_of(int mx, int my, int mz, int ns, int& n2) {
  n2 = mx * mx + my * my + mz * mz;                 // < 3 (N/2)^2: exact in int32 and in float
  if (n2 == 0 || 4 * n2 >= N * N) return -1;
  const long long M = 4LL * ns * ns * (long long)n2;
  int b = (int)(sqrtf((float)n2) * (2.0f * (float)ns / (float)N));
  while (b > 0 && (long long)(b * N) * (long long)(b * N) > M) --b;
  while ((long long)((b + 1) * N) * (long long)((b + 1) * N) <= M) ++b;
  return b;
}

// Square of the CIC window W = prod_i sinc^2(pi m_i / N) of mode (mx, my, mz).
__device__ __forceinline__ float sinc2_pi(int m, int n) {
  if (m == 0) return 1.f;
  const float x = (float)m / (float)n;
  const float s = sinpif(x) / (3.14159265358979f * x);
  return s * s;
}
__device__ __forceinline__ float cic_window2(int mx, int my, int mz, int n) {
  const float w = sinc2_pi(mx, n) * sinc2_pi(my, n) * sinc2_pi(mz, n);
  return w * w;
}

// Sum of a float over the warp (all lanes participate).
__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  return x;
}

// Minimum resident CTAs per SM for an x-pass mode: the one-transform shell-sum modes fit
// in 64 registers a thread (twice the CTAs); the others are capped at 128.
template <int N> constexpr int x_minb(int mode) {
  return (mode == X_PK || mode == X_PKP)
             ? (PassCfg<N>::XT >= 1024 ? 1 : 1024 / PassCfg<N>::XT)
             : PassCfg<N>::XMINB;
}

// Tile inputs of the adjoint modes already in shared memory (element (kx, w) at kx W + w):
// `summed` = v holds the sum of the transformed x-order groups; hpsi, delta, s replace the
// global reads of hpsi_in, delta_in and s_in (null: read from global memory).
struct XSmemIn {
  bool summed = false;
  const float2* hpsi = nullptr;
  const float2* delta = nullptr;
  const float2* s = nullptr;
};

// One x-pass tile: kz block kzb (W consecutive kz), fixed ky, instance inst, all kx.
// Thread tid = t * W + w; kx = elem(t, r).  v holds the tile's input (non-adjoint modes;
// the adjoint modes load their x-order groups here), sm is the tile's exchange buffer,
// s_acc the per-warp accumulators (zeroed by the caller), blk the tile's linear index,
// s_sc the tile of the scf field staged in shared memory (element (kx, w) at kx W + w), or
// null to read a.scf from global memory.
template <int N, int MODE>
__device__ __forceinline__ void x_tile(const XArgs& a, float2 (&v)[PassCfg<N>::RMAX], int kzb, int ky, int inst,
                                       size_t blk, const SmemCol<PassCfg<N>::W>& sm, const float2* s_tw,
                                       double* s_acc, const float* s_sc = nullptr, XSmemIn si = {}) {
  using C = PassCfg<N>;
  const int w = threadIdx.x % C::W, t = threadIdx.x / C::W;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NWARP = C::XT / 32;
  const int kz = kzb * C::W + w;
  const size_t base = inst * ((size_t)N * N * C::H) + (size_t)ky * C::H + kz;   // + kx * N * H
  const size_t stride = (size_t)N * C::H;
  const int my = mode_of(ky, N), mz = kz;
  const bool ny_nyq = (ky == C::H);
  const float kf = a.g.kf;
  (void)warp;
  (void)lane;
  const bool adjoint = (MODE == X_ADJ_SOURCE || MODE == X_ADJ_DELTA);
  if (adjoint && !si.summed) {
    // forward x transform of each x-order group, summed with conj((i kx)^m)
    const int ng = (MODE == X_ADJ_SOURCE) ? 2 : 3;
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) v[r] = make_float2(0.f, 0.f);
    for (int gi = 0; gi < ng; ++gi) {
      float2 u[C::RMAX];
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) u[r] = a.in2[gi][base + (size_t)(elem<N>(t, r)) * stride];
      fft<N, false>(u, t, sm, s_tw);
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) {
        const int kx = elem<N>(t, r);
        v[r] = acc_dconj(v[r], u[r], kf * (float)mode_of(kx, N), gi);
      }
    }
  } else if (!adjoint) {
    if (MODE == X_MUL) {   // full-source diagnostic: multiplier, then inverse x
      const size_t toff = (size_t)inst * mode_table_len(N);
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) {
        const int kx = elem<N>(t, r);
        const int mx = mode_of(kx, N);
        const int n2 = mx * mx + my * my + mz * mz;
        const bool zero = ny_nyq || kx == C::H || n2 == 0;
        const float4 mt = zero ? make_float4(0.f, 0.f, 0.f, 0.f) : __ldg(a.mt0 + toff + n2);
        const float q = kf * kf * (float)n2 * a.mul_inv_a2;   // k^2 / a^2
        float gk;
        switch (a.mul_g) {
          case G_POT: gk = mt.z * mt.y; break;                                          // D1 / (k^2 N^3)
          case G_MUPOT: gk = mt.z * mt.y * (1.f + q / (3.f * (q + a.mul_m2a))); break;
          case G_PSI: gk = mt.z * a.g.inv_n3 / (q + a.mul_m2a); break;
          case G_POT0: gk = a.mul_d1gr * mt.y; break;
          default: gk = mt.z * a.g.inv_n3; break;                                       // G_D1
        }
        float2 u = zero ? make_float2(0.f, 0.f) : cscale(v[r], gk);
        u = deriv(u, kf * (float)mx, a.mul_ord[0]);
        u = deriv(u, kf * (float)my, a.mul_ord[1]);
        v[r] = deriv(u, kf * (float)mz, a.mul_ord[2]);
      }
      fft<N, true>(v, t, sm, s_tw);
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) a.out[0][base + (size_t)(elem<N>(t, r)) * stride] = v[r];
      return;
    }
    if (MODE == X_INV) {
      fft<N, true>(v, t, sm, s_tw);
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) a.out[0][base + (size_t)(elem<N>(t, r)) * stride] = v[r];
      return;
    }
    fft<N, false>(v, t, sm, s_tw);
    if (MODE == X_FWD) {
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) a.out[0][base + (size_t)(elem<N>(t, r)) * stride] = v[r];
      return;
    }
  }

  if (MODE == X_PKI) {
    // interlacing: the second grid (particles shifted by +h/2 on every axis) sees the
    // density at x - h/2; its spectrum is realigned by exp(+i pi (mx + my + mz) / N) and
    // the two are averaged, which cancels the odd aliasing images of the first grid
    float2 u[C::RMAX];
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) u[r] = a.in2[0][base + (size_t)(elem<N>(t, r)) * stride];
    fft<N, false>(u, t, sm, s_tw);
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) {
      const int mx = mode_of(elem<N>(t, r), N);
      float sn, cs;
      sincospif((float)(mx + my + mz) / (float)N, &sn, &cs);
      const float2 w = cmul(u[r], make_float2(cs, sn));
      v[r] = make_float2(0.5f * (v[r].x + w.x), 0.5f * (v[r].y + w.y));
    }
  }
  if (MODE == X_PKP || MODE == X_PKI) {
    // P(k) shells (mode counts and mean |k| come from the cached shell geometry).  At one
    // register slot a warp holds a compact patch of modes (consecutive kx and kz), which
    // mostly falls in one or two shells: the warp finds its smallest and largest shell
    // (two reductions), sums V |delta|^2 / N^6 over the lanes of each (warp sums) and one
    // lane adds the sums to the warp's own FP32 histogram in shared memory; a patch over
    // more shells takes them one at a time.  At most 32 x RMAX values per shell and warp
    // (relative error below 4e-5 even when every rounding goes one way); the sums over
    // warps and blocks are FP64.
    const float pnorm = a.g.box * a.g.box * a.g.box * a.g.inv_n3 * a.g.inv_n3;
    const int ns = a.n_shells;
    float* s_mine = reinterpret_cast<float*>(s_acc) + warp * ns;
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) {
      const int kx = elem<N>(t, r);
      int n2;
      const int b = shell_of<N>(mode_of(kx, N), my, mz, ns, n2);
      float pv = 0.f;
      if (b >= 0) {
        pv = (v[r].x * v[r].x + v[r].y * v[r].y) * pnorm * (mz == 0 ? 1.f : 2.f);
        if (a.pk_deconv) pv /= cic_window2(mode_of(kx, N), my, mz, N);
      }
      const int lo = (int)__reduce_min_sync(0xffffffffu, (unsigned)(b < 0 ? 0x7fffffff : b));
      const int hi = (int)__reduce_max_sync(0xffffffffu, (unsigned)(b < 0 ? 0 : b + 1)) - 1;
      if (lo > hi) continue;                         // no mode of the patch in a shell
      const float s0 = warp_sum(b == lo ? pv : 0.f);
      if (lane == 0) s_mine[lo] += s0;
      if (hi == lo) continue;
      const float s1 = warp_sum(b == hi ? pv : 0.f);
      if (lane == 0) s_mine[hi] += s1;
      for (int k = lo + 1; k < hi; ++k) {            // shells strictly between (rare)
        const float sk = warp_sum(b == k ? pv : 0.f);
        if (lane == 0) s_mine[k] += sk;
      }
    }
    __syncthreads();
    const float* s_all = reinterpret_cast<const float*>(s_acc);
    for (int b = threadIdx.x; b < ns; b += blockDim.x) {
      double acc = 0.0;
      for (int wi = 0; wi < NWARP; ++wi) acc += (double)s_all[wi * ns + b];   // fixed order
      a.pk_part[blk * ns + b] = acc;
    }
    return;
  }
  if (MODE == X_PK) {
    // P(k) shells.  Lanes of a warp see neighbouring modes, so they fall in few
    // shells: for each distinct shell in the warp the lanes of that shell are
    // summed and one lane adds the sum to this warp's own accumulator, a
    // Kahan-compensated FP32 pair (FP64-class accuracy without FP64 adds, which
    // are slow on this part); the sums over warps and blocks are FP64.  X_PK also
    // sums |k| and the mode counts; X_PKP leaves them to the cached shell geometry.
    constexpr bool GEO = true;
    constexpr int NQ = 5;             // per warp: P, its compensation, |k|, compensation, count
    const float pnorm = a.g.box * a.g.box * a.g.box * a.g.inv_n3 * a.g.inv_n3;
    const int ns = a.n_shells;
    float* s_mine = reinterpret_cast<float*>(s_acc) + warp * NQ * ns;
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) {
      const int kx = elem<N>(t, r);
      int n2;
      const int b = shell_of<N>(mode_of(kx, N), my, mz, ns, n2);
      const int wgt = (b < 0) ? 0 : ((mz == 0) ? 1 : 2);
      const float pv = (v[r].x * v[r].x + v[r].y * v[r].y) * pnorm * (float)wgt;
      const float kv = kf * sqrtf((float)n2) * (float)wgt;
      unsigned todo = __ballot_sync(0xffffffffu, b >= 0);
      while (todo) {
        const int leader = __ffs(todo) - 1;
        const int key = __shfl_sync(0xffffffffu, b, leader);
        const bool mine = (b == key);
        float sp = mine ? pv : 0.f, sk = mine ? kv : 0.f;
        int sc = mine ? wgt : 0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          sp += __shfl_xor_sync(0xffffffffu, sp, off);
          if (GEO) {
            sk += __shfl_xor_sync(0xffffffffu, sk, off);
            sc += __shfl_xor_sync(0xffffffffu, sc, off);
          }
        }
        if (lane == leader) {   // this warp's own accumulators: no atomics
          {
            const float y = sp - s_mine[ns + key], t2 = s_mine[key] + y;
            s_mine[ns + key] = (t2 - s_mine[key]) - y;
            s_mine[key] = t2;
          }
          if (GEO) {
            const float y = sk - s_mine[3 * ns + key], t2 = s_mine[2 * ns + key] + y;
            s_mine[3 * ns + key] = (t2 - s_mine[2 * ns + key]) - y;
            s_mine[2 * ns + key] = t2;
            s_mine[4 * ns + key] += (float)sc;   // integer counts <= 2 * 32 * RMAX: exact
          }
        }
        todo &= ~__ballot_sync(0xffffffffu, mine);
      }
    }
    __syncthreads();
    const float* s_all = reinterpret_cast<const float*>(s_acc);
    constexpr int NOUT = GEO ? 3 : 1;
    for (int i = threadIdx.x; i < NOUT * ns; i += blockDim.x) {
      const int q = i / ns, b = i % ns;   // quantity (P, |k|, count), shell
      double acc = 0.0;
      for (int wi = 0; wi < NWARP; ++wi) {   // fixed order
        const float* wv = s_all + wi * NQ * ns;
        acc += (q < 2) ? (double)wv[2 * q * ns + b] - (double)wv[(2 * q + 1) * ns + b] : (double)wv[4 * ns + b];
      }
      a.pk_part[blk * NOUT * ns + i] = acc;
    }
    return;
  }

  if (MODE == X_PKADJ) {
    // d P_b / d delta_rho: multiply delta_rho(k) by the per-shell weight, back along x
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) {
      const int kx = elem<N>(t, r);
      int n2;
      const int b = shell_of<N>(mode_of(kx, N), my, mz, a.n_shells, n2);
      v[r] = cscale(v[r], b < 0 ? 0.f : __ldg(a.shell_w + b));
    }
    fft<N, true>(v, t, sm, s_tw);
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) a.out[0][base + (size_t)(elem<N>(t, r)) * stride] = v[r];
    return;
  }

  if (MODE == X_SOURCE && a.s_out) {
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) a.s_out[base + (size_t)(elem<N>(t, r)) * stride] = v[r];
  }

  // k-space multipliers from the per-|n|^2 tables.  g = potential to transform back along x.
  // The modes of a warp hit scattered table entries (a sector each); where the multiplier is
  // sqrt(P N^3/V) and 1/(k^2 N^3) only, the first comes from the scf field (coalesced, or
  // staged with the tile) and the second is computed.
  const size_t toff = (size_t)inst * mode_table_len(N);
  const bool field = (MODE == X_DELTA && !a.split && (s_sc || a.scf)) || (MODE == X_ADJ_DELTA && a.scf);
  float2 g[C::RMAX], hpot[C::RMAX];
  float theta = 0.f;
#pragma unroll
  for (int r = 0; r < C::RMAX; ++r) {
    const int kx = elem<N>(t, r);
    const int mx = mode_of(kx, N);
    const bool zero = ny_nyq || kx == C::H || (mx == 0 && my == 0 && mz == 0);
    const int n2 = mx * mx + my * my + mz * mz;
    const size_t e = base + (size_t)kx * stride;
    float4 mt;
    if (field) {
      const float inv_c = zero ? 0.f : __frcp_rn((float)n2 * a.g.kf2n3);
      float sc_f = 0.f;
      sc_f = s_sc ? s_sc[kx * C::W + w] : __ldg(a.scf + e);
      mt = make_float4(sc_f, inv_c, 0.f, 0.f);
    } else {
      mt = zero ? make_float4(0.f, 0.f, 0.f, 0.f) : __ldg(a.mt0 + toff + n2);
    }
    const float sc = mt.x, inv = mt.y, d1 = mt.z, d2 = mt.w;   // sqrt(P N^3/V), 1/(k^2 N^3), D1, D2
    if (MODE == X_DELTA) {
      const float2 d = cscale(v[r], sc);
      if (a.delta_out) a.delta_out[e] = d;
      g[r] = cscale(d, inv);                                // phi1 = delta / k^2 (1/N^3 folded)
      if (a.split) hpot[r] = cscale(g[r], d1);
    } else if (MODE == X_SOURCE) {                        // v = S(k)
      float2 u = cscale(v[r], -d2 * inv);                   // phi2 = -S D2 / k^2
      if (!a.split) {
        const float2 dl = a.delta_in[e];
        u = cadd(u, cscale(dl, d1 * inv));                  // + phi1 D1 (total potential)
      }
      g[r] = u;
    } else if (MODE == X_ADJ_SOURCE) {                    // v = g_u(k)
      const float2 gu = zero ? make_float2(0.f, 0.f) : v[r];
      a.hpsi_out[e] = cscale(gu, d1 * inv);                 // h_Psi = D1 g_u / (k^2 N^3)
      g[r] = cscale(gu, -d2 * inv);                         // h_S = -D2 g_u / (k^2 N^3)
      if (!zero) {                                          // dL/dln|fR0| contribution
        const float2 tt = __ldg(a.mt1 + toff + n2);
        const float2 dl = si.delta ? si.delta[kx * C::W + w] : a.delta_in[e];
        const float2 sk = si.s ? si.s[kx * C::W + w] : a.s_in[e];
        const float cx = __fmaf_rn(tt.x, dl.x, -__fmul_rn(tt.y, sk.x));
        const float cy = __fmaf_rn(tt.x, dl.y, -__fmul_rn(tt.y, sk.y));
        theta = __fmaf_rn(__fmul_rn(__fmaf_rn(cx, gu.x, __fmul_rn(cy, gu.y)), inv), mz == 0 ? 1.f : 2.f, theta);
      }
    } else {                                                // X_ADJ_DELTA: v = sum of h_phi groups
      const float2 hp = si.hpsi ? si.hpsi[kx * C::W + w] : a.hpsi_in[e];
      // explicit FMAs: the same rounding in every kernel that inlines this tile
      const float2 h = make_float2(__fmaf_rn(v[r].x, inv, hp.x), __fmaf_rn(v[r].y, inv, hp.y));
      g[r] = cscale(h, sc);                                 // s(k) (h_Psi + h_phi)
    }
  }
  if (MODE == X_ADJ_SOURCE) {
    const float ws = warp_sum(theta);
    if (lane == 0) s_acc[warp] = (double)ws;
  }
  // x-inverse transforms with x-derivative orders (the exchange buffer may hold the
  // shared-memory inputs read above: every thread has read its own first)
  if (si.summed) __syncthreads();
  int nout;
  if (MODE == X_DELTA) nout = a.split ? 5 : 3;
  else if (MODE == X_SOURCE) nout = 2;
  else nout = 1;
  for (int o = 0; o < nout; ++o) {
    const bool fromh = (MODE == X_DELTA) && o >= 3;
    const int m = MODE == X_DELTA ? (o < 3 ? o : o - 3) : (MODE == X_SOURCE ? o : 0);
    float2 u[C::RMAX];
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) {
      const int kx = elem<N>(t, r);
      u[r] = deriv(fromh ? hpot[r] : g[r], kf * (float)mode_of(kx, N), m);
    }
    fft<N, true>(u, t, sm, s_tw);
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) a.out[o][base + (size_t)(elem<N>(t, r)) * stride] = u[r];
  }
  if (MODE == X_ADJ_SOURCE && threadIdx.x == 0) {
    double acc = 0.0;
    for (int wi = 0; wi < NWARP; ++wi) acc += s_acc[wi];   // fixed order (barriers inside fft)
    a.theta_part[blk] = acc;
  }
}

// Tile loads from global memory (one CTA per tile): the adjoint modes, whose tiles are sums
// over several inputs, and any mode when the bulk-tensor path is off.
template <int N, int MODE>
__global__ void __launch_bounds__(PassCfg<N>::XT, x_minb<N>(MODE)) k_x(XArgs a) {
  using C = PassCfg<N>;
  extern __shared__ float2 smem[];
  float2* s_tw = smem;
  load_twiddles(s_tw, a.tw, N);
  const int w = threadIdx.x % C::W, t = threadIdx.x / C::W;
  const SmemCol<C::W> sm{smem + N + w};
  double* s_acc = reinterpret_cast<double*>(smem + N + N * C::W);   // per-warp accumulators
  constexpr int NWARP = C::XT / 32;
  if (MODE == X_PK || MODE == X_PKP || MODE == X_PKI) {
    float* s_accf = reinterpret_cast<float*>(s_acc);
    for (int i = threadIdx.x; i < NWARP * (MODE == X_PK ? 5 : 1) * a.n_shells; i += blockDim.x) s_accf[i] = 0.f;
  } else if (MODE == X_ADJ_SOURCE) {
    for (int i = threadIdx.x; i < NWARP; i += blockDim.x) s_acc[i] = 0.0;
  }
  __syncthreads();
  float2 v[C::RMAX];
  if (MODE != X_ADJ_SOURCE && MODE != X_ADJ_DELTA) {
    const size_t base = blockIdx.z * ((size_t)N * N * C::H) + (size_t)blockIdx.y * C::H + blockIdx.x * C::W + w;
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) v[r] = a.in[base + (size_t)(elem<N>(t, r)) * ((size_t)N * C::H)];
  }
  const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  x_tile<N, MODE>(a, v, blockIdx.x, blockIdx.y, blockIdx.z, blk, sm, s_tw, s_acc);
}

// Tile loads by the tensor-memory accelerator: a persistent CTA walks the tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... and keeps two in flight in a shared-memory ring
// (cp.async.bulk.tensor on an mbarrier: no registers, no load instructions), so the load
// of the next tile overlaps the transforms of the current one.  A tile lands in the
// layout of the FFT exchange buffer (kx major, the W kz of a row contiguous), which the
// tile's transforms then use in place.  Every wait is bounded; a CTA whose wait runs out
// waits (default budget) for its copies in flight, sets the error word and returns.
#ifndef LPT2_X_TMA
#define LPT2_X_TMA 1
#endif
// SC: each ring stage also holds the tile of the scf field (TILE floats after the TILE
// float2 of the input).
template <int N, bool SC = false> struct XTmaCfg {
  using C = PassCfg<N>;
  static constexpr int TILE = N * C::W;                 // float2 per tile
  static constexpr int STAGE = TILE + (SC ? TILE / 2 : 0);   // float2 per ring stage
  static constexpr unsigned STAGE_BYTES = STAGE * 8u;
  static constexpr int NBOX = N > 256 ? N / 256 : 1;    // bulk-tensor boxes per tile (<= 256 kx each)
  static constexpr int BOXROWS = N / NBOX;
  static constexpr int KZB = C::H / C::W;               // kz blocks per (ky, instance)
  static constexpr int BAR_OFF = (N + 2 * STAGE) * 8;   // bytes: twiddles, ring, then two barriers
  static constexpr int ACC_OFF = BAR_OFF + 16;
  static_assert((2 * C::W * 4) % 16 == 0 && (!SC || (C::W * 4) % 16 == 0),
                "the boxes' innermost extents must be multiples of 16 bytes");
};

template <int N, int MODE, bool SC>
__global__ void __launch_bounds__(PassCfg<N>::XT, x_minb<N>(MODE)) k_x_tma(const __grid_constant__ XArgs a) {
  using C = PassCfg<N>;
  using Q = XTmaCfg<N, SC>;
  extern __shared__ __align__(128) unsigned char xs_raw[];
  float2* s_tw = reinterpret_cast<float2*>(xs_raw);
  float2* ring = s_tw + N;
  uint64_t* bar = reinterpret_cast<uint64_t*>(xs_raw + Q::BAR_OFF);
  double* s_acc = reinterpret_cast<double*>(xs_raw + Q::ACC_OFF);
  __shared__ int s_fail;
  constexpr int NWARP = C::XT / 32;
  const int w = threadIdx.x % C::W, t = threadIdx.x / C::W;
  const int ntiles = Q::KZB * N * a.g.batch;
  auto issue = [&](int st, int tile) {   // one thread
    const int kzb = tile % Q::KZB, ky = (tile / Q::KZB) % N, inst = tile / (Q::KZB * N);
    mbar_expect_tx(&bar[st], Q::STAGE_BYTES);
#pragma unroll
    for (int j = 0; j < Q::NBOX; ++j)
      tensor_load_4d(ring + st * Q::STAGE + j * Q::BOXROWS * C::W, &a.tmap, 2 * kzb * C::W, ky, j * Q::BOXROWS,
                     inst, &bar[st]);
    if constexpr (SC) {
      float* scs = reinterpret_cast<float*>(ring + st * Q::STAGE + Q::TILE);
#pragma unroll
      for (int j = 0; j < Q::NBOX; ++j)
        tensor_load_4d(scs + j * Q::BOXROWS * C::W, &a.tmap_sc, kzb * C::W, ky, j * Q::BOXROWS, inst, &bar[st]);
    }
  };
  if (threadIdx.x == 0) {
    s_fail = 0;
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
    for (int i = 0; i < 2; ++i)
      if (blockIdx.x + i * gridDim.x < ntiles) issue(i, blockIdx.x + i * gridDim.x);
  }
  load_twiddles(s_tw, a.tw, N);
  __syncthreads();
  for (int i = 0, tile = blockIdx.x; tile < ntiles; ++i, tile += gridDim.x) {
    const int st = i & 1;
    if (MODE == X_PK || MODE == X_PKP) {
      float* s_accf = reinterpret_cast<float*>(s_acc);
      for (int k = threadIdx.x; k < NWARP * (MODE == X_PK ? 5 : 1) * a.n_shells; k += blockDim.x) s_accf[k] = 0.f;
    }
    const bool ok = mbar_wait(&bar[st], (i >> 1) & 1, a.g.wait);
    if (!ok) s_fail = 1;
    float2 v[C::RMAX];
    const float2* tl = ring + st * Q::STAGE;
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) v[r] = ok ? tl[elem<N>(t, r) * C::W + w] : make_float2(0.f, 0.f);
    __syncthreads();   // tile read by every thread before the transforms reuse the buffer
    if (s_fail) {
      if (threadIdx.x == 0) {
        mbar_wait(&bar[st], (i >> 1) & 1);                                           // this tile's copy
        if (tile + gridDim.x < ntiles) mbar_wait(&bar[st ^ 1], ((i + 1) >> 1) & 1);  // the next tile's
        report_device_error(a.g.err, LPT2_DEV_ETIMEOUT_X);
      }
      return;
    }
    const int kzb = tile % Q::KZB, ky = (tile / Q::KZB) % N, inst = tile / (Q::KZB * N);
    const SmemCol<C::W> sm{ring + st * Q::STAGE + w};
    const float* s_sc = SC ? reinterpret_cast<const float*>(ring + st * Q::STAGE + Q::TILE) : nullptr;
    x_tile<N, MODE>(a, v, kzb, ky, inst, (size_t)tile, sm, s_tw, s_acc, s_sc);
    __syncthreads();   // ring stage and accumulators free
    if (threadIdx.x == 0 && tile + 2 * gridDim.x < ntiles) {
      fence_proxy_async_smem();
      issue(st, tile + 2 * gridDim.x);
    }
  }
}

// Adjoint x modes with their tile inputs staged by the tensor-memory accelerator: a
// persistent CTA walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ... and streams each
// tile's four inputs (X_ADJ_DELTA: the x-order groups 0, 1, 2 and h_Psi; X_ADJ_SOURCE: the
// groups 0, 1, delta(k) and S(k)) through a three-stage shared-memory ring in that order:
// input c sits in stage c mod 3.  A group's forward transform runs in place in its stage,
// after which the stage takes input c + 3; the tile's last inputs are read by the
// multiplier and the inverse transform runs in the last stage.  The loads of the next
// tile's first groups overlap this tile's multiplier and inverse transform.  Every wait is
// bounded; a CTA whose wait runs out waits (default budget) for its copies in flight, sets
// the error word and returns.
template <int N> struct XAdjCfg {
  using C = PassCfg<N>;
  static constexpr int TILE = N * C::W;
  static constexpr int NBOX = N > 256 ? N / 256 : 1;
  static constexpr int BOXROWS = N / NBOX;
  static constexpr int KZB = C::H / C::W;
  static constexpr int BAR_OFF = (N + 3 * TILE) * 8;   // twiddles, three stages, barriers
  static constexpr int ACC_OFF = BAR_OFF + 32;
};

template <int N, int MODE>
__global__ void __launch_bounds__(PassCfg<N>::XT, x_minb<N>(MODE)) k_x_tma_adj(const __grid_constant__ XArgs a) {
  using C = PassCfg<N>;
  using Q = XAdjCfg<N>;
  constexpr int NG = MODE == X_ADJ_SOURCE ? 2 : 3;   // transformed groups per tile (then 4 - NG plain inputs)
  constexpr int NWARP = C::XT / 32;
  extern __shared__ __align__(128) unsigned char xa_raw[];
  float2* s_tw = reinterpret_cast<float2*>(xa_raw);
  float2* ring = s_tw + N;
  uint64_t* bar = reinterpret_cast<uint64_t*>(xa_raw + Q::BAR_OFF);
  double* s_acc = reinterpret_cast<double*>(xa_raw + Q::ACC_OFF);
  __shared__ int s_fail;
  const int w = threadIdx.x % C::W, t = threadIdx.x / C::W;
  const int ntiles = Q::KZB * N * a.g.batch;
  const int mine = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int nload = 4 * mine;
  int issued = 0;                      // thread 0: inputs issued so far (0 .. nload)
  auto issue = [&]() {                 // thread 0: the next input into its stage
    const int c = issued++;
    const int tile = blockIdx.x + (c >> 2) * gridDim.x, j = c & 3, st = c % 3;
    const int kzb = tile % Q::KZB, ky = (tile / Q::KZB) % N, inst = tile / (Q::KZB * N);
    mbar_expect_tx(&bar[st], Q::TILE * 8u);
#pragma unroll
    for (int b = 0; b < Q::NBOX; ++b)
      tensor_load_4d(ring + st * Q::TILE + b * Q::BOXROWS * C::W, &a.tmap_l[j], 2 * kzb * C::W, ky, b * Q::BOXROWS,
                     inst, &bar[st]);
  };
  auto drain = [&](int c) {            // thread 0: wait (default budget) for the copies in flight
    for (int g = c; g < issued; ++g) mbar_wait(&bar[g % 3], (g / 3) & 1);
    report_device_error(a.g.err, LPT2_DEV_ETIMEOUT_X);
  };
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int st = 0; st < 3; ++st) mbar_init(&bar[st], 1);
    mbar_init_fence();
    while (issued < 3 && issued < nload) issue();
  }
  load_twiddles(s_tw, a.tw, N);
  __syncthreads();
  int c = 0;                           // next input to wait for
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int kzb = tile % Q::KZB, ky = (tile / Q::KZB) % N, inst = tile / (Q::KZB * N);
    if (MODE == X_ADJ_SOURCE)
      for (int i = threadIdx.x; i < NWARP; i += blockDim.x) s_acc[i] = 0.0;
    float2 v[C::RMAX];
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) v[r] = make_float2(0.f, 0.f);
    for (int j = 0; j < NG; ++j, ++c) {
      const int st = c % 3;
      const bool ok = mbar_wait(&bar[st], (c / 3) & 1, a.g.wait);
      if (!ok) s_fail = 1;
      float2 u[C::RMAX];
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) u[r] = ok ? ring[st * Q::TILE + elem<N>(t, r) * C::W + w] : make_float2(0.f, 0.f);
      __syncthreads();   // stage read by every thread before the transform reuses it (and s_fail seen)
      if (s_fail) {
        if (threadIdx.x == 0) drain(c);
        return;
      }
      fft<N, false>(u, t, SmemCol<C::W>{ring + st * Q::TILE + w}, s_tw);   // ends past its last shared read
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) v[r] = acc_dconj(v[r], u[r], a.g.kf * (float)mode_of(elem<N>(t, r), N), j);
      __syncthreads();   // every warp is past the transform: the stage is free
      if (threadIdx.x == 0 && issued < nload) {
        fence_proxy_async_smem();
        issue();
      }
    }
    bool ok = true;
    for (int j = 0; j < 4 - NG; ++j) ok = mbar_wait(&bar[(c + j) % 3], ((c + j) / 3) & 1, a.g.wait) && ok;
    if (!ok) s_fail = 1;
    __syncthreads();
    if (s_fail) {
      if (threadIdx.x == 0) drain(c);
      return;
    }
    XSmemIn si;
    si.summed = true;
    const int s0 = c % 3, s1 = (c + 1) % 3;
    float2* ex;
    if (MODE == X_ADJ_DELTA) {
      si.hpsi = ring + s0 * Q::TILE;
      ex = ring + s0 * Q::TILE;
    } else {
      si.delta = ring + s0 * Q::TILE;
      si.s = ring + s1 * Q::TILE;
      ex = ring + s1 * Q::TILE;
    }
    x_tile<N, MODE>(a, v, kzb, ky, inst, (size_t)tile, SmemCol<C::W>{ex + w}, s_tw, s_acc, nullptr, si);
    __syncthreads();   // stages and accumulators free
    if (threadIdx.x == 0) {
      fence_proxy_async_smem();
      for (int j = 0; j < 4 - NG && issued < nload; ++j) issue();
    }
    c += 4 - NG;
  }
}

// ================================================================ launchers
// every launcher refuses a batch outside [1, 65535] (grid z) before launching
#define LPT2_CHECK_BATCH(a) \
  if ((a).g.batch < 1 || (a).g.batch > 65535) return cudaErrorInvalidValue

template <int N, int SRC> cudaError_t launch_z_r2c_m(const ZR2CArgs& a, cudaStream_t s) {
  using C = PassCfg<N>;
  LPT2_CHECK_BATCH(a);
  constexpr int smem = zr2c_smem<N, SRC>();
  cudaFuncSetAttribute(k_z_r2c<N, SRC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_z_r2c<N, SRC><<<dim3(N * N / 2 / C::ZP, 1, a.g.batch), C::ZT, smem, s>>>(a);
  return cudaGetLastError();
}
template <int N> cudaError_t launch_z_r2c_t(const ZR2CArgs& a, cudaStream_t s) {
  switch (a.src) {
    case Z_NOISE: return launch_z_r2c_m<N, Z_NOISE>(a, s);
    case Z_REAL: return launch_z_r2c_m<N, Z_REAL>(a, s);
    case Z_DENSITY: return launch_z_r2c_m<N, Z_DENSITY>(a, s);
    default: return cudaErrorInvalidValue;
  }
}
template <int N> cudaError_t launch_z_c2r_t(const ZC2RArgs& a, cudaStream_t s) {
  using C = PassCfg<N>;
  LPT2_CHECK_BATCH(a);
  cudaFuncSetAttribute(k_z_c2r<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::ZSMEM);
  k_z_c2r<N><<<dim3(N * N / 2 / C::ZP, 1, a.g.batch), C::ZT, C::ZSMEM, s>>>(a);
  return cudaGetLastError();
}
template <int N> cudaError_t launch_z_source_t(const ZSourceArgs& a, cudaStream_t s) {
  using C = PassCfg<N>;
  LPT2_CHECK_BATCH(a);
  using Q = ZSrcCfg<N>;
  cudaFuncSetAttribute(k_z_source<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, Q::SMEM);
  k_z_source<N><<<dim3(N * N / Q::ROWS, 1, a.g.batch), C::ZT, Q::SMEM, s>>>(a);
  return cudaGetLastError();
}
template <int N> cudaError_t launch_z_final_t(const ZFinalArgs& a, cudaStream_t s) {
  using C = PassCfg<N>;
  LPT2_CHECK_BATCH(a);
  using Q = ZSrcCfg<N>;
  auto k = a.split ? k_z_final<N, true> : k_z_final<N, false>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Q::SMEM);
  k<<<dim3(N * N / Q::ROWS, 1, a.g.batch), C::ZT, Q::SMEM, s>>>(a);
  return cudaGetLastError();
}
template <int N> cudaError_t launch_z_adj_source_t(const ZAdjSourceArgs& a, cudaStream_t s) {
  using C = PassCfg<N>;
  using Q = ZSrcCfg<N>;
  LPT2_CHECK_BATCH(a);
  if constexpr (zadj_field_pairs<N>()) {
    using F = ZAdjFpCfg<N>;
    cudaFuncSetAttribute(k_z_adj_source_fp<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, F::SMEM);
    k_z_adj_source_fp<N><<<dim3(N * N / F::ROWS, 1, a.g.batch), F::THREADS, F::SMEM, s>>>(a);
    return cudaGetLastError();
  }
  cudaFuncSetAttribute(k_z_adj_source<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, Q::SMEM);
  k_z_adj_source<N><<<dim3(N * N / Q::ROWS, 1, a.g.batch), C::ZT, Q::SMEM, s>>>(a);
  return cudaGetLastError();
}
template <int N, int KIND, int WY> cudaError_t launch_y_k(const YArgs& a, cudaStream_t s) {
  using C = YCfg<N, WY>;
  LPT2_CHECK_BATCH(a);
  cudaFuncSetAttribute(k_y<N, KIND, WY>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::XSMEM);
  k_y<N, KIND, WY><<<dim3(C::H / C::W, N, a.g.batch), C::XT, C::XSMEM, s>>>(a);
  return cudaGetLastError();
}
template <int N, int WY> cudaError_t launch_y_w(const YArgs& a, cudaStream_t s) {
  if (a.job.sum) return launch_y_k<N, Y_SUM, WY>(a, s);
  if (a.job.n_in == 1 && a.job.n_out == 1 && a.job.ord[0] == 0 && a.job.src[0] == 0)
    return launch_y_k<N, Y_ONE, WY>(a, s);
  return launch_y_k<N, Y_MULTI, WY>(a, s);
}
// y pencils per CTA: Geo::ytile 0 (build default), 8 or 16 (where they tile N/2)
template <int N> cudaError_t launch_y_t(const YArgs& a, cudaStream_t s) {
  if constexpr (N >= 32 && YCfg<N>::W != 8) {
    if (a.g.ytile == 8) return launch_y_w<N, 8>(a, s);
  }
  if constexpr (N >= 32 && YCfg<N>::W != 16) {
    if (a.g.ytile == 16) return launch_y_w<N, 16>(a, s);
  }
  if (a.g.ytile != 0 && a.g.ytile != YCfg<N>::W) return cudaErrorInvalidValue;
  return launch_y_w<N, 0>(a, s);
}
// persistent bulk-tensor x pass: as many CTAs as fit on the GPU at once, or one per tile
template <int N, int MODE, bool SC> cudaError_t launch_x_tma(const XArgs& a, int acc, cudaStream_t s) {
  using C = PassCfg<N>;
  using Q = XTmaCfg<N, SC>;
  XArgs b = a;
  if (!encode_x_tile_map(&b.tmap, a.in, N, N, 2 * C::W, a.g.batch)) return cudaErrorInvalidValue;
  if (SC && !encode_x_tile_map(&b.tmap_sc, a.scf, N / 2, N, C::W, a.g.batch)) return cudaErrorInvalidValue;
  const int smem = Q::ACC_OFF + acc;
  cudaError_t e = cudaFuncSetAttribute(k_x_tma<N, MODE, SC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_x_tma<N, MODE, SC>, C::XT, smem)) != cudaSuccess)
    return e;
  const long long tiles = (long long)Q::KZB * N * a.g.batch;
  const int grid = (int)std::min<long long>(tiles, (long long)sms * std::max(per_sm, 1));
  k_x_tma<N, MODE, SC><<<grid, C::XT, smem, s>>>(b);
  return cudaGetLastError();
}
#ifndef LPT2_X_TMA_ADJ
#define LPT2_X_TMA_ADJ 1
#endif
template <int N, int MODE> cudaError_t launch_x_tma_adj(const XArgs& a, int acc, cudaStream_t s) {
  using C = PassCfg<N>;
  using Q = XAdjCfg<N>;
  XArgs b = a;
  const float2* src[4] = {a.in2[0], a.in2[1], MODE == X_ADJ_DELTA ? a.in2[2] : a.delta_in,
                          MODE == X_ADJ_DELTA ? a.hpsi_in : a.s_in};
  for (int j = 0; j < 4; ++j)
    if (!src[j] || !encode_x_tile_map(&b.tmap_l[j], src[j], N, N, 2 * C::W, a.g.batch)) return cudaErrorInvalidValue;
  const int smem = Q::ACC_OFF + acc;
  cudaError_t e = cudaFuncSetAttribute(k_x_tma_adj<N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_x_tma_adj<N, MODE>, C::XT, smem)) != cudaSuccess)
    return e;
  const long long tiles = (long long)Q::KZB * N * a.g.batch;
  const int grid = (int)std::min<long long>(tiles, (long long)sms * std::max(per_sm, 1));
  k_x_tma_adj<N, MODE><<<grid, C::XT, smem, s>>>(b);
  return cudaGetLastError();
}
template <int N, int MODE> cudaError_t launch_x_m(const XArgs& a, cudaStream_t s) {
  using C = PassCfg<N>;
  LPT2_CHECK_BATCH(a);
  const int acc = MODE == X_PK ? (C::XT / 32) * 5 * a.n_shells * 4
                  : (MODE == X_PKP || MODE == X_PKI) ? (C::XT / 32) * a.n_shells * 4
                                                     : (MODE == X_ADJ_SOURCE ? (C::XT / 32) * 8 : 0);
  // The delta mode and the two adjoint modes have two tile paths: bulk-tensor tiles
  // (default: measured faster at 512^3, x_delta 0.91 -> 0.86 ms, x_adj_delta 1.245 -> 1.113)
  // and global loads; Geo::xtile picks one per grid-size group (0 the build default, 1
  // bulk-tensor, 2 global) and the other modes ignore it.  The one-transform shell-sum modes keep the global-load kernel at twice
  // the CTAs per SM, and the source multiplier, which also reads delta(k) per mode, measured
  // 0.73 -> 0.76 ms with bulk-tensor tiles.
  if (a.g.xtile < 0 || a.g.xtile > 2) return cudaErrorInvalidValue;
  if constexpr (MODE == X_ADJ_DELTA || MODE == X_ADJ_SOURCE) {
    if (a.g.xtile == 0 ? LPT2_X_TMA_ADJ != 0 : a.g.xtile == 1) return launch_x_tma_adj<N, MODE>(a, acc, s);
  }
  if constexpr (MODE == X_DELTA) {
    if (a.g.xtile == 0 ? LPT2_X_TMA != 0 : a.g.xtile == 1) {
      if constexpr (MODE == X_DELTA) {
        if (a.scf && !a.split) return launch_x_tma<N, MODE, true>(a, acc, s);
      }
      return launch_x_tma<N, MODE, false>(a, acc, s);
    }
  }
  const int smem = C::XSMEM + acc;
  cudaFuncSetAttribute(k_x<N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_x<N, MODE><<<dim3(C::H / C::W, N, a.g.batch), C::XT, smem, s>>>(a);
  return cudaGetLastError();
}
template <int N> cudaError_t launch_x_t(const XArgs& a, cudaStream_t s) {
  switch (a.mode) {
    case X_DELTA: return launch_x_m<N, X_DELTA>(a, s);
    case X_SOURCE: return launch_x_m<N, X_SOURCE>(a, s);
    case X_PK: return launch_x_m<N, X_PK>(a, s);
    case X_PKP: return launch_x_m<N, X_PKP>(a, s);
    case X_MUL: return launch_x_m<N, X_MUL>(a, s);
    case X_PKI: return launch_x_m<N, X_PKI>(a, s);
    case X_FWD: return launch_x_m<N, X_FWD>(a, s);
    case X_INV: return launch_x_m<N, X_INV>(a, s);
    case X_PKADJ: return launch_x_m<N, X_PKADJ>(a, s);
    case X_ADJ_SOURCE: return launch_x_m<N, X_ADJ_SOURCE>(a, s);
    case X_ADJ_DELTA: return launch_x_m<N, X_ADJ_DELTA>(a, s);
    default: return cudaErrorInvalidValue;
  }
}
template <int N> int x_blocks_t() { return (PassCfg<N>::H / PassCfg<N>::W) * N; }

}  // namespace lpt2

#define LPT2_INSTANTIATE(N)                                                                          \
  namespace lpt2 {                                                                                   \
  cudaError_t launch_z_r2c_##N(const ZR2CArgs& a, cudaStream_t s) { return launch_z_r2c_t<N>(a, s); } \
  cudaError_t launch_z_c2r_##N(const ZC2RArgs& a, cudaStream_t s) { return launch_z_c2r_t<N>(a, s); } \
  cudaError_t launch_z_source_##N(const ZSourceArgs& a, cudaStream_t s) {                            \
    return launch_z_source_t<N>(a, s);                                                               \
  }                                                                                                  \
  cudaError_t launch_z_final_##N(const ZFinalArgs& a, cudaStream_t s) {                              \
    return launch_z_final_t<N>(a, s);                                                                \
  }                                                                                                  \
  cudaError_t launch_y_##N(const YArgs& a, cudaStream_t s) { return launch_y_t<N>(a, s); }           \
  cudaError_t launch_z_adj_source_##N(const ZAdjSourceArgs& a, cudaStream_t s) {                     \
    return launch_z_adj_source_t<N>(a, s);                                                           \
  }                                                                                                  \
  cudaError_t launch_x_##N(const XArgs& a, cudaStream_t s) { return launch_x_t<N>(a, s); }           \
  int x_blocks_##N() { return x_blocks_t<N>(); }                                                     \
  }
