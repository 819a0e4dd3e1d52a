// FP64 set-up kernels: Eisenstein-Hu constants and sigma_8 normalisation of
// P(k), and the batched RK4 integration of the growth tables D1(k,a), D2(k,a)
// (T1 triangle by default, or another triangle of the Sec. 3 comparison) with
// their ln|f_R0| tangents.
//
// Equations (units h/Mpc, s = ln a, flat E^2 = Om a^-3 + OL):
//   D1_ss + (2 - 1.5 Om(a)) D1_s = 1.5 Om(a) mu(k,a) D1                    (Eq. d1)
//   D2_ss + (2 - 1.5 Om(a)) D2_s - 1.5 Om(a) mu(k) D2
//       = -1.5 Om(a) D1(k/sqrt2)^2 [mu(k) - B(k,a)],                     (Eq. full-d2, T1)
//   B = (2/27) 4 pi G rho (k^2/a^2) M2(a) / (Pi(k) Pi(k/sqrt2)^2),
//   mu = 1 + (k^2/a^2) / (3 Pi), Pi = k^2/a^2 + m^2, m^2 = M1/3    (Eq. mihusawicki, Sec. 2.4)
// with D2 taken with the sign that gives -3/7 D1^2 in GR, the EdS growing mode at
// a_init and D1 normalised to the GR solution at a = 1.  Tangents use
// dm^2/dln|fR0| = -m^2 and dM2/dln|fR0| = -2 M2.
// Other triangles (k1 = r k2 at angle theta between k1 and k2, |k1 + k2| = k): the
// source is -1.5 Om D1(k1) D1(k2) times the Eq. full-d2 braces
//   mu - c^2 (mu1 + mu2 - mu) + m^2/Pi [2 c^2 (mu1 + mu2 - 2) + (c/r)(mu1 - 1) + r c (mu2 - 1)]
//   - (2/27) 4piGrho (k^2/a^2) M2 / (Pi Pi1 Pi2),   c = cos theta,
// divided by sin^2 theta so that every triangle keeps the GR limit; Winther's variant
// takes D1(k)^2 with the T1 braces; the GR variant solves the D2 equation with mu = 1.
#include <math.h>

#include "passes.h"

namespace lpt2 {

static constexpr double kH0c = 1.0 / 2997.92458;   // H0 / c in h/Mpc
static constexpr int kSigmaPts = 20001;            // Simpson points in ln k on [1e-5, 1e3]
static constexpr int kPartBlocks = 64;

struct EhConst { double theta2, omh, alpha, s; };

__device__ EhConst eh_constants(const GrowthParams& p) {
  const double h = p.h, wm = p.omega_m * h * h, wb = p.omega_b * h * h, fb = p.omega_b / p.omega_m;
  const double theta = p.t_cmb / 2.7;
  EhConst c;
  c.theta2 = theta * theta;
  c.s = 44.5 * log(9.83 / wm) / sqrt(1.0 + 10.0 * pow(wb, 0.75));                 // EH Eq. 26
  c.alpha = 1.0 - 0.328 * log(431.0 * wm) * fb + 0.38 * log(22.3 * wm) * fb * fb;   // EH Eq. 31
  c.omh = p.omega_m * h;
  return c;
}

__device__ double eh_T64(const EhConst& c, double k, double h) {
  const double sk = 0.43 * k * h * c.s;
  const double gamma = c.omh * (c.alpha + (1.0 - c.alpha) / (1.0 + sk * sk * sk * sk));  // Eq. 30
  const double q = k * c.theta2 / gamma;                                                  // Eq. 28
  const double L0 = log(2.0 * 2.718281828459045 + 1.8 * q);                              // Eq. 29
  const double C0 = 14.2 + 731.0 / (1.0 + 62.5 * q);
  return L0 / (L0 + C0 * q * q);
}

__global__ void k_sigma_partial(GrowthParams p, double* part) {
  const EhConst c = eh_constants(p);
  const double lo = log(1e-5), hi = log(1e3), dl = (hi - lo) / (kSigmaPts - 1);
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kSigmaPts; i += gridDim.x * blockDim.x) {
    const double k = exp(lo + i * dl);
    const double T = eh_T64(c, k, p.h);
    const double x = 8.0 * k;
    const double W = 3.0 * (sin(x) - x * cos(x)) / (x * x * x);
    const double f = k * k * k * pow(k, p.n_s) * T * T * W * W / (2.0 * M_PI * M_PI);
    const double w = (i == 0 || i == kSigmaPts - 1) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
    acc += w * f;
  }
  __shared__ double s[256];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0] * dl / 3.0;
}

__global__ void k_sigma_final(GrowthParams p, const double* part, DevCosmo* out) {
  if (threadIdx.x != 0) return;
  double s2 = 0.0;
  for (int b = 0; b < kPartBlocks; ++b) s2 += part[b];
  const EhConst c = eh_constants(p);
  DevCosmo d;
  d.sigma_sq = s2;
  d.amp = p.sigma8 * p.sigma8 / s2;
  d.sqrt_amp = (float)sqrt(d.amp);
  d.ns_half = (float)(0.5 * p.n_s);
  d.theta2 = (float)c.theta2;
  d.omh = (float)c.omh;
  d.alpha = (float)c.alpha;
  d.s043h = (float)(0.43 * c.s * p.h);
  d.lnkmin = (float)log(p.k_min);
  d.inv_dlnk = (float)((p.nk - 1) / (log(p.k_max) - log(p.k_min)));
  d.nk = p.nk;
  *out = d;
}

int cosmo_partial_blocks() { return kPartBlocks; }

cudaError_t launch_cosmo_setup(const GrowthParams& p, double* partials, DevCosmo* out, cudaStream_t s) {
  k_sigma_partial<<<kPartBlocks, 256, 0, s>>>(p, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sigma_final<<<1, 32, 0, s>>>(p, partials, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ growth RK4
// Background at every half step, shared by the block: 1/a^2, 1.5 Om(a),
// 2 - 1.5 Om(a), m^2(a), (2/27) 4 pi G rho M2(a).
struct Bg { double inv_a2, cc, damp, m2, bfac; };

__device__ Bg background(const GrowthParams& p, double s, bool gr) {
  const double a = exp(s);
  const double a3 = 1.0 / (a * a * a);
  const double e2 = p.omega_m * a3 + p.omega_l;
  const double om = p.omega_m * a3 / e2;
  Bg b;
  b.inv_a2 = 1.0 / (a * a);
  b.cc = 1.5 * om;
  b.damp = 2.0 - 1.5 * om;
  if (gr) {
    b.m2 = 0.0;
    b.bfac = 0.0;
  } else {
    const double x = p.omega_m * a3 + 4.0 * p.omega_l, x0 = p.omega_m + 4.0 * p.omega_l;
    const double x2 = x * x, x02 = x0 * x0;
    b.m2 = 0.5 * kH0c * kH0c * x2 * x / (p.fr0_abs * x02);
    const double M2 = 2.25 * kH0c * kH0c * x2 * x2 * x / (p.fr0_abs * p.fr0_abs * x02 * x02);
    b.bfac = (2.0 / 27.0) * 1.5 * p.omega_m * a3 * kH0c * kH0c * M2;
  }
  return b;
}

// Triangle of a D2 variant: fa, fb = (k1/k)^2, (k2/k)^2, c = cos theta, r = k1/k2.
struct D2Geo {
  double fa, fb, c, c2, inv_s2, r;
  int winther, gr2;
  int fit;   // D2 from the LCDM fit Eq. lcdm-fit with the scale-dependent D1 (no D2 equation)
};

__host__ __device__ inline D2Geo d2_geo(int variant) {
  // (r, theta in degrees) of the Sec. 3 comparison; Winther and GR use the T1 geometry
  double r = 1.0, th = 90.0;
  switch (variant) {
    case 1: th = 80.0; break;
    case 2: th = 70.0; break;
    case 3: r = 2.0; th = 80.0; break;
    case 4: r = 2.0; th = 70.0; break;
    case 7: th = 60.0; break;    // isosceles 60 deg (the text's "equilateral")
    case 8: r = 1e-3; break;     // squeezed: k1 = 1e-3 k2 at 90 deg (k1 ~ 0, k2 ~ k)
    default: break;              // T1; Winther, GR and the LCDM fit use its geometry
  }
  D2Geo g;
  g.c = th == 90.0 ? 0.0 : cos(th * (M_PI / 180.0));
  g.c2 = g.c * g.c;
  g.inv_s2 = 1.0 / (1.0 - g.c2);
  g.r = r;
  const double k2sq = 1.0 / (r * r + 1.0 + 2.0 * r * g.c);   // (k2/k)^2
  g.fb = k2sq;
  g.fa = r * r * k2sq;
  g.winther = variant == 5;
  g.gr2 = variant == 6;
  g.fit = variant == 9;
  return g;
}

// GEO 0: r = 1, c = 0 (T1, Winther, GR): one extra chain, the T1 braces mu - B.
// GEO 1: r = 1, c != 0: one extra chain (k1 = k2), full braces.
// GEO 2: r != 1: chains at k1 and k2, full braces.
template <int GEO> struct Layout {
  static constexpr int NB = GEO == 2 ? 8 : 6;   // states per set: D1, D1s, Da, Das, (Db, Dbs,) D2, D2s
  static constexpr int A = 2, B = GEO == 2 ? 4 : 2, D2 = GEO == 2 ? 6 : 4;
};

// right-hand side; y = [set] (+ [tangent set] when TAN)
template <bool TAN, int GEO>
__device__ __forceinline__ void rhs(const Bg& b, double k2, bool gr, const D2Geo& g, const double* y, double* dy) {
  using L = Layout<GEO>;
  constexpr int T = L::NB;
  const double q = k2 * b.inv_a2, qa = q * g.fa, qb = q * g.fb;
  double mu_k = 1.0, mu_a = 1.0, mu_b = 1.0, mu_kt = 0.0, mu_at = 0.0, mu_bt = 0.0, br = 1.0, brt = 0.0;
  if (!gr) {
    const double rpk = 1.0 / (q + b.m2), rpa = 1.0 / (qa + b.m2);
    const double rpb = GEO == 2 ? 1.0 / (qb + b.m2) : rpa;
    mu_k = 1.0 + q * rpk * (1.0 / 3.0);
    mu_a = 1.0 + qa * rpa * (1.0 / 3.0);
    mu_b = GEO == 2 ? 1.0 + qb * rpb * (1.0 / 3.0) : mu_a;
    const double B = b.bfac * q * rpk * rpa * rpb;
    if (TAN) {
      mu_kt = q * b.m2 * rpk * rpk * (1.0 / 3.0);
      mu_at = qa * b.m2 * rpa * rpa * (1.0 / 3.0);
      mu_bt = GEO == 2 ? qb * b.m2 * rpb * rpb * (1.0 / 3.0) : mu_at;
    }
    if (g.gr2) {             // the GR D2 variant: mu = 1 in its chains and equation
      mu_a = mu_b = 1.0;
      mu_at = mu_bt = 0.0;
    } else if (GEO == 0) {
      br = mu_k - B;
      if (TAN) brt = mu_kt - B * (-2.0 + b.m2 * rpk + 2.0 * b.m2 * rpa);
    } else {
      const double G = b.m2 * rpk;
      const double lin = 2.0 * g.c2 * (mu_a + mu_b - 2.0) + (g.c / g.r) * (mu_a - 1.0) + g.r * g.c * (mu_b - 1.0);
      br = (mu_k - g.c2 * (mu_a + mu_b - mu_k) + G * lin - B) * g.inv_s2;
      if (TAN) {
        const double Gt = -G * q * rpk;
        const double lint = 2.0 * g.c2 * (mu_at + mu_bt) + (g.c / g.r) * mu_at + g.r * g.c * mu_bt;
        const double Bt = B * (-2.0 + b.m2 * rpk + b.m2 * rpa + b.m2 * rpb);
        brt = (mu_kt - g.c2 * (mu_at + mu_bt - mu_kt) + Gt * lin + G * lint - Bt) * g.inv_s2;
      }
    }
  }
  const double mu_2 = g.gr2 ? 1.0 : mu_k, mu_2t = g.gr2 ? 0.0 : mu_kt;
  // D1(k1) D1(k2) of the source (Winther: D1(k)^2)
  const double Pa = g.winther ? y[0] : y[L::A], Pb = g.winther ? y[0] : y[L::B];
  dy[0] = y[1];
  dy[1] = -b.damp * y[1] + b.cc * mu_k * y[0];
  dy[L::A] = y[L::A + 1];
  dy[L::A + 1] = -b.damp * y[L::A + 1] + b.cc * mu_a * y[L::A];
  if (GEO == 2) {
    dy[L::B] = y[L::B + 1];
    dy[L::B + 1] = -b.damp * y[L::B + 1] + b.cc * mu_b * y[L::B];
  }
  dy[L::D2] = y[L::D2 + 1];
  dy[L::D2 + 1] = -b.damp * y[L::D2 + 1] + b.cc * mu_2 * y[L::D2] - b.cc * Pa * Pb * br;
  if (TAN) {
    const double Pat = g.winther ? y[T] : y[T + L::A], Pbt = g.winther ? y[T] : y[T + L::B];
    dy[T] = y[T + 1];
    dy[T + 1] = -b.damp * y[T + 1] + b.cc * (mu_k * y[T] + mu_kt * y[0]);
    dy[T + L::A] = y[T + L::A + 1];
    dy[T + L::A + 1] = -b.damp * y[T + L::A + 1] + b.cc * (mu_a * y[T + L::A] + mu_at * y[L::A]);
    if (GEO == 2) {
      dy[T + L::B] = y[T + L::B + 1];
      dy[T + L::B + 1] = -b.damp * y[T + L::B + 1] + b.cc * (mu_b * y[T + L::B] + mu_bt * y[L::B]);
    }
    dy[T + L::D2] = y[T + L::D2 + 1];
    dy[T + L::D2 + 1] = -b.damp * y[T + L::D2 + 1] + b.cc * (mu_2 * y[T + L::D2] + mu_2t * y[L::D2]) -
                        b.cc * ((Pat * Pb + Pa * Pbt) * br + Pa * Pb * brt);
  }
}

template <int NY, bool TAN, int GEO>
__device__ void rk4(const Bg* tab, int n_steps, double h, double k2, bool gr, const D2Geo& g, double* y) {
  double k1[NY], k2v[NY], k3[NY], k4[NY], t[NY];
  for (int i = 0; i < n_steps; ++i) {
    const Bg& b0 = tab[2 * i];
    const Bg& bm = tab[2 * i + 1];
    const Bg& b1 = tab[2 * i + 2];
    rhs<TAN, GEO>(b0, k2, gr, g, y, k1);
#pragma unroll
    for (int j = 0; j < NY; ++j) t[j] = y[j] + 0.5 * h * k1[j];
    rhs<TAN, GEO>(bm, k2, gr, g, t, k2v);
#pragma unroll
    for (int j = 0; j < NY; ++j) t[j] = y[j] + 0.5 * h * k2v[j];
    rhs<TAN, GEO>(bm, k2, gr, g, t, k3);
#pragma unroll
    for (int j = 0; j < NY; ++j) t[j] = y[j] + h * k3[j];
    rhs<TAN, GEO>(b1, k2, gr, g, t, k4);
#pragma unroll
    for (int j = 0; j < NY; ++j) y[j] = y[j] + (h / 6.0) * (k1[j] + 2.0 * k2v[j] + 2.0 * k3[j] + k4[j]);
  }
}

__device__ void fill_bg(Bg* tab, const GrowthParams& p, double s0, double h, int n_steps, bool gr) {
  for (int j = threadIdx.x; j <= 2 * n_steps; j += blockDim.x) {
    const int i = j >> 1;
    const double s = (j & 1) ? (s0 + i * h) + 0.5 * h : s0 + i * h;
    tab[j] = background(p, s, gr);
  }
}

template <bool TAN, int GEO>
__global__ void k_growth(GrowthParams p, double* tab, float* tabf) {
  using L = Layout<GEO>;
  extern __shared__ Bg s_bg[];
  if (p.fr0s) p.fr0_abs = p.fr0s[blockIdx.y];     // instance blockIdx.y
  tab += (size_t)blockIdx.y * 4 * p.nk;
  tabf += (size_t)blockIdx.y * 4 * p.nk;
  const bool gr = (p.fr0_abs == 0.0);
  const D2Geo geo = d2_geo(p.d2_variant);
  const double s0 = log(p.a_init);
  // GR normalisation D1_GR(a = 1)
  const double hg = (0.0 - s0) / p.n_steps;
  fill_bg(s_bg, p, s0, hg, p.n_steps, true);
  __syncthreads();
  double g[6] = {p.a_init, p.a_init, p.a_init, p.a_init, 0.0, 0.0};
  rk4<6, false, 0>(s_bg, p.n_steps, hg, 1.0, true, d2_geo(0), g);
  const double norm = g[0];
  __syncthreads();
  const double h = (log(p.a_out) - s0) / p.n_steps;
  fill_bg(s_bg, p, s0, h, p.n_steps, gr);
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.nk) return;
  const double k = p.k_min * pow(p.k_max / p.k_min, (double)t / (double)(p.nk - 1));
  constexpr int NY = TAN ? 2 * L::NB : L::NB;
  double y[NY];
#pragma unroll
  for (int j = 0; j < NY; ++j) y[j] = 0.0;
#pragma unroll
  for (int j = 0; j < L::D2; ++j) y[j] = p.a_init;
  y[L::D2] = -3.0 / 7.0 * p.a_init * p.a_init;
  y[L::D2 + 1] = -6.0 / 7.0 * p.a_init * p.a_init;
  rk4<NY, TAN, GEO>(s_bg, p.n_steps, h, k * k, gr, geo, y);
  const int nk = p.nk;
  const int T = L::NB;
  tab[t] = y[0] / norm;
  tab[nk + t] = y[L::D2] / (norm * norm);
  tab[2 * nk + t] = TAN ? y[T] / norm : 0.0;
  tab[3 * nk + t] = TAN ? y[T + L::D2] / (norm * norm) : 0.0;
  if (geo.fit) {   // D2 = -(3/7) D1^2 Omega_m(a)^(-1/143), tangent -(6/7) D1 dD1 Omega_m(a)^(-1/143)
    const double a3 = 1.0 / (p.a_out * p.a_out * p.a_out);
    const double f = pow(p.omega_m * a3 / (p.omega_m * a3 + p.omega_l), -1.0 / 143.0);
    tab[nk + t] = -3.0 / 7.0 * tab[t] * tab[t] * f;
    tab[3 * nk + t] = -6.0 / 7.0 * tab[t] * tab[2 * nk + t] * f;
  }
  tabf[t] = (float)(y[0] / norm);
  tabf[nk + t] = (float)tab[nk + t];
  tabf[2 * nk + t] = (float)tab[2 * nk + t];
  tabf[3 * nk + t] = (float)tab[3 * nk + t];
}

#ifndef LPT2_GROWTH_THREADS
#define LPT2_GROWTH_THREADS 32   // k nodes per block (measured best: the RK4 chains are FP64-latency bound)
#endif
template <int GEO>
static cudaError_t launch_growth_geo(const GrowthParams& p, double* tab, float* tabf, cudaStream_t s) {
  const int threads = LPT2_GROWTH_THREADS;
  const int blocks = (p.nk + threads - 1) / threads;
  const size_t smem = (size_t)(2 * p.n_steps + 1) * sizeof(Bg);
  cudaFuncSetAttribute(k_growth<true, GEO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_growth<true, GEO><<<dim3(blocks, p.n_inst > 0 ? p.n_inst : 1), threads, smem, s>>>(p, tab, tabf);
  return cudaGetLastError();
}

cudaError_t launch_growth(const GrowthParams& p, double* tab, float* tabf, cudaStream_t s) {
  const D2Geo g = d2_geo(p.d2_variant);
  if (g.r != 1.0) return launch_growth_geo<2>(p, tab, tabf, s);
  if (g.c != 0.0) return launch_growth_geo<1>(p, tab, tabf, s);
  return launch_growth_geo<0>(p, tab, tabf, s);
}

// ------------------------------------------------------------- mode tables
// For every integer |n|^2 of an n^3 grid: k = (2 pi / L) sqrt(|n|^2),
//   x = sqrt(P_lin(k) N^3 / V)  (EH no-wiggle, sigma_8 amplitude),
//   y = 1 / (k^2 N^3),
//   z, w = D1(k), D2(k) and (mt1) dD1, dD2 / dln|fR0|, linear in ln k between the
// growth-table nodes and clamped at the ends - all in FP64, rounded once.
__device__ double interp_lnk64(const double* t, int nk, double lnkmin, double dlnk, double lnk) {
  double x = (lnk - lnkmin) / dlnk;
  if (x <= 0.0) return t[0];
  if (x >= (double)(nk - 1)) return t[nk - 1];
  int i = (int)x;
  if (i > nk - 2) i = nk - 2;
  const double f = x - (double)i;
  return t[i] + f * (t[i + 1] - t[i]);
}

__global__ void k_mode_tables(GrowthParams p, const DevCosmo* cosmo, const double* tab, int inst0, int n, double box,
                              float4* mt0, float2* mt1) {
  const int len = mode_table_len(n);
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= len) return;
  const int inst = inst0 + blockIdx.y;
  const double* tb = tab + (size_t)inst * 4 * p.nk;
  float4* o0 = mt0 + (size_t)blockIdx.y * len;
  float2* o1 = mt1 + (size_t)blockIdx.y * len;
  if (idx == 0) {
    o0[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    o1[0] = make_float2(0.f, 0.f);
    return;
  }
  const double nd = n, kf = 2.0 * M_PI / box;
  const double k = kf * sqrt((double)idx);
  const EhConst c = eh_constants(p);
  const double T = eh_T64(c, k, p.h);
  const double sp = sqrt(cosmo->amp) * pow(k, 0.5 * p.n_s) * T * sqrt(nd * nd * nd / (box * box * box));
  const double inv = 1.0 / (k * k * nd * nd * nd);
  const double lnkmin = log(p.k_min), dlnk = (log(p.k_max) - log(p.k_min)) / (p.nk - 1), lk = log(k);
  const double d1 = interp_lnk64(tb, p.nk, lnkmin, dlnk, lk);
  const double d2 = interp_lnk64(tb + p.nk, p.nk, lnkmin, dlnk, lk);
  const double t1 = interp_lnk64(tb + 2 * p.nk, p.nk, lnkmin, dlnk, lk);
  const double t2 = interp_lnk64(tb + 3 * p.nk, p.nk, lnkmin, dlnk, lk);
  o0[idx] = make_float4((float)sp, (float)inv, (float)d1, (float)d2);
  o1[idx] = make_float2((float)t1, (float)t2);
}

cudaError_t launch_mode_tables(const GrowthParams& p, const DevCosmo* cosmo, const double* tab, int inst0, int count,
                               int n, double box, float4* mt0, float2* mt1, cudaStream_t s) {
  const int len = mode_table_len(n);
  k_mode_tables<<<dim3((len + 127) / 128, count), 128, 0, s>>>(p, cosmo, tab, inst0, n, box, mt0, mt1);
  return cudaGetLastError();
}

}  // namespace lpt2
