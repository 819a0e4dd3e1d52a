// Size-independent kernels: CIC deposit from positions, zero fill, P(k) shell
// finalisation, white noise and raw Philox words.
#include <math.h>

#include "passes.cuh"

namespace lpt2 {

// Periodic cloud-in-cell deposit of unit-mass particles (Sec. 4 density),
// Lagrangian-tile form.  A CTA takes the CIC_T^3 particles of one block of
// Lagrangian cells.  Their positions mostly stay within CIC_H cells of the block,
// so the CTA sums the eight weights of each such particle in a shared-memory window
// (the block grown by CIC_H cells on every side, by a 4-aligned CIC_HZ below in z)
// and then adds the window to the density with one 16-byte vector reduction per
// non-zero group of four cells: about one L2 reduction per particle instead of the
// five of a direct deposit, whose rate the L2 request throughput limits.  Window
// sums are integers in units of 2^-19 of a particle mass (integer shared atomics;
// a window cell receives at most the block's 4096 masses < 2^13, so the sum cannot
// overflow; each weight is rounded by at most 2^-20).  Particles displaced further
// than the halo are deposited directly.
#ifndef LPT2_CIC_MINB
#define LPT2_CIC_MINB 2   // resident CIC CTAs per SM: register cap (3 fit in shared memory but spill)
#endif
namespace {
constexpr int CIC_T = 16, CIC_H = 4, CIC_HZ = 4;
constexpr int CIC_E = CIC_T + 2 * CIC_H + 1;                        // window cells along x and y
constexpr int CIC_EZ = (CIC_T + CIC_HZ + CIC_H + 1 + 3) / 4 * 4;    // along z, whole groups of 4
constexpr int CIC_QZ = CIC_EZ / 4;
constexpr int CIC_THREADS = 512;
constexpr int CIC_PER = CIC_T * CIC_T * CIC_T / CIC_THREADS;         // particles per thread
constexpr int CIC_SMEM = CIC_E * CIC_E * CIC_EZ * 4;
constexpr float CIC_SCALE = 524288.0f;                              // 2^19
static_assert(CIC_HZ % 4 == 0 && CIC_T % 4 == 0, "window groups of four must align with the grid's");
static_assert(CIC_T * CIC_T * CIC_T < (1 << 13), "window sums must stay below 2^32 / 2^19");
}  // namespace

template <int N>
__device__ __forceinline__ int wrap_cell(int i) {   // i in (-N, 2N) -> [0, N)
  return i < 0 ? i + N : (i >= N ? i - N : i);
}

template <int N>
__global__ void __launch_bounds__(CIC_THREADS, LPT2_CIC_MINB) k_cic(CicArgs a) {
  static_assert(N % CIC_T == 0 && N % 4 == 0, "grid side must be a multiple of the tile");
  extern __shared__ __align__(16) unsigned int win[];   // [CIC_E][CIC_E][CIC_EZ]
  const size_t n3 = (size_t)N * N * N;
  a.pos += (size_t)blockIdx.y * 3 * n3;   // instance blockIdx.y
  a.rho += (size_t)blockIdx.y * n3;
  constexpr int NT = N / CIC_T;
  const int b = blockIdx.x;
  const int x0 = (b / (NT * NT)) * CIC_T, y0 = ((b / NT) % NT) * CIC_T, z0 = (b % NT) * CIC_T;
  const int ox = x0 - CIC_H, oy = y0 - CIC_H, oz = z0 - CIC_HZ;   // window origin (may be < 0)
  const bool wraps = ox < 0 || oy < 0 || oz < 0 || ox + CIC_E > N || oy + CIC_E > N || oz + CIC_EZ > N;
  // all position loads of this thread first: their latency overlaps the zeroing
  float u[CIC_PER][3];
#pragma unroll
  for (int k = 0; k < CIC_PER; ++k) {
    const int p = threadIdx.x + k * CIC_THREADS;
    const int i = p / (CIC_T * CIC_T), j = (p / CIC_T) % CIC_T, l = p % CIC_T;
    const size_t e = ((size_t)(x0 + i) * N + (y0 + j)) * N + (z0 + l);
#pragma unroll
    for (int c = 0; c < 3; ++c) u[k][c] = __ldg(a.pos + c * n3 + e);
  }
  for (int i = threadIdx.x; i < CIC_E * CIC_E * CIC_QZ; i += blockDim.x)
    reinterpret_cast<uint4*>(win)[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
#pragma unroll
  for (int k = 0; k < CIC_PER; ++k) {
    const float ux = wrapN<N>(u[k][0] * a.g.inv_cell + a.shift);
    const float uy = wrapN<N>(u[k][1] * a.g.inv_cell + a.shift);
    const float uz = wrapN<N>(u[k][2] * a.g.inv_cell + a.shift);
    const float fx = floorf(ux), fy = floorf(uy), fz = floorf(uz);
    // window cell of the lower corner: offset from the origin, periodic only for a window
    // that crosses the grid boundary (elsewhere a negative offset is simply outside)
    int rx = (int)fx - ox, ry = (int)fy - oy, rz = (int)fz - oz;
    if (wraps) {
      rx = wrap_cell<N>(rx);
      ry = wrap_cell<N>(ry);
      rz = wrap_cell<N>(rz);
    }
    if ((unsigned)rx < CIC_E - 1 && (unsigned)ry < CIC_E - 1 && (unsigned)rz < CIC_EZ - 1) {
      const float dx = ux - fx, dy = uy - fy, dz = uz - fz;   // exact
      const float wx0 = 1.f - dx, wy0 = 1.f - dy, wz0 = 1.f - dz;
      unsigned int* c = win + (rx * CIC_E + ry) * CIC_EZ + rz;
      float w = wx0 * wy0;
      atomicAdd(c, __float2uint_rn(w * wz0 * CIC_SCALE));
      atomicAdd(c + 1, __float2uint_rn(w * dz * CIC_SCALE));
      w = wx0 * dy;
      atomicAdd(c + CIC_EZ, __float2uint_rn(w * wz0 * CIC_SCALE));
      atomicAdd(c + CIC_EZ + 1, __float2uint_rn(w * dz * CIC_SCALE));
      w = dx * wy0;
      atomicAdd(c + CIC_E * CIC_EZ, __float2uint_rn(w * wz0 * CIC_SCALE));
      atomicAdd(c + CIC_E * CIC_EZ + 1, __float2uint_rn(w * dz * CIC_SCALE));
      w = dx * dy;
      atomicAdd(c + CIC_E * CIC_EZ + CIC_EZ, __float2uint_rn(w * wz0 * CIC_SCALE));
      atomicAdd(c + CIC_E * CIC_EZ + CIC_EZ + 1, __float2uint_rn(w * dz * CIC_SCALE));
    } else {
      cic_deposit_vec<N>(a.rho, ux, uy, uz);
    }
  }
  __syncthreads();
  const float inv_scale = 1.0f / CIC_SCALE;
  // group q = (wx * CIC_E + wy) * CIC_QZ + qz, advanced by the CTA size without divisions
  static_assert(CIC_THREADS / CIC_QZ / CIC_E < CIC_E, "flush stride must advance wx by less than a window");
  constexpr int SQZ = CIC_THREADS % CIC_QZ, SR = CIC_THREADS / CIC_QZ;   // stride in (qz, row)
  constexpr int SWY = SR % CIC_E, SWX = SR / CIC_E;                      // row stride in (wy, wx)
  int qz = threadIdx.x % CIC_QZ, wy = (threadIdx.x / CIC_QZ) % CIC_E, wx = threadIdx.x / CIC_QZ / CIC_E;
  for (int q = threadIdx.x; q < CIC_E * CIC_E * CIC_QZ; q += blockDim.x) {
    const uint4 iv = reinterpret_cast<const uint4*>(win)[q];
    const int cz = qz, cy = wy, cx = wx;
    qz += SQZ;
    wy += SWY;
    wx += SWX;
    if (qz >= CIC_QZ) { qz -= CIC_QZ; ++wy; }
    if (wy >= CIC_E) { wy -= CIC_E; ++wx; }
    if ((iv.x | iv.y | iv.z | iv.w) == 0u) continue;
    int gx = ox + cx, gy = oy + cy, gz = oz + 4 * cz;   // gz a multiple of 4: the group never straddles the wrap
    if (wraps) {
      gx = wrap_cell<N>(gx);
      gy = wrap_cell<N>(gy);
      gz = wrap_cell<N>(gz);
    }
    atomicAdd(reinterpret_cast<float4*>(a.rho + ((size_t)gx * N + gy) * N + gz),
              make_float4((float)iv.x * inv_scale, (float)iv.y * inv_scale, (float)iv.z * inv_scale,
                          (float)iv.w * inv_scale));
  }
}

// Transpose of the CIC deposit, tile by tile like k_cic: the CTA of a Lagrangian CIC_T^3
// tile loads the window of dL/d(density) around it into shared memory (coalesced groups
// of four along z) and each particle gathers the derivative of its eight CIC weights,
//   dL/dx = (1/h) sum_corners g_c (+-1) w_y w_z   (and y, z alike),
// from the window; a particle outside the window gathers from global memory.  The
// three components go to real fields at the particle's Lagrangian cell.
template <int N>
__global__ void __launch_bounds__(CIC_THREADS, LPT2_CIC_MINB) k_cic_grad(CicGradArgs a) {
  static_assert(N % CIC_T == 0 && N % 4 == 0, "grid side must be a multiple of the tile");
  extern __shared__ __align__(16) float gw[];   // [CIC_E][CIC_E][CIC_EZ]
  const size_t n3 = (size_t)N * N * N;
  constexpr int NT = N / CIC_T;
  const int b = blockIdx.x;
  const int x0 = (b / (NT * NT)) * CIC_T, y0 = ((b / NT) % NT) * CIC_T, z0 = (b % NT) * CIC_T;
  const int ox = x0 - CIC_H, oy = y0 - CIC_H, oz = z0 - CIC_HZ;
  const bool wraps = ox < 0 || oy < 0 || oz < 0 || ox + CIC_E > N || oy + CIC_E > N || oz + CIC_EZ > N;
  float u[CIC_PER][3];
#pragma unroll
  for (int k = 0; k < CIC_PER; ++k) {
    const int p = threadIdx.x + k * CIC_THREADS;
    const int i = p / (CIC_T * CIC_T), j = (p / CIC_T) % CIC_T, l = p % CIC_T;
    const size_t e = ((size_t)(x0 + i) * N + (y0 + j)) * N + (z0 + l);
#pragma unroll
    for (int c = 0; c < 3; ++c) u[k][c] = __ldg(a.pos + c * n3 + e);
  }
  // group q = (wx * CIC_E + wy) * CIC_QZ + qz, advanced by the CTA size without divisions
  constexpr int SQZ = CIC_THREADS % CIC_QZ, SR = CIC_THREADS / CIC_QZ;
  constexpr int SWY = SR % CIC_E, SWX = SR / CIC_E;
  int qz = threadIdx.x % CIC_QZ, wy = (threadIdx.x / CIC_QZ) % CIC_E, wx = threadIdx.x / CIC_QZ / CIC_E;
  for (int q = threadIdx.x; q < CIC_E * CIC_E * CIC_QZ; q += blockDim.x) {
    int gx = ox + wx, gy = oy + wy, gz = oz + 4 * qz;   // gz a multiple of 4
    qz += SQZ;
    wy += SWY;
    wx += SWX;
    if (qz >= CIC_QZ) { qz -= CIC_QZ; ++wy; }
    if (wy >= CIC_E) { wy -= CIC_E; ++wx; }
    if (wraps) {
      gx = wrap_cell<N>(gx);
      gy = wrap_cell<N>(gy);
      gz = wrap_cell<N>(gz);
    }
    reinterpret_cast<float4*>(gw)[q] = __ldg(reinterpret_cast<const float4*>(a.grho + ((size_t)gx * N + gy) * N + gz));
  }
  __syncthreads();
  const float ic = a.g.inv_cell;
#pragma unroll
  for (int k = 0; k < CIC_PER; ++k) {
    const int p = threadIdx.x + k * CIC_THREADS;
    const int i = p / (CIC_T * CIC_T), j = (p / CIC_T) % CIC_T, l = p % CIC_T;
    const size_t e = ((size_t)(x0 + i) * N + (y0 + j)) * N + (z0 + l);
    const float ux = wrapN<N>(u[k][0] * ic), uy = wrapN<N>(u[k][1] * ic), uz = wrapN<N>(u[k][2] * ic);
    const float fx = floorf(ux), fy = floorf(uy), fz = floorf(uz);
    int rx = (int)fx - ox, ry = (int)fy - oy, rz = (int)fz - oz;
    if (wraps) {
      rx = wrap_cell<N>(rx);
      ry = wrap_cell<N>(ry);
      rz = wrap_cell<N>(rz);
    }
    float gxv, gyv, gzv;
    if ((unsigned)rx < CIC_E - 1 && (unsigned)ry < CIC_E - 1 && (unsigned)rz < CIC_EZ - 1) {
      const float dx = ux - fx, dy = uy - fy, dz = uz - fz;
      const float wx[2] = {1.f - dx, dx}, wy[2] = {1.f - dy, dy}, wz[2] = {1.f - dz, dz};
      const float* c = gw + (rx * CIC_E + ry) * CIC_EZ + rz;
      float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
      for (int cx = 0; cx < 2; ++cx)
#pragma unroll
        for (int cy = 0; cy < 2; ++cy)
#pragma unroll
          for (int cz = 0; cz < 2; ++cz) {
            const float gc = c[(cx * CIC_E + cy) * CIC_EZ + cz];
            const float sx = cx ? 1.f : -1.f, sy = cy ? 1.f : -1.f, sz = cz ? 1.f : -1.f;
            ax = fmaf(gc * sx, wy[cy] * wz[cz], ax);
            ay = fmaf(gc * sy, wx[cx] * wz[cz], ay);
            az = fmaf(gc * sz, wx[cx] * wy[cy], az);
          }
      gxv = ax * ic;
      gyv = ay * ic;
      gzv = az * ic;
    } else {
      cic_gather_grad<N>(a.grho, a.pos, e, n3, ic, gxv, gyv, gzv);
    }
    if (a.gpos) {
      gxv += __ldg(a.gpos + e);
      gyv += __ldg(a.gpos + n3 + e);
      gzv += __ldg(a.gpos + 2 * n3 + e);
    }
    a.gx[e] = gxv;
    a.gy[e] = gyv;
    a.gz[e] = gzv;
  }
}

template <int N>
cudaError_t launch_cic_grad_n(const CicGradArgs& a, cudaStream_t s) {
  cudaFuncSetAttribute(k_cic_grad<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, CIC_SMEM);
  k_cic_grad<N><<<(unsigned)((N / CIC_T) * (N / CIC_T) * (N / CIC_T)), CIC_THREADS, CIC_SMEM, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_cic_grad(const CicGradArgs& a, cudaStream_t s) {
  if (a.g.batch != 1) return cudaErrorInvalidValue;
  switch (a.g.n) {
    case 16: return launch_cic_grad_n<16>(a, s);
    case 32: return launch_cic_grad_n<32>(a, s);
    case 64: return launch_cic_grad_n<64>(a, s);
    case 96: return launch_cic_grad_n<96>(a, s);
    case 128: return launch_cic_grad_n<128>(a, s);
    case 192: return launch_cic_grad_n<192>(a, s);
    case 256: return launch_cic_grad_n<256>(a, s);
    case 512: return launch_cic_grad_n<512>(a, s);
    case 1024: return launch_cic_grad_n<1024>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int N>
cudaError_t launch_cic_n(const CicArgs& a, cudaStream_t s) {
  cudaFuncSetAttribute(k_cic<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, CIC_SMEM);
  const dim3 blocks((unsigned)((N / CIC_T) * (N / CIC_T) * (N / CIC_T)), a.g.batch);
  k_cic<N><<<blocks, CIC_THREADS, CIC_SMEM, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_cic(const CicArgs& a, cudaStream_t s) {
  if (a.g.batch < 1 || a.g.batch > 65535) return cudaErrorInvalidValue;
  switch (a.g.n) {
    case 16: return launch_cic_n<16>(a, s);
    case 32: return launch_cic_n<32>(a, s);
    case 64: return launch_cic_n<64>(a, s);
    case 96: return launch_cic_n<96>(a, s);
    case 128: return launch_cic_n<128>(a, s);
    case 192: return launch_cic_n<192>(a, s);
    case 256: return launch_cic_n<256>(a, s);
    case 512: return launch_cic_n<512>(a, s);
    case 1024: return launch_cic_n<1024>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

__global__ void k_fill0(float4* p, size_t n4) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x)
    p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

cudaError_t launch_fill0(float* p, size_t n, cudaStream_t s) {
  // n is a multiple of 4 for every buffer of this library (N >= 16)
  k_fill0<<<152 * 8, 256, 0, s>>>(reinterpret_cast<float4*>(p), n / 4);
  return cudaGetLastError();
}

// density contrast delta = rho N^3 / N_p - 1 with one particle per cell
__global__ void k_contrast(const float* __restrict__ rho, float* __restrict__ out, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = rho[i] - 1.0f;
}

cudaError_t launch_contrast(const float* rho, float* out, size_t n, cudaStream_t s) {
  k_contrast<<<152 * 8, 256, 0, s>>>(rho, out, n);
  return cudaGetLastError();
}

// One block per shell: fixed-order strided sums then a tree (deterministic).
__global__ void k_pk_finalize(const double* part, int n_blocks, int ns, double* pk, double* kmean,
                              int64_t* nmodes) {
  const int b = blockIdx.x;
  part += (size_t)blockIdx.y * n_blocks * 3 * ns;       // instance blockIdx.y
  pk += (size_t)blockIdx.y * ns;
  if (kmean) kmean += (size_t)blockIdx.y * ns;
  if (nmodes) nmodes += (size_t)blockIdx.y * ns;
  double sp = 0.0, sk = 0.0, sc = 0.0;
  // unrolled: eight rows' loads in flight per thread; the adds keep their order
#pragma unroll 8
  for (int i = threadIdx.x; i < n_blocks; i += blockDim.x) {
    const double* q = part + (size_t)i * 3 * ns;
    sp += q[b];
    sk += q[ns + b];
    sc += q[2 * ns + b];
  }
  __shared__ double s[3][256];
  s[0][threadIdx.x] = sp;
  s[1][threadIdx.x] = sk;
  s[2][threadIdx.x] = sc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s[0][threadIdx.x] += s[0][threadIdx.x + o];
      s[1][threadIdx.x] += s[1][threadIdx.x + o];
      s[2][threadIdx.x] += s[2][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double c = s[2][0];
    pk[b] = c > 0 ? s[0][0] / c : 0.0;
    if (kmean) kmean[b] = c > 0 ? s[1][0] / c : 0.0;
    if (nmodes) nmodes[b] = (int64_t)(c + 0.5);
  }
}

cudaError_t launch_pk_finalize(const double* part, int n_blocks, int n_shells, double* pk, double* k_mean,
                               int64_t* n_modes, cudaStream_t s, int batch) {
  k_pk_finalize<<<dim3(n_shells, batch), 256, 0, s>>>(part, n_blocks, n_shells, pk, k_mean, n_modes);
  return cudaGetLastError();
}

// Shell geometry of the P(k) estimator: for every mode of the stored half spectrum
// (kz < N/2; kz > 0 stands for itself and its conjugate, so it counts twice) with
// 0 < |n| < N/2, shell b = floor(2 n_shells |n| / N) by exact integer comparison,
// the weighted mode count and sum of |k|.  One thread per (kx, ky) walks kz, where
// |n| grows monotonically, and flushes its running sums when the shell changes.
__device__ __forceinline__ int shell_index_int(long long n2, int n, int ns) {
  // largest b with (b n)^2 <= 4 ns^2 n2
  const long long M = 4LL * ns * ns * n2;
  int b = (int)(sqrtf((float)n2) * (2.0f * (float)ns / (float)n));
  while (b > 0 && (long long)b * n * (long long)b * n > M) --b;
  while ((long long)(b + 1) * n * (long long)(b + 1) * n <= M) ++b;
  return b;
}

__global__ void k_shell_geometry(int n, float kf, int ns, double* ksum, unsigned long long* count) {
  extern __shared__ double s_geo[];   // [ns] |k| sums, then [ns] counts
  unsigned long long* s_cnt = reinterpret_cast<unsigned long long*>(s_geo + ns);
  for (int i = threadIdx.x; i < ns; i += blockDim.x) { s_geo[i] = 0.0; s_cnt[i] = 0ull; }
  __syncthreads();
  const int h = n / 2;
  const int ky = blockIdx.x;
  const int my = ky < h ? ky : ky - n;
  for (int kx = threadIdx.x; kx < n; kx += blockDim.x) {
    const int mx = kx < h ? kx : kx - n;
    int cur = -1;
    double ks = 0.0;
    unsigned long long c = 0;
    for (int kz = 0; kz < h; ++kz) {
      const long long n2 = (long long)mx * mx + (long long)my * my + (long long)kz * kz;
      if (n2 == 0 || 4 * n2 >= (long long)n * n) continue;
      const int b = shell_index_int(n2, n, ns);
      if (b != cur) {
        if (cur >= 0) { atomicAdd(&s_geo[cur], ks); atomicAdd(&s_cnt[cur], c); }
        cur = b;
        ks = 0.0;
        c = 0;
      }
      const unsigned w = kz == 0 ? 1u : 2u;
      ks += (double)w * (double)(kf * sqrtf((float)n2));   // n2 < 2^24: exact in FP32
      c += w;
    }
    if (cur >= 0) { atomicAdd(&s_geo[cur], ks); atomicAdd(&s_cnt[cur], c); }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ns; i += blockDim.x) {
    if (s_cnt[i]) {
      atomicAdd(&ksum[i], s_geo[i]);
      atomicAdd(&count[i], s_cnt[i]);
    }
  }
}

cudaError_t launch_shell_geometry(int n, double box, int n_shells, double* ksum, unsigned long long* nmodes,
                                  cudaStream_t s) {
  const float kf = (float)(2.0 * M_PI / box);
  k_shell_geometry<<<n, 128, n_shells * 16, s>>>(n, kf, n_shells, ksum, nmodes);
  return cudaGetLastError();
}

// Shell sums of the per-block P partials in two fixed-order stages (the result does not
// depend on scheduling).  Stage 1: CTA (g, instance) takes rows [g R, g R + R) of the
// partials; thread (lane, b) = (tid / ns, tid % ns) sums rows lane, lane + L, ... of shell b
// (L = 256 / ns lanes; a warp reads consecutive shells of a row, i.e. contiguous doubles),
// then the lanes are summed in order into scratch[instance][g][b].  Stage 2 sums the G
// rows of scratch per shell (a warp per shell: strided lane sums, then a fixed shuffle
// tree) and divides by the shell's mode count.
__global__ void k_pk_rows(const double* __restrict__ part, int n_blocks, int ns, int rows, double* __restrict__ scratch) {
  const int g = blockIdx.x, inst = blockIdx.y;
  part += (size_t)inst * n_blocks * ns;
  const int L = blockDim.x / ns, lane = threadIdx.x / ns, b = threadIdx.x % ns;
  const int r0 = g * rows, r1 = min(n_blocks, r0 + rows);
  double acc = 0.0;
  if (lane < L) {
#pragma unroll 4
    for (int r = r0 + lane; r < r1; r += L) acc += part[(size_t)r * ns + b];
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < ns) {
    double sum = 0.0;
    for (int l = 0; l < L; ++l) sum += sh[l * ns + threadIdx.x];
    scratch[((size_t)inst * gridDim.x + g) * ns + threadIdx.x] = sum;
  }
}

__global__ void k_pk_finalize_p(const double* __restrict__ scratch, int G, int ns, const double* ksum,
                                const unsigned long long* count, double* pk, double* kmean, int64_t* nmodes) {
  const int inst = blockIdx.x, lane = threadIdx.x & 31;
  // a warp per shell: lane l sums rows l, l + 32, ... in order, then a fixed shuffle tree
  for (int b = threadIdx.x >> 5; b < ns; b += blockDim.x >> 5) {
    double sp = 0.0;
    for (int g = lane; g < G; g += 32) sp += scratch[((size_t)inst * G + g) * ns + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sp += __shfl_xor_sync(0xffffffffu, sp, o);
    if (lane == 0) {
      const double c = (double)count[b];
      pk[(size_t)inst * ns + b] = c > 0 ? sp / c : 0.0;
      if (kmean) kmean[(size_t)inst * ns + b] = c > 0 ? ksum[b] / c : 0.0;
      if (nmodes) nmodes[(size_t)inst * ns + b] = (int64_t)count[b];
    }
  }
}

cudaError_t launch_pk_finalize_p(const double* part, int n_blocks, int n_shells, const double* ksum,
                                 const unsigned long long* count, double* pk, double* k_mean, int64_t* n_modes,
                                 cudaStream_t s, int batch) {
  if (n_shells < 1 || n_shells > 256 || n_blocks < 1 || batch < 1 || batch > 65535) return cudaErrorInvalidValue;
  // the stage-1 sums follow the partials in their buffer (sized for three quantities per
  // row and shell, of which P uses one): batch * G * n_shells <= batch * n_blocks * n_shells
  const int G = n_blocks < 128 ? n_blocks : 128;
  const int rows = (n_blocks + G - 1) / G;
  double* scratch = const_cast<double*>(part) + (size_t)batch * n_blocks * n_shells;
  k_pk_rows<<<dim3(G, batch), 256, 0, s>>>(part, n_blocks, n_shells, rows, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_pk_finalize_p<<<batch, 256, 0, s>>>(scratch, G, n_shells, ksum, count, pk, k_mean, n_modes);
  return cudaGetLastError();
}

__global__ void k_noise(int n, uint32_t k0, uint32_t k1, const float4* __restrict__ g_bm, float* out) {
  __shared__ float4 bm[kBmTableLen];
  bm_load_table(bm, g_bm);
  __syncthreads();
  const size_t n3 = (size_t)n * n * n;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
    const bool odd = ((i / n) % n) & 1;   // iy odd: sine output of the draw at iy - 1
    const float2 g2 = philox_gauss2(odd ? i - n : i, k0, k1, bm);
    out[i] = odd ? g2.y : g2.x;
  }
}

cudaError_t launch_noise(const Geo& g, uint32_t k0, uint32_t k1, const float4* bm, float* out, cudaStream_t s) {
  k_noise<<<152 * 8, 256, 0, s>>>(g.n, k0, k1, bm, out);
  return cudaGetLastError();
}

__global__ void k_box_muller(const uint2* __restrict__ w, int64_t count, const float4* __restrict__ g_bm,
                             float2* out) {
  __shared__ float4 bm[kBmTableLen];
  bm_load_table(bm, g_bm);
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const uint2 x = w[i];
    out[i] = bm_pair(x.x, x.y, bm);
  }
}

cudaError_t launch_box_muller(const uint32_t* words, int64_t count, const float4* bm, float* out, cudaStream_t s) {
  k_box_muller<<<152 * 4, 256, 0, s>>>(reinterpret_cast<const uint2*>(words), count, bm,
                                       reinterpret_cast<float2*>(out));
  return cudaGetLastError();
}

// Bulk-tensor map of an x-pass input (see passes.h).  cuTensorMapEncodeTiled is a
// host-only driver call, resolved through the runtime (no link against the driver).
bool encode_x_tile_map(CUtensorMap* map, const void* base, int inner, int n, int box_inner, int batch) {
  typedef CUresult (*Encode)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode encode = nullptr;
  if (!encode) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !f)
      return false;
    encode = (Encode)f;
  }
  const cuuint64_t nn = (cuuint64_t)n, in = (cuuint64_t)inner;
  const cuuint64_t dims[4] = {in, nn, nn, (cuuint64_t)batch};                  // kz floats, ky, kx, instance
  const cuuint64_t strides[3] = {in * 4, in * nn * 4, in * nn * nn * 4};       // bytes of dims 1..3
  const cuuint32_t box[4] = {(cuuint32_t)box_inner, 1u, (cuuint32_t)(n > 256 ? 256 : n), 1u};
  const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// sqrt(P N^3/V) of every stored mode (kx, ky, kz < N/2) of `count` half spectra, from the
// instances' mode tables; zero on the modes the x passes zero (a Nyquist kx or ky, and the
// mean), so the field can stand in for the table entry with no test of its own.
__global__ void k_sc_field(const float4* __restrict__ mt0, int n, float* __restrict__ scf) {
  const int h = n / 2;
  const size_t per = (size_t)n * n * h;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= per) return;
  const int kz = (int)(e % h), ky = (int)((e / h) % n), kx = (int)(e / ((size_t)n * h));
  const int mx = mode_of(kx, n), my = mode_of(ky, n), mz = kz;
  const int n2 = mx * mx + my * my + mz * mz;
  const bool zero = ky == h || kx == h || n2 == 0;
  const size_t inst = blockIdx.y;
  scf[inst * per + e] = zero ? 0.f : mt0[inst * mode_table_len(n) + n2].x;
}

cudaError_t launch_sc_field(const float4* mt0, int n, int count, float* scf, cudaStream_t s) {
  const size_t per = (size_t)n * n * (n / 2);
  if (count < 1 || count > 65535) return cudaErrorInvalidValue;
  k_sc_field<<<dim3((unsigned)((per + 255) / 256), count), 256, 0, s>>>(mt0, n, scf);
  return cudaGetLastError();
}

// Box-Muller tables (layout in boxmuller.cuh): FP64 values, each split into the float
// nearest to it and the float nearest to the remainder.
void bm_table(float4* t) {
  auto split = [](double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
  };
  for (int j = 0; j < kBmSinCos; ++j) {
    const double a = M_PI * (double)j / 2048.0;   // 2 pi j / 4096
    split(cos(a), t[j].x, t[j].y);
    split(sin(a), t[j].z, t[j].w);
  }
  for (int j = kBmLogLo; j <= kBmLogHi; ++j) {
    const float c = (float)(1.0 / (1.0 + j / 128.0));
    float4& e = t[kBmLog0 + (j - kBmLogLo)];
    e.x = c;
    split(-log((double)c), e.y, e.z);
    e.w = 0.f;
  }
  float4& k = t[kBmConst];
  split(2.0 * M_PI, k.x, k.y);
  split(M_LN2, k.z, k.w);
}

__global__ void k_philox_words(uint32_t k0, uint32_t k1, uint64_t first, int64_t count, uint4* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t c = first + (uint64_t)i;
    out[i] = philox4x32_10(make_uint4((uint32_t)c, (uint32_t)(c >> 32), 0u, 0u), k0, k1);
  }
}

cudaError_t launch_philox_words(uint32_t k0, uint32_t k1, uint64_t first, int64_t count, uint32_t* out,
                                cudaStream_t s) {
  k_philox_words<<<152 * 4, 256, 0, s>>>(k0, k1, first, count, reinterpret_cast<uint4*>(out));
  return cudaGetLastError();
}

// Per-shell weight of the P(k) transpose: dP_b/d delta(k) = 2 V delta(k)/(N^6 c_b),
// so the density cotangent gains IDFT[w_b delta(k)] with w_b = 2 V g_pk[b] / (N^6 c_b).
__global__ void k_pk_adj_weights(const double* g_pk, const int64_t* n_modes, int ns, double v_over_n6,
                                 float* w) {
  for (int b = threadIdx.x; b < ns; b += blockDim.x) {
    const double c = (double)n_modes[b];
    w[b] = (c > 0 && g_pk) ? (float)(2.0 * v_over_n6 * g_pk[b] / c) : 0.f;
  }
}

cudaError_t launch_pk_adj_weights(const double* g_pk, const int64_t* n_modes, int n_shells, double v_over_n6,
                                  float* w, cudaStream_t s) {
  k_pk_adj_weights<<<1, 256, 0, s>>>(g_pk, n_modes, n_shells, v_over_n6, w);
  return cudaGetLastError();
}

// Deterministic sum of n FP64 partials (fixed-order strided sums, then a tree).
__global__ void k_sum_partials(const double* part, int n, double* out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
  __shared__ double s[256];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

cudaError_t launch_sum_partials(const double* part, int n, double* out, cudaStream_t s) {
  k_sum_partials<<<1, 256, 0, s>>>(part, n, out);
  return cudaGetLastError();
}

}  // namespace lpt2
