// Size-independent kernels: CIC deposit from positions, zero fill, P(k) shell
// finalisation, white noise and raw Philox words.
#include "passes.cuh"

namespace lpt2 {

// Periodic cloud-in-cell deposit of unit-mass particles (one thread per particle).
template <int N>
__global__ void __launch_bounds__(256) k_cic(CicArgs a) {
  const size_t n3 = (size_t)N * N * N;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;   // grid covers n3 exactly
  a.pos += (size_t)blockIdx.y * 3 * n3;                               // instance blockIdx.y
  a.rho += (size_t)blockIdx.y * n3;
  float u[3];
  for (int c = 0; c < 3; ++c) u[c] = wrapN<N>(__ldg(a.pos + c * n3 + i) * a.g.inv_cell);
  cic_deposit_vec<N>(a.rho, u[0], u[1], u[2]);   // fastest of scalar / neighbour-merged / vector on real positions
}

cudaError_t launch_cic(const CicArgs& a, cudaStream_t s) {
  const size_t n3 = (size_t)a.g.n * a.g.n * a.g.n;   // every supported N^3 is a multiple of 256
  if (a.g.batch < 1 || a.g.batch > 65535) return cudaErrorInvalidValue;
  const dim3 blocks((unsigned)(n3 / 256), a.g.batch);
  switch (a.g.n) {
    case 16: k_cic<16><<<blocks, 256, 0, s>>>(a); break;
    case 32: k_cic<32><<<blocks, 256, 0, s>>>(a); break;
    case 64: k_cic<64><<<blocks, 256, 0, s>>>(a); break;
    case 96: k_cic<96><<<blocks, 256, 0, s>>>(a); break;
    case 128: k_cic<128><<<blocks, 256, 0, s>>>(a); break;
    case 192: k_cic<192><<<blocks, 256, 0, s>>>(a); break;
    case 256: k_cic<256><<<blocks, 256, 0, s>>>(a); break;
    case 512: k_cic<512><<<blocks, 256, 0, s>>>(a); break;
    default: k_cic<1024><<<blocks, 256, 0, s>>>(a); break;
  }
  return cudaGetLastError();
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

__global__ void k_noise(int n, uint32_t k0, uint32_t k1, float* out) {
  const size_t n3 = (size_t)n * n * n;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
    const bool odd = ((i / n) % n) & 1;   // iy odd: sine output of the draw at iy - 1
    const float2 g2 = philox_gauss2(odd ? i - n : i, k0, k1);
    out[i] = odd ? g2.y : g2.x;
  }
}

cudaError_t launch_noise(const Geo& g, uint32_t k0, uint32_t k1, float* out, cudaStream_t s) {
  k_noise<<<152 * 8, 256, 0, s>>>(g.n, k0, k1, out);
  return cudaGetLastError();
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
