// Full second-order source term of Sec. 3 (Eqs. full, s1-s4) and its ratio to GR.
//
// Real-space sources, accumulated over the pairs (i, j) (off-diagonal pairs twice):
//   s1 = phi_,ij (mu * phi_,ij),  s2 = (phi_,ii)^2 + phi_,ij phi_,ij,  s3 = psi^2,
//   s4 = 2 phi_,ij psi_,ij - delta1_,j psi_,j,  s_GR = phi0_,ij phi0_,ij - (phi0_,ii)^2,
// with the fields evolved by D1(k, a) (phi0 by D1_GR(a)); the printed "-" inside S2 is
// read as "+" (the reading under which S1 + S2 reduces to the GR source at mu = 1 and
// reproduces the first bracket of Eq. full-d2).  In k space:
//   S_MG = 4piGrho F[s1] - 2piGrho mu F[s2] + (8piGrho/3)^2 M2/12 (k^2/a^2)/Pi F[s3]
//          - (8piGrho/3) m^2/(2a^2)/Pi F[s4],     S_GR = 2piGrho F[s_GR],
// and the per-mode ratio Re(S_MG / S_GR) is binned in the P(k) shells (modes with
// |S_GR| below 1e-8 of its rms skipped): mean, scatter and count per shell.
#include <math.h>

#include "passes.cuh"

namespace lpt2 {

__global__ void k_src_pair(size_t cells, const float* __restrict__ phi, const float* __restrict__ muphi,
                           const float* __restrict__ psi_ij, const float* __restrict__ phi0, float w, int diag,
                           SrcAccum acc) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += (size_t)gridDim.x * blockDim.x) {
    const float p = phi[i], p0 = phi0[i];
    acc.s1[i] = fmaf(w * p, muphi[i], acc.s1[i]);
    acc.s2[i] = fmaf(w * p, p, acc.s2[i]);
    acc.s4[i] = fmaf(2.f * w * p, psi_ij[i], acc.s4[i]);
    acc.sg[i] = fmaf(w * p0, p0, acc.sg[i]);
    if (diag) {
      acc.tr[i] += p;
      acc.tr0[i] += p0;
    }
  }
}

__global__ void k_src_grad(size_t cells, const float* __restrict__ del_j, const float* __restrict__ psi_j,
                           float* __restrict__ s4) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += (size_t)gridDim.x * blockDim.x)
    s4[i] = fmaf(-del_j[i], psi_j[i], s4[i]);   // phi_,iij psi_,j with phi_,iij = -delta1_,j
}

__global__ void k_src_final(size_t cells, SrcAccum acc, float* __restrict__ psi_to_s3) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += (size_t)gridDim.x * blockDim.x) {
    const float t = acc.tr[i], t0 = acc.tr0[i], ps = psi_to_s3[i];
    acc.s2[i] = fmaf(t, t, acc.s2[i]);
    acc.sg[i] = fmaf(-t0, t0, acc.sg[i]);
    psi_to_s3[i] = ps * ps;
  }
}

static unsigned grid_for(size_t cells) {
  const size_t b = (cells + 255) / 256;
  return (unsigned)(b < 152 * 16 ? b : 152 * 16);
}

cudaError_t launch_src_pair(size_t cells, const float* phi, const float* muphi, const float* psi_ij,
                            const float* phi0, float w, int diag, SrcAccum acc, cudaStream_t s) {
  k_src_pair<<<grid_for(cells), 256, 0, s>>>(cells, phi, muphi, psi_ij, phi0, w, diag, acc);
  return cudaGetLastError();
}
cudaError_t launch_src_grad(size_t cells, const float* del_j, const float* psi_j, float* s4, cudaStream_t s) {
  k_src_grad<<<grid_for(cells), 256, 0, s>>>(cells, del_j, psi_j, s4);
  return cudaGetLastError();
}
cudaError_t launch_src_final(size_t cells, SrcAccum acc, float* psi_to_s3, cudaStream_t s) {
  k_src_final<<<grid_for(cells), 256, 0, s>>>(cells, acc, psi_to_s3);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- per-mode ratio
// One thread per (kx, ky) walks kz in [0, N/2) (the stored half spectrum; kz > 0 counts
// for itself and its conjugate, whose ratio has the same real part).  Pass 0 sums
// w |S_GR|^2 and w over the shelled modes; pass 1 bins Re(S_MG / S_GR) above the floor.
// Shell b = floor(2 n_bins |n| / N) by exact integer comparison, 0 < |n| < N/2.
__device__ __forceinline__ int src_shell(long long n2, int n, int ns) {
  if (n2 == 0 || 4 * n2 >= (long long)n * n) return -1;
  const long long M = 4LL * ns * ns * n2;
  int b = (int)(sqrtf((float)n2) * (2.0f * (float)ns / (float)n));
  while (b > 0 && (long long)b * n * (long long)b * n > M) --b;
  while ((long long)(b + 1) * n * (long long)(b + 1) * n <= M) ++b;
  return b;
}

__device__ __forceinline__ void src_mode(const SrcRatioArgs& a, size_t e, float n2f, float2& smg, float2& sgr) {
  const float q = a.kf * a.kf * n2f * a.inv_a2;   // k^2 / a^2
  float mu = 1.f, c3 = 0.f, c4 = 0.f;
  if (a.fr0 > 0.f) {
    const float pi = q + a.m2a;
    mu = 1.f + q / (3.f * pi);
    c3 = a.e3 * a.e3 * a.M2a / 12.f * q / pi;
    c4 = -a.e3 * a.m2a * 0.5f * a.inv_a2 / pi;
  }
  const float2 f1 = a.f1[e], f2 = a.f2[e], f3 = a.f3[e], f4 = a.f4[e], fg = a.fg[e];
  const float h = -0.5f * a.fpg * mu;
  smg = make_float2(a.fpg * f1.x + h * f2.x + c3 * f3.x + c4 * f4.x, a.fpg * f1.y + h * f2.y + c3 * f3.y + c4 * f4.y);
  sgr = make_float2(0.5f * a.fpg * fg.x, 0.5f * a.fpg * fg.y);
}

constexpr int kSrcThreads = 128;
int src_ratio_blocks(int n) { return (n * n + kSrcThreads - 1) / kSrcThreads; }

__global__ void __launch_bounds__(kSrcThreads) k_src_ratio(SrcRatioArgs a, int pass, const double* rms_part, int nblk) {
  extern __shared__ double s_acc[];   // pass 0: [2]; pass 1: [3][n_bins]
  __shared__ double s_floor2;
  const int nq = pass == 0 ? 2 : 3 * a.n_bins;
  for (int i = threadIdx.x; i < nq; i += blockDim.x) s_acc[i] = 0.0;
  if (pass == 1 && threadIdx.x == 0) {   // (1e-8 rms)^2 from the pass-0 partials, fixed order
    double sg = 0.0, w = 0.0;
    for (int b = 0; b < nblk; ++b) { sg += rms_part[2 * b]; w += rms_part[2 * b + 1]; }
    s_floor2 = w > 0 ? 1e-16 * sg / w : 0.0;
  }
  __syncthreads();
  const double floor2 = pass == 1 ? s_floor2 : 0.0;
  const int n = a.n, h = n / 2;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;   // (kx, ky)
  if (row < n * n) {
    const int kx = row / n, ky = row % n;
    const int mx = kx < h ? kx : kx - n, my = ky < h ? ky : ky - n;
    int cur = -1;
    double sr = 0.0, sr2 = 0.0, sw = 0.0;
    for (int kz = 0; kz < h; ++kz) {
      const long long n2 = (long long)mx * mx + (long long)my * my + (long long)kz * kz;
      const int b = src_shell(n2, n, a.n_bins);
      const size_t e = (size_t)row * h + kz;
      float2 smg, sgr;
      src_mode(a, e, (float)n2, smg, sgr);
      if (a.smg) {   // DC and the Nyquist planes are zero, as in delta(k) and phi2(k)
        const bool z = n2 == 0 || kx == h || ky == h;
        a.smg[e] = z ? make_float2(0.f, 0.f) : smg;
        a.sgr[e] = z ? make_float2(0.f, 0.f) : sgr;
      }
      if (b < 0) continue;
      const double w = kz == 0 ? 1.0 : 2.0;
      const double g2 = (double)sgr.x * sgr.x + (double)sgr.y * sgr.y;
      if (pass == 0) {
        sr += w * g2;
        sw += w;
        continue;
      }
      if (g2 < floor2 || g2 == 0.0) continue;
      if (b != cur) {
        if (cur >= 0) {
          atomicAdd(&s_acc[cur], sr);
          atomicAdd(&s_acc[a.n_bins + cur], sr2);
          atomicAdd(&s_acc[2 * a.n_bins + cur], sw);
        }
        cur = b;
        sr = sr2 = sw = 0.0;
      }
      // Re(smg / sgr) = Re(smg conj(sgr)) / |sgr|^2
      const double r = ((double)smg.x * sgr.x + (double)smg.y * sgr.y) / g2;
      sr += w * r;
      sr2 += w * r * r;
      sw += w;
    }
    if (pass == 0) {
      atomicAdd(&s_acc[0], sr);
      atomicAdd(&s_acc[1], sw);
    } else if (cur >= 0) {
      atomicAdd(&s_acc[cur], sr);
      atomicAdd(&s_acc[a.n_bins + cur], sr2);
      atomicAdd(&s_acc[2 * a.n_bins + cur], sw);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nq; i += blockDim.x) a.part[(size_t)blockIdx.x * nq + i] = s_acc[i];
}

cudaError_t launch_src_ratio(const SrcRatioArgs& a, int pass, const double* rms_part, cudaStream_t s) {
  const int nblk = src_ratio_blocks(a.n);
  const int smem = (pass == 0 ? 2 : 3 * a.n_bins) * (int)sizeof(double);
  SrcRatioArgs b = a;
  if (pass == 0) b.smg = b.sgr = nullptr;   // the optional spectra are written once, in pass 1
  k_src_ratio<<<nblk, kSrcThreads, smem, s>>>(b, pass, rms_part, nblk);
  return cudaGetLastError();
}

__global__ void k_src_finalize(const double* part, int n_blocks, int nb, double* mean, double* sigma,
                               int64_t* count) {
  const int b = blockIdx.x;
  double s = 0.0, s2 = 0.0, w = 0.0;
  for (int i = threadIdx.x; i < n_blocks; i += blockDim.x) {
    const double* q = part + (size_t)i * 3 * nb;
    s += q[b];
    s2 += q[nb + b];
    w += q[2 * nb + b];
  }
  __shared__ double sh[3][256];
  sh[0][threadIdx.x] = s;
  sh[1][threadIdx.x] = s2;
  sh[2][threadIdx.x] = w;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double W = sh[2][0];
    const double m = W > 0 ? sh[0][0] / W : 0.0;
    mean[b] = m;
    sigma[b] = W > 0 ? sqrt(fmax(sh[1][0] / W - m * m, 0.0)) : 0.0;
    count[b] = (int64_t)(W + 0.5);
  }
}

cudaError_t launch_src_finalize(const double* part, int n_blocks, int n_bins, double* mean, double* sigma,
                                int64_t* count, cudaStream_t s) {
  k_src_finalize<<<n_bins, 256, 0, s>>>(part, n_blocks, n_bins, mean, sigma, count);
  return cudaGetLastError();
}

// Shell mean |k| (sum of |k| / mode count of the cached shell geometry) and the T1 curve
// there: (D1(k/sqrt2) / D1_GR)^2 [mu(k) - (2/27) 4piGrho (k^2/a^2) M2 / (Pi(k) Pi(k/sqrt2)^2)],
// D1 linear in ln k on the FP64 growth table (clamped).
__global__ void k_src_t1(int nb, const double* ksum, const unsigned long long* cnt, double* kmean_out,
                         const double* d1, int nk, double k_min, double k_max, const double* d1gr, double a,
                         double m2a, double M2a, double fpg, int gr, double* t1) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const double k = cnt[b] ? ksum[b] / (double)cnt[b] : 0.0;
  if (kmean_out) kmean_out[b] = k;
  if (!t1) return;
  if (!(k > 0)) { t1[b] = 0.0; return; }
  const double kh = k / sqrt(2.0);
  double x = (log(kh) - log(k_min)) / (log(k_max) - log(k_min)) * (nk - 1);
  x = fmin(fmax(x, 0.0), (double)(nk - 1));
  const int i0 = (int)fmin(floor(x), (double)(nk - 2));
  const double f = x - i0;
  const double d1h = d1[i0] * (1.0 - f) + d1[i0 + 1] * f;
  double br = 1.0;
  if (!gr) {
    const double q = k * k / (a * a), qh = 0.5 * q;
    br = 1.0 + q / (3.0 * (q + m2a)) - 2.0 / 27.0 * fpg * q * M2a / ((q + m2a) * (qh + m2a) * (qh + m2a));
  }
  const double r = d1h / d1gr[0];
  t1[b] = r * r * br;
}

cudaError_t launch_src_t1(int n_bins, const double* ksum, const unsigned long long* count, double* kmean,
                          const double* tab_d1, int nk, double k_min, double k_max, const double* d1gr, double a,
                          double m2a, double M2a, double fpg, int gr, double* t1, cudaStream_t s) {
  k_src_t1<<<(n_bins + 63) / 64, 64, 0, s>>>(n_bins, ksum, count, kmean, tab_d1, nk, k_min, k_max, d1gr, a, m2a,
                                             M2a, fpg, gr, t1);
  return cudaGetLastError();
}

}  // namespace lpt2
