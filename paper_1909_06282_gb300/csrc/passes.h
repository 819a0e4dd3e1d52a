// Host/device shared declarations of the pass kernels' argument blocks and the
// per-grid-size launcher entry points (instantiated in inst_<N>.cu).
#pragma once
#include <cuda.h>   // CUtensorMap (a plain 128-byte descriptor; no driver call is linked)
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace lpt2 {

// Written by the cosmology set-up kernels (FP64 in, FP32 constants out).
struct DevCosmo {
  double amp;        // P(k) amplitude A (sigma_8 normalisation), (Mpc/h)^(3+n_s)
  double sigma_sq;   // sigma^2(8 Mpc/h) of the unnormalised shape
  float sqrt_amp;    // sqrt(A)
  float ns_half;     // n_s / 2
  float theta2;      // (T_CMB / 2.7)^2
  float omh;         // Omega_m h
  float alpha;       // alpha_Gamma (EH Eq. 31)
  float s043h;       // 0.43 s h  (EH Eq. 30 written for k in h/Mpc)
  float lnkmin;      // ln k_min of the growth table
  float inv_dlnk;    // 1 / (ln k spacing)
  int nk;
};

struct Geo {
  int n;
  float kf;             // 2 pi / L
  float box;            // L
  float cell;           // L / N
  float inv_cell;       // N / L
  float inv_n3;         // 1 / N^3 (inverse-transform normalisation)
  float sqrt_n3_over_v; // sqrt(N^3 / L^3)
  float kf2n3;          // kf^2 N^3: a mode's 1/(k^2 N^3) is 1 / (|n|^2 kf2n3)
  // batching: grid z runs over `batch` instances of this grid size; instance z of
  // the launch is global instance inst0 + z (growth tables, seeds, outputs)
  int batch;
  int inst0;
  int tab_stride;       // floats per instance in the float growth tables
  int* err;             // device error word (0 = ok), may be null
  long long wait;       // cycle budget of the bounded consumer waits (0: give up at once)
  // tile schedule of this grid-size group (0 = build default): y-pass pencils per CTA
  // (8 or 16) and the x-pass tile path of the delta and adjoint modes (1 bulk-tensor, 2 global)
  int ytile;
  int xtile;
};

// Codes a kernel writes into Geo::err when a bounded wait gives up.
enum { LPT2_DEV_ETIMEOUT_ZSOURCE = 1, LPT2_DEV_ETIMEOUT_ZFINAL = 2, LPT2_DEV_ETIMEOUT_ZADJSOURCE = 3,
       LPT2_DEV_ETIMEOUT_X = 4 };

enum ZSrc { Z_NOISE = 0, Z_REAL = 1, Z_DENSITY = 2 };

struct ZR2CArgs {      // forward z pass: real rows -> half-spectrum rows
  Geo g;
  const float2* tw;
  int src;             // ZSrc
  const float* in;     // Z_REAL / Z_DENSITY
  uint32_t seed_lo, seed_hi;
  const uint64_t* seeds;  // per global instance (Z_NOISE), or null to use seed_lo/hi
  const float4* bm;       // Box-Muller tables (Z_NOISE; boxmuller.cuh)
  float2* out;         // [N*N][N/2]
};

struct ZC2RArgs {      // inverse z pass of one field: half-spectrum rows -> real rows
  Geo g;
  const float2* tw;
  const float2* in;
  float* out;
  const float* add_in;   // added to the result when not null
};

struct CicGradArgs {   // transpose of the CIC deposit: dL/d(position) of every particle
  Geo g;
  const float* grho;   // dL/d(density contrast) per cell [N^3]
  const float* pos;    // [3][N^3] particle positions of the forward
  const float* gpos;   // [3][N^3] dL/dpositions added to the gathered gradient, or null
  float* gx;           // [N^3] outputs at each particle's Lagrangian cell
  float* gy;
  float* gz;
};
cudaError_t launch_cic_grad(const CicGradArgs& a, cudaStream_t s);


struct ZAdjSourceArgs {  // transpose of k_z_source
  Geo g;
  const float2* tw;
  const float* gs;       // g_S = dL/dS in real space [N^3] (inverse z of h_S)
  const float2* in[6];   // phi_xx, phi_yy, phi_zz, phi_xy, phi_xz, phi_yz (recomputed, after y)
  int ord[6];            // their z derivative orders
  float2* out[6];        // conj z-derivative of FFT_z(g_phi_ij), same order
};

struct ZSourceArgs {   // inverse z pass of the six phi_ij, source term, forward z pass of S
  Geo g;
  const float2* tw;
  const float2* in[6]; // phi_xx, phi_yy, phi_zz, phi_xy, phi_xz, phi_yz (after the y pass)
  int ord[6];          // z derivative order still to apply to each
  float2* out;         // S, z-transformed
};

struct ZFinalArgs {    // inverse z pass of the displacement potentials, positions
  Geo g;
  const float2* tw;
  int split;           // 1: separate Psi1 / Psi2 inputs; 0: total only
  const float2* a[3];  // total (or Psi1) inputs: (order z1 -> Psi_z, z0 -> Psi_y, z0 -> Psi_x)
  const float2* b[3];  // Psi2 inputs when split
  float* psi1;         // float[3][N^3] or null
  float* psi2;
  float* pos;
};

struct YJob {          // y pass: each output = transform of (i k_y)^ord * input
  int n_in, n_out;
  const float2* in[6];
  float2* out[9];
  int src[9];
  int ord[9];
  // sum mode (transpose of the above): out[dst[i]] += conj((i k_y)^ord[i]) FFT_y(in[i]),
  // times conj((i k_z)^zord[i]) (z-derivative of the transposed z pass, 0 = none)
  int sum;
  int dst[6];
  int zord[6];
};
struct YArgs {
  Geo g;
  const float2* tw;
  int inverse;
  YJob job;
};

enum XMode {
  X_DELTA = 0,      // fwd x of the noise spectrum, sqrt(P), delta(k), inverse x of the phi (+Psi1) potentials
  X_SOURCE = 1,     // fwd x of S, -D2/k^2 (+D1 delta/k^2), inverse x orders 0, 1
  X_PK = 2,         // fwd x, shell sums of |delta|^2
  X_FWD = 3,        // plain forward x
  X_INV = 4,        // plain inverse x
  X_PHI = 5,        // (unused: the adjoint reads the forward's phi_ij)
  X_PKADJ = 6,      // fwd x, times per-shell weight, inverse x  (P(k) transpose)
  X_ADJ_SOURCE = 7, // transpose of X_SOURCE: h_Psi, h_S, dL/dln|fR0| partials
  X_ADJ_DELTA = 8,  // transpose of X_DELTA: s(k) (h_Psi + h_phi), inverse x
  X_PKP = 9,        // fwd x, shell sums of |delta|^2 only (mode counts and mean |k| cached)
  X_MUL = 10,       // k-space multiplier (i k)^ord g(|k|) of the full-source diagnostic, inverse x
  X_PKI = 11,       // as X_PKP for two grids (the second shifted by h/2) combined by interlacing
};
struct XArgs {
  Geo g;
  const float2* tw;
  int mode;
  int split;
  const float2* in;       // tile source (after the y pass / in k space for X_INV, X_PHI)
  const float2* in2[3];   // adjoint modes: the x-order 0, 1, 2 groups
  float2* delta_out;      // X_DELTA: delta(k)
  const float2* delta_in; // X_SOURCE total mode, X_ADJ_SOURCE: delta(k)
  float2* s_out;          // X_SOURCE: S(k), kept for the adjoint (or null)
  const float2* s_in;     // X_ADJ_SOURCE: S(k)
  float2* hpsi_out;       // X_ADJ_SOURCE: h_Psi(k)
  const float2* hpsi_in;  // X_ADJ_DELTA: h_Psi(k)
  float2* out[5];         // x-inverse outputs
  const DevCosmo* cosmo;
  const float* d1f;       // float growth tables [nk]
  const float* d2f;
  const float* t1f;       // float d/dln|fR0| tables [nk]
  const float* t2f;
  double* pk_part;        // X_PK: per-block partials [blocks][3][n_shells]
  int n_shells;
  const float* shell_w;   // X_PKADJ: weight per shell
  // per-|n|^2 multiplier tables of the group (index = global instance - inst0 of the
  // group, then |n|^2): {sqrt(P N^3/V), 1/(k^2 N^3), D1, D2} and {dD1, dD2}/dln|fR0|
  const float4* mt0;
  const float2* mt1;
  // X_DELTA (without the split) and X_ADJ_DELTA: sqrt(P N^3/V) of every mode of the group's
  // half spectra, float[batch][N][N][N/2] in the fields' layout (zero on the modes the
  // passes zero), or null for the mode table; with it, 1/(k^2 N^3) is computed
  // from |n|^2, so these modes read no table entry
  const float* scf;
  double* theta_part;     // X_ADJ_SOURCE: per-block partial of dL/dln|fR0|
  // X_MUL: multiplier (i kx)^ord[0] (i ky)^ord[1] (i kz)^ord[2] g(|k|) / N^3, g one of MulG,
  // with m^2(a), 1/a^2 and D1_GR(a) for mu(k) and Pi(k)
  int pk_deconv;          // X_PKP, X_PKI: divide |delta|^2 by the CIC window squared
  int mul_g;
  int mul_ord[3];
  float mul_m2a, mul_inv_a2, mul_d1gr;
  CUtensorMap tmap;       // bulk-tensor maps of `in` and `scf` (set by the launcher)
  CUtensorMap tmap_sc;
  CUtensorMap tmap_l[4];  // adjoint modes: the tile inputs in the order the ring takes them
};

// Bulk-tensor map of a batch of fields float[batch][N][N][inner] (inner floats along kz:
// N for a half spectrum of float2, N/2 for the scf field; then ky, kx, instance) whose box
// is one x-pass tile: box_inner floats x 1 ky x min(N, 256) kx x 1 instance.  False if the
// driver refuses it.
bool encode_x_tile_map(CUtensorMap* map, const void* base, int inner, int n, int box_inner, int batch);
// Fills scf (XArgs) for `count` instances of an n^3 grid from their mode tables mt0.
cudaError_t launch_sc_field(const float4* mt0, int n, int count, float* scf, cudaStream_t s);

// Radial factors of the full-source diagnostic (Sec. 3, Eqs. s1-s4):
enum MulG {
  G_POT = 0,    // D1(k) / k^2               phi
  G_MUPOT = 1,  // D1(k) mu(k) / k^2         mu * phi
  G_PSI = 2,    // D1(k) / Pi(k)             psi
  G_POT0 = 3,   // D1_GR / k^2               phi of the GR realisation
  G_D1 = 4      // D1(k)                     delta1
};

struct CicArgs {
  Geo g;
  const float* pos;      // [3][N^3]
  float* rho;
  float shift;           // added to every coordinate (cells) before the deposit; 0.5 for the
                         // interlaced grid of the P(k) estimator
};

// Per grid size launchers (return cudaError_t of the launch).
#define LPT2_DECLARE_LAUNCHERS(N)                                                  \
  cudaError_t launch_z_r2c_##N(const ZR2CArgs&, cudaStream_t);                   \
  cudaError_t launch_z_c2r_##N(const ZC2RArgs&, cudaStream_t);                   \
  cudaError_t launch_z_source_##N(const ZSourceArgs&, cudaStream_t);             \
  cudaError_t launch_z_final_##N(const ZFinalArgs&, cudaStream_t);               \
  cudaError_t launch_y_##N(const YArgs&, cudaStream_t);                          \
  cudaError_t launch_z_adj_source_##N(const ZAdjSourceArgs&, cudaStream_t);      \
  cudaError_t launch_x_##N(const XArgs&, cudaStream_t);                          \
  int x_blocks_##N();

LPT2_DECLARE_LAUNCHERS(16)
LPT2_DECLARE_LAUNCHERS(32)
LPT2_DECLARE_LAUNCHERS(64)
LPT2_DECLARE_LAUNCHERS(96)
LPT2_DECLARE_LAUNCHERS(128)
LPT2_DECLARE_LAUNCHERS(192)
LPT2_DECLARE_LAUNCHERS(256)
LPT2_DECLARE_LAUNCHERS(512)
LPT2_DECLARE_LAUNCHERS(1024)

// Size-independent kernels (misc.cu / growth.cu).
cudaError_t launch_cic(const CicArgs&, cudaStream_t);   // grid y = a.g.batch
cudaError_t launch_fill0(float* p, size_t n, cudaStream_t);
cudaError_t launch_contrast(const float* rho, float* out, size_t n, cudaStream_t);
cudaError_t launch_pk_finalize(const double* part, int n_blocks, int n_shells, double* pk,
                               double* k_mean, int64_t* n_modes, cudaStream_t, int batch = 1);
// Mode count and sum of |k| per shell (0 < |n| < N/2, half spectrum kz < N/2, kz > 0
// counted twice) for n_shells shells of width k_Ny / n_shells: the data-independent
// part of the P(k) estimator.  kmean and nmodes must be zeroed before the launch.
cudaError_t launch_shell_geometry(int n, double box, int n_shells, double* ksum, unsigned long long* nmodes,
                                  cudaStream_t s);
// Full-source diagnostic (source.cu): real-space accumulations over the pairs (i, j),
// the per-mode ratio of the MG to the GR source, its shell mean / scatter, the T1 curve.
struct SrcAccum {
  float *s1, *s2, *s4, *sg, *tr, *tr0;   // accumulators [N^3]
};
cudaError_t launch_src_pair(size_t cells, const float* phi, const float* muphi, const float* psi_ij,
                            const float* phi0, float w, int diag, SrcAccum acc, cudaStream_t s);
cudaError_t launch_src_grad(size_t cells, const float* del_j, const float* psi_j, float* s4, cudaStream_t s);
cudaError_t launch_src_final(size_t cells, SrcAccum acc, float* psi_to_s3, cudaStream_t s);
struct SrcRatioArgs {
  int n, n_bins;
  float kf, fpg, e3, m2a, inv_a2, M2a, fr0;   // 4 pi G rho, 8 pi G rho / 3, m^2(a), 1/a^2, M2(a)
  const float2 *f1, *f2, *f3, *f4, *fg;       // DFT of s1, s2, s3, s4, s_GR (half spectra)
  float2 *smg, *sgr;                          // optional per-mode sources out
  double* part;                               // [blocks][2] for pass 0, [blocks][3][n_bins] for pass 1
};
int src_ratio_blocks(int n);
cudaError_t launch_src_ratio(const SrcRatioArgs& a, int pass, const double* rms_part, cudaStream_t s);
cudaError_t launch_src_finalize(const double* part, int n_blocks, int n_bins, double* mean, double* sigma,
                                int64_t* count, cudaStream_t s);
cudaError_t launch_src_t1(int n_bins, const double* ksum, const unsigned long long* count, double* kmean,
                          const double* tab_d1, int nk, double k_min, double k_max, const double* d1gr, double a,
                          double m2a, double M2a, double fpg, int gr, double* t1, cudaStream_t s);

// P(k) from per-block |delta|^2 shell sums [batch][n_blocks][n_shells] and the cached
// geometry; the buffer `part` must hold twice the partials (the first stage's sums follow
// them), n_shells in [1, 256].
cudaError_t launch_pk_finalize_p(const double* part, int n_blocks, int n_shells, const double* ksum,
                                 const unsigned long long* count, double* pk, double* k_mean, int64_t* n_modes,
                                 cudaStream_t s, int batch);
cudaError_t launch_noise(const Geo& g, uint32_t seed_lo, uint32_t seed_hi, const float4* bm, float* out,
                         cudaStream_t);
// Box-Muller transform of given word pairs (x0, x1) [count][2] -> floats [count][2].
cudaError_t launch_box_muller(const uint32_t* words, int64_t count, const float4* bm, float* out, cudaStream_t);
cudaError_t launch_philox_words(uint32_t seed_lo, uint32_t seed_hi, uint64_t first, int64_t count,
                                uint32_t* out, cudaStream_t);

// Sets the thread-local message returned by lpt2_last_error().
void set_last_error(const char* msg);
inline void set_last_error(const std::string& msg) { set_last_error(msg.c_str()); }

struct GrowthParams {
  double omega_m, omega_l, omega_b, h, n_s, sigma8, t_cmb, fr0_abs, a_init, a_out;
  double k_min, k_max;
  int nk, n_steps;
  int n_inst;            // tables for n_inst instances (grid y)
  const double* fr0s;    // device |fR0| per instance, or null for fr0_abs
  int d2_variant;        // triangle configuration of D2 (include/lpt2.h LPT2_D2_*)
};
int cosmo_partial_blocks();
cudaError_t launch_cosmo_setup(const GrowthParams&, double* partials, DevCosmo* out, cudaStream_t);
cudaError_t launch_growth(const GrowthParams&, double* tab /*[4][nk]*/, float* tabf /*[4][nk]*/,
                          cudaStream_t);
// Multiplier tables of one group of `count` instances of grid n, box L: entries
// |n|^2 = 0 .. 3 (n/2)^2 per instance (FP64 evaluation, rounded once).
__host__ __device__ inline int mode_table_len(int n) { return 3 * (n / 2) * (n / 2) + 1; }
cudaError_t launch_mode_tables(const GrowthParams&, const DevCosmo* cosmo, const double* tab, int inst0, int count,
                               int n, double box, float4* mt0, float2* mt1, cudaStream_t);
cudaError_t launch_pk_adj_weights(const double* g_pk, const int64_t* n_modes, int n_shells, double v_over_n6,
                                  float* w, cudaStream_t);
cudaError_t launch_sum_partials(const double* part, int n, double* out, cudaStream_t);

}  // namespace lpt2
