/*
 * lpt2.h - C ABI of the GB300 (sm_103a) library for second-order Lagrangian
 * perturbation theory (2LPT) displacements in Hu-Sawicki f(R) gravity, after
 * Moretti, Mozzon, Monaco, Munari & Baldi (2019), "Fast numerical method to
 * generate halo catalogs in modified gravity (part I): second-order Lagrangian
 * Perturbation Theory".
 *
 * Every function returns an int status: LPT2_OK (0) or a negative error code.
 * Arguments are validated on the host before any launch; on error nothing is
 * launched and lpt2_last_error() gives a message (thread-local).  No C++
 * exception crosses this boundary.
 *
 * Memory: all field pointers are DEVICE pointers owned by the caller.  The
 * plan owns only small tables (twiddles, growth tables, cosmology constants,
 * Box-Muller tables), allocated by lpt2_plan.  Large scratch ("workspace") is
 * caller-owned too: query lpt2_workspace_size() (or, before making the plan,
 * lpt2_workspace_bytes()) and hand a device buffer to lpt2_set_workspace()
 * before lpt2_displace / lpt2_cic_pk / lpt2_displace_vjp / lpt2_fft_* and the
 * other calls that say they need it.  The device buffers of lpt2_displace_host
 * (plan flag LPT2_HOST_IO) and the tables of the output times of
 * lpt2_set_outputs (plan flag LPT2_MAX_OUTPUTS(n)) are part of that workspace.
 * No call after lpt2_plan allocates device memory.  All launches go to the
 * stream given to lpt2_plan and are asynchronous with respect to the host;
 * results are ready after the caller synchronises that stream.
 *
 * Layouts.  Grid side N (16, 32, 64, 96, 128, 192, 256, 512 or 1024), box side L in
 * Mpc/h.  A real field is float[N][N][N] (x, y, z; z fastest), cell (ix,iy,iz)
 * at Lagrangian position q = (ix, iy, iz) L / N (cell corner).  Vector fields
 * and particle positions are SoA float[3][N^3].  A spectrum ("half spectrum")
 * is float2[N][N][N/2]: modes (kx, ky, kz) with kz in [0, N/2); index i maps to
 * mode number n = i for i < N/2 and i - N otherwise, k = 2 pi n / L.  The
 * kz = N/2 plane is not stored: the method zeroes every Nyquist plane.
 *
 * Threading: a plan is not thread-safe; distinct plans are independent.
 */
#ifndef LPT2_H
#define LPT2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  LPT2_OK = 0,
  LPT2_EINVAL = -1,       /* bad argument (pointer, size, parameter range)      */
  LPT2_ENOMEM = -2,       /* plan-time device allocation failed                  */
  LPT2_ECUDA = -3,        /* a CUDA runtime call or kernel launch failed         */
  LPT2_EUNSUPPORTED = -4, /* valid but not supported (grid size, hs_n != 1, ...) */
  LPT2_ETIMEOUT = -5,     /* a bounded device-side wait gave up                  */
  LPT2_ENOWORKSPACE = -6  /* workspace missing or smaller than required          */
};

/* Plan flags. */
enum {
  LPT2_GRAPH = 1,   /* capture lpt2_displace / lpt2_cic_pk into CUDA graphs on first use and
                       replay them while the argument pointers stay the same (needs a stream
                       other than the legacy default stream) */
  LPT2_HOST_IO = 2, /* single-instance plans: the workspace also holds the two device buffer
                       sets of lpt2_displace_host (each N^3 + 3 N^3 floats + 256 doubles) and
                       the plan makes its two copy streams */
  LPT2_KEEP_STATE = 4 /* single-instance plans: lpt2_displace to the CIC density only (psi1, psi2
                       and pos NULL) also keeps S(k) and the positions in the workspace, so that
                       a following lpt2_displace_vjp with the same noise starts from the kept
                       forward map instead of recomputing it (see lpt2_displace_vjp) */
};
/* Single-instance plans: room in the workspace for the tables of up to n (<= 64) output
 * scale factors of lpt2_set_outputs (per output: growth tables 4 n_k doubles and floats,
 * multiplier tables (3 (N/2)^2 + 1) x 24 bytes).  Or it with the other flags. */
#define LPT2_MAX_OUTPUTS(n) (((unsigned)(n) & 0xffu) << 8)

/* D2 variants: the triangle configuration (k1, k2, angle theta between the vectors k1 and
 * k2, |k1 + k2| = k) at which the second-order growth of Eq. full-d2 is solved (Sec. 3,
 * the comparison of the full source term with triangles).  The source is D1(k1) D1(k2)
 * times the braces of Eq. full-d2 divided by sin^2 theta, so that every configuration keeps
 * the GR limit -3/7 D1^2. */
enum {
  LPT2_D2_T1 = 0,       /* k1 = k2 = k/sqrt2, theta = 90 deg: the paper's choice (T1)       */
  LPT2_D2_T2 = 1,       /* k1 = k2, theta = 80 deg (T2)                                      */
  LPT2_D2_ISO70 = 2,    /* k1 = k2, theta = 70 deg                                           */
  LPT2_D2_R2_80 = 3,    /* k1 = 2 k2, theta = 80 deg                                         */
  LPT2_D2_R2_70 = 4,    /* k1 = 2 k2, theta = 70 deg                                         */
  LPT2_D2_WINTHER = 5,  /* T1 braces with D1(k)^2 in place of D1(k1) D1(k2) (Winther et al.) */
  LPT2_D2_GR = 6,       /* the D2 equation of GR (mu = 1): scale-independent                 */
  LPT2_D2_ISO60 = 7,    /* k1 = k2, theta = 60 deg (the text's "equilateral", as printed)    */
  LPT2_D2_SQUEEZED = 8, /* k1 = 1e-3 k2, theta = 90 deg (squeezed: k1 ~ 0, k2 ~ k)           */
  LPT2_D2_LCDM_FIT = 9  /* Eq. lcdm-fit: D2 = -(3/7) D1(k,a)^2 Omega_m(a)^(-1/143), no D2 ODE */
};

/* Background cosmology and f(R) parameters. fr0_abs = |f_R0|; 0 selects GR
 * (mu = 1).  Flat: omega_m + omega_l must equal 1 to 1e-6.  hs_n must be 1
 * (Eq. mihusawicki is given for n = 1). a_init is the start of the growth
 * integration (Einstein-de Sitter growing mode there, Sec. 2.4). */
typedef struct {
  double omega_m, omega_l, omega_b, h, n_s, sigma8, t_cmb;
  double fr0_abs;
  int hs_n;
  double a_init;
  int d2_variant;
} lpt2_cosmo;

/* One realisation: grid side n, box side (Mpc/h), Philox seed, output scale
 * factor a_out (0 < a_init < a_out <= 1). */
typedef struct {
  int n;
  double box;
  uint64_t seed;
  double a_out;
  lpt2_cosmo cosmo;
} lpt2_instance;

typedef struct lpt2_plan_s* lpt2_plan_t;

/* lpt2_plan: create a plan for n_inst instances (1 <= n_inst <= 65535) with
 * growth tables on n_k log-spaced wavenumbers in [k_min, k_max] h/Mpc (Sec. 2.4:
 * D1(k,a) is solved per k and interpolated), integrated with n_steps classical
 * RK4 steps in ln a.  Instances share the background cosmology and a_out; seed
 * and fr0_abs may differ (one growth table per instance).  Instances of equal
 * grid size must be contiguous in `inst` and share the box; each such group runs
 * as one batch (every pass kernel covers all its instances).  Per-instance
 * arrays of the other calls are the instances' arrays concatenated in plan
 * order.  cuda_stream is a cudaStream_t (NULL = legacy default stream).  flags:
 * 0 or an or of LPT2_GRAPH, LPT2_HOST_IO, LPT2_KEEP_STATE and LPT2_MAX_OUTPUTS(n) (the
 * last three for single-instance plans only).  Allocates the plan's small device tables and computes the
 * P(k) normalisation (sigma_8) and the growth tables on the stream.  Errors:
 * LPT2_EINVAL (null pointers, n_k < 2, k_min <= 0, k_max <= k_min, box <= 0,
 * a range, non-flat cosmology, fr0_abs < 0, n_steps < 1, instance ordering or
 * differing backgrounds, unknown flags), LPT2_EUNSUPPORTED (n not in the list
 * above, hs_n != 1, d2_variant outside LPT2_D2_T1 .. LPT2_D2_LCDM_FIT, differing boxes within a grid size),
 * LPT2_ENOMEM, LPT2_ECUDA.  lpt2_white_noise, lpt2_fft_*, lpt2_set_fr0 and
 * lpt2_displace_vjp need a single-instance plan. */
int lpt2_plan(lpt2_plan_t* out, const lpt2_instance* inst, int n_inst, int n_k,
              double k_min, double k_max, int n_steps, void* cuda_stream,
              unsigned flags);

/* Frees the plan's device tables, captured graphs, streams and events (the caller's
 * workspace stays the caller's).  NULL is a no-op.  Plan management: no counterpart
 * in the paper. */
int lpt2_plan_destroy(lpt2_plan_t plan);

/* Bytes of caller-owned device scratch the plan needs: 21 slots of the largest
 * group (count N^3 floats each), the CIC density of every instance, small
 * per-block partial sums and a P(k) per instance, plus the LPT2_HOST_IO buffer
 * sets and the LPT2_MAX_OUTPUTS tables when the plan has those flags.  Memory
 * management: no counterpart in the paper. */
int lpt2_workspace_size(lpt2_plan_t plan, size_t* bytes);

/* lpt2_workspace_bytes: the same number for a plan not made yet (the arguments of
 * lpt2_plan that decide it), computed on the host without touching a GPU, so that a
 * caller can reserve the memory first.  Errors as lpt2_plan's host-side checks
 * (LPT2_EINVAL, LPT2_EUNSUPPORTED).  No counterpart in the paper. */
int lpt2_workspace_bytes(const lpt2_instance* inst, int n_inst, int n_k, unsigned flags, size_t* bytes);

/* Attach scratch: dev_ptr must be 256-byte aligned and >= lpt2_workspace_size
 * bytes; it must stay valid while calls using this plan are in flight. */
int lpt2_set_workspace(lpt2_plan_t plan, void* dev_ptr, size_t bytes);

/* lpt2_growth_tables: D1(k,a_out), D2(k,a_out) of the plan's D2 variant (T1 by
 * default) and their derivatives with respect to ln|f_R0| (Eq. d1, Eq. full-d2 at
 * the variant's triangle, T1: k1 = k2 = k/sqrt2, theta = 90 deg; D2 sign such
 * that GR gives -3/7 D1^2), recomputed
 * on the plan's stream by the batched FP64 RK4 kernel (one thread per
 * (instance, k)) and copied into the caller's device arrays double[n_inst][n_k]
 * (each pointer may be NULL). */
int lpt2_growth_tables(lpt2_plan_t plan, double* d1, double* d2,
                       double* dd1_dlogf, double* dd2_dlogf);

/* lpt2_white_noise: the unit Gaussian white noise the plan draws for the linear
 * field of Sec. 3 (Philox4x32-10 of Salmon et al. 2011 keyed by the seed, counter
 * = flat cell index; one Box-Muller transform of words 0 and 1 of the even cell
 * (x, 2j, z) gives its cosine to that cell and its sine to (x, 2j+1, z); each value
 * rounded once to FP32 as in lpt2_box_muller), written to float[N^3]. */
int lpt2_white_noise(lpt2_plan_t plan, float* noise);

/* lpt2_box_muller: the Box-Muller transform behind lpt2_white_noise applied to given Philox
 * word pairs (Sec. 3's Gaussian white noise; exposed so that the transform can be checked on
 * chosen words, e.g. u0 = 1, u0 = 2^-24 and the quadrant boundaries of the angle):
 *   words  device uint32[count][2] = (x0, x1)
 *   out    device float[count][2] = sqrt(-2 ln u0) (cos, sin)(2 pi u1), u_j = ((x_j >> 8) + 1) 2^-24,
 *          each evaluated in float-float arithmetic (relative error below about 2^-44) and rounded
 *          once to FP32, so it equals the correctly rounded value except within that distance of a
 *          rounding midpoint
 * Runs on the plan's stream (the plan holds the transform's tables).  0 <= count <= 2^31; both
 * pointers 8-byte aligned.  LPT2_EINVAL otherwise. */
int lpt2_box_muller(lpt2_plan_t plan, const uint32_t* words, int64_t count, float* out);

/* lpt2_philox_words: raw Philox4x32-10 output (Salmon et al. 2011; the generator
 * behind lpt2_white_noise, exposed for bit-exact checks) for counters (c, 0) with
 * c in [first, first + count): uint32 out[count][4].  count <= 2^31. */
int lpt2_philox_words(uint64_t seed, uint64_t first, int64_t count,
                      uint32_t* out, void* cuda_stream);

/* lpt2_displace: the forward 2LPT map (Sec. 2.1 Eq. second-ini, Sec. 2.4).
 *   noise : float[N^3] unit white noise, or NULL to draw it with Philox
 *   psi1  : float[3][N^3] first-order displacement Psi1 = i k D1 delta/k^2, or NULL
 *   psi2  : float[3][N^3] second-order displacement Psi2 = i k D2 (-S(k)/k^2), or NULL
 *   pos   : float[3][N^3] particle positions q + Psi1 + Psi2 wrapped into [0, L), or NULL
 *   dk    : float2 half spectrum of the linear density delta(k), or NULL
 * When psi1 and psi2 are both NULL the two potentials are summed in k space
 * and only the total displacement is transformed.  The CIC density of the
 * displaced particles is always deposited into the workspace, for
 * lpt2_cic_pk(plan, NULL, ...).  Needs the workspace. */
int lpt2_displace(lpt2_plan_t plan, const float* noise, float* psi1, float* psi2,
                  float* pos, void* dk);

/* lpt2_cic_pk (Sec. 4, the power-spectrum comparison, here of the matter field):
 * cloud-in-cell density contrast of N^3 unit-mass particles and
 * its power spectrum P(k) = V |delta(k)|^2 / N^6 averaged over n_shells linear
 * shells of width k_Ny / n_shells in [0, k_Ny) (DC excluded).
 *   pos     : float[3][N^3] positions in [0, L), or NULL to use the density
 *             deposited by the last lpt2_displace on this plan
 *   density : float[N^3] density contrast output, or NULL
 *   pk, k_mean : double[n_shells] shell mean of P and of |k| (0 if empty)
 *   n_modes : int64[n_shells] number of modes per shell (full spectrum count)
 * 1 <= n_shells <= 256; per-instance outputs are [n_inst][n_shells].  Needs the
 * workspace. */
int lpt2_cic_pk(lpt2_plan_t plan, const float* pos, float* density, double* pk,
                double* k_mean, int64_t* n_modes, int n_shells);

/* lpt2_displace_host: the forward step (lpt2_displace to positions, then the CIC shell
 * P(k) of lpt2_cic_pk: Sec. 2.1 Eq. second-ini, Sec. 2.4, Sec. 4) end to end from and to
 * HOST memory, for n_real realisations of a single-instance plan.  For r in [0, n_real):
 *   noise_h + r * noise_stride  host float[N^3] white noise, or noise_h NULL to draw the
 *                               plan's Philox noise on the device (nothing uploaded)
 *   pos_h + r * pos_stride      host float[3][N^3] positions in [0, L), or pos_h NULL
 *   pk_h + r * pk_stride        host double[n_shells] shell P(k), or pk_h NULL
 * Strides are in elements; a stride of 0 makes every realisation use the one buffer
 * (every copy still happens, and the last realisation's result is what remains);
 * otherwise a stride is at least one realisation's size.  The steps are pipelined:
 * while realisation r computes on the plan's stream, the upload of r + 1 and the
 * download of r - 1 (and of r's positions, during r's P(k)) run on two copy streams of
 * the plan, through two device buffer sets in the caller's workspace (the plan must be made
 * with LPT2_HOST_IO; 4 N^3 floats + 256 doubles each).  Page-locked host buffers
 * (cudaHostAlloc, cudaHostRegister) let the copies overlap the kernels; pageable ones
 * give the same results with less overlap.  The call returns when every result is in
 * host memory.  It synchronises, so it cannot be captured in a CUDA graph; the plan's
 * lpt2_displace / lpt2_cic_pk graphs are not used.  Needs the workspace.
 * Errors: LPT2_EUNSUPPORTED for a batched plan; LPT2_EINVAL for a plan made without
 * LPT2_HOST_IO, n_real < 1, n_shells outside [1, 256], pos_h and pk_h both NULL, or a
 * too-small non-zero stride; LPT2_ECUDA from a copy or launch (the call still waits for
 * everything it queued before returning). */
int lpt2_displace_host(lpt2_plan_t plan, int n_real, const float* noise_h, int64_t noise_stride,
                       float* pos_h, int64_t pos_stride, double* pk_h, int64_t pk_stride, int n_shells);

/* Several output times from one realisation (the paper evaluates its fields at one
 * scale factor at a time; Sec. 2.4 and Eq. second-ini give the time dependence, which
 * enters only through D1(k, a) and D2(k, a)).  The six phi_ij, and so S, are built from
 * the z = 0 linear field delta_0 whatever the output time, so noise -> delta(k) -> phi_ij
 * -> S(k) is the same for every a and is computed once; only the multipliers
 * -S D2(k, a)/k^2 + delta D1(k, a)/k^2 and what follows them (Psi, positions, CIC,
 * P(k)) are repeated per a.
 *
 * lpt2_set_outputs: the output scale factors a_out[0 .. n_a-1] (host array, each in
 * (a_init, 1], any order, 1 <= n_a <= 64) of a single-instance plan.  Computes and
 * keeps, per a_j, the FP64 RK4 growth tables from a_init to a_j (the plan's k table,
 * step count, cosmology and D2 variant) and the per-|n|^2 multiplier tables, on the
 * plan's stream, in the caller's workspace (room for n_a of them: plan flag
 * LPT2_MAX_OUTPUTS(n) with n >= n_a); lpt2_set_fr0 and lpt2_set_workspace recompute them.
 * Replaces an earlier list.  Errors: LPT2_EUNSUPPORTED for a batched plan, LPT2_EINVAL for
 * a bad list or n_a above the plan's LPT2_MAX_OUTPUTS, LPT2_ENOWORKSPACE. */
int lpt2_set_outputs(lpt2_plan_t plan, int n_a, const double* a_out);

/* lpt2_displace_outputs (Sec. 2.4, the time dependence through D1(k,a), D2(k,a)):
 * one realisation at every output scale factor of
 * lpt2_set_outputs (device pointers):
 *   noise    float[N^3] white noise, or NULL for the plan's Philox noise
 *   pos      float[n_a][3][N^3] positions in [0, L) at a_j, or NULL
 *   pk       double[n_a][n_shells] CIC shell P(k) at a_j (as lpt2_cic_pk)
 *   k_mean, n_modes  double / int64 [n_shells] (the same for every a_j), or NULL
 * Each a_j's outputs equal those of lpt2_displace + lpt2_cic_pk on a plan made with
 * a_out = a_j (the same kernels in the same order after the shared prefix).  The CIC
 * density left in the workspace is the last a_j's.  Not graph-captured.  Needs the
 * workspace.  Errors: LPT2_EINVAL if no output list is set, pk is NULL or n_shells is
 * outside [1, 256]; LPT2_EUNSUPPORTED for a batched plan. */
int lpt2_displace_outputs(lpt2_plan_t plan, const float* noise, float* pos, double* pk,
                          double* k_mean, int64_t* n_modes, int n_shells);

/* Launch schedule of a batched plan (no counterpart in the paper: how the batched form
 * of the path is cut into launches).  Instances of one grid size form a group whose
 * fields lie consecutively in every workspace slot; lpt2_displace and lpt2_cic_pk run a
 * group in chunks of `chunk` instances per launch (default: the whole group), so that a
 * chunk's fields can stay in L2 between the passes of small grids.  Outputs do not depend
 * on the schedule (each instance's kernels are the same; the CIC float reductions may
 * add in another order).
 *
 * lpt2_schedule: the number of groups (in order of the instances' first appearance) and,
 * if chunk is not NULL, up to max_groups current chunk sizes.
 * lpt2_set_schedule: chunk[n_groups] instances per launch (each >= 1, clamped to the
 * group's size); drops the plan's captured graphs (recaptured on the next call).
 * lpt2_tiles: the number of groups and, where the arrays are not NULL, up to max_groups
 * tile choices per group: ytile = pencils per CTA of the y passes (0 = build default, 8 or
 * 16) and xtile = tile path of the x passes of delta(k) and of the adjoint's x transposes
 * (0 = build default, 1 = bulk-tensor tiles staged in shared memory, 2 = global loads).
 * lpt2_set_tiles: sets them for every group (ytile 16 needs N >= 32); results are the
 * same bit for bit for every choice, only the speed differs.  Drops the captured graphs.
 * lpt2_autotune: times every group's forward step (Philox noise -> positions -> CIC ->
 * n_shells-shell P(k)) on the plan's stream at chunk sizes count, ceil(count/2), ..., 1,
 * `reps` timed repetitions after one warm-up each, keeps the fastest per group; then, at
 * that chunk size, tries ytile 8 and 16 and xtile 1 and 2 in turn and keeps what is faster;
 * and drops the captured graphs.  Plan-time work: it synchronises and overwrites the
 * workspace; not capturable.  Needs the workspace.
 * Errors: LPT2_EINVAL (bad count, chunk, tile choice, n_shells, or reps outside [1, 100]),
 * LPT2_ECUDA. */
int lpt2_schedule(lpt2_plan_t plan, int* chunk, int max_groups, int* n_groups);
int lpt2_set_schedule(lpt2_plan_t plan, const int* chunk, int n_groups);
int lpt2_tiles(lpt2_plan_t plan, int* ytile, int* xtile, int max_groups, int* n_groups);
int lpt2_set_tiles(lpt2_plan_t plan, const int* ytile, const int* xtile, int n_groups);
int lpt2_autotune(lpt2_plan_t plan, int n_shells, int reps);

/* lpt2_set_fr0: change |f_R0| of the plan (it enters Eq. d1 and Eq. full-d2
 * through m^2(a) and M2(a), Eq. mihusawicki) and recompute its growth tables
 * (the FP64 RK4 kernel) on the plan's stream.  fr0_abs >= 0 (0 = GR). */
int lpt2_set_fr0(lpt2_plan_t plan, double fr0_abs);

/* lpt2_displace_vjp: hand-written adjoint (vector-Jacobian product) of the map
 * (white noise, ln|f_R0|) -> (CIC density contrast, shell P(k)) of
 * lpt2_displace + lpt2_cic_pk, and of the particle positions (the paper has
 * no gradients: this is the transpose
 * of the steps of Sec. 2.1 Eq. second-ini and Sec. 2.4 taken in reverse order).
 * The forward map is recomputed inside (delta(k), S(k), the positions and the six phi_ij
 * stay in the workspace for the transposes: the forward's phi_ij are checkpointed in
 * slots that nothing overwrites before the source-term transpose reads them), except on a
 * plan made with
 * LPT2_KEEP_STATE whose last lpt2_displace (to the density only) used the same noise
 * pointer and whose workspace no call has overwritten since (lpt2_cic_pk of that density
 * keeps it too, and also leaves the density spectrum the adjoint needs): then the adjoint
 * starts from that forward map.  The noise buffer must still hold the values it had then;
 * a call that overwrites the kept state (lpt2_displace, lpt2_cic_pk with positions,
 * lpt2_displace_vjp itself, lpt2_set_fr0, lpt2_set_workspace, ...) makes the next adjoint
 * recompute the forward map.
 *   noise      float[N^3] white noise, or NULL for the plan's Philox noise
 *   g_pos      float[3][N^3] dL/d(positions), or NULL (zero)
 *   g_density  float[N^3] dL/d(density contrast), or NULL (zero)
 *   g_pk       double[n_shells] dL/dP_b, or NULL (zero); shells as lpt2_cic_pk
 *   g_noise    float[N^3] output dL/dnoise, or NULL
 *   g_log_fr0  double[1] output dL/dln|f_R0| (FP64 reduction), or NULL
 * All pointers are device pointers.  Needs the workspace. */
int lpt2_displace_vjp(lpt2_plan_t plan, const float* noise, const float* g_pos,
                      const float* g_density, const double* g_pk, int n_shells, float* g_noise,
                      double* g_log_fr0);

/* Refinements of the P(k) estimator that Sec. 4 does not apply (its P(k) is the raw CIC
 * estimate of lpt2_cic_pk); the method of Sefusatti et al. 2016:
 *   LPT2_PK_DECONVOLVE  divide |delta(k)|^2 by the CIC window squared, W = prod_i sinc^2(pi n_i/N)
 *   LPT2_PK_INTERLACE   deposit a second grid of the particles shifted by +h/2 along every
 *                       axis (h = L/N) and use delta(k) = [F1 + F2 exp(i pi (nx+ny+nz)/N)] / 2,
 *                       which cancels the odd aliasing images; needs pos (not NULL)
 * Arguments, layouts and shells as lpt2_cic_pk (density, when given, is the first grid's
 * contrast); flags = 0 gives the lpt2_cic_pk result.  Needs the workspace; not captured in
 * a graph.  LPT2_EINVAL for unknown flags or interlacing without positions. */
enum { LPT2_PK_DECONVOLVE = 1, LPT2_PK_INTERLACE = 2 };
int lpt2_cic_pk_est(lpt2_plan_t plan, const float* pos, float* density, double* pk, double* k_mean,
                    int64_t* n_modes, int n_shells, unsigned flags);

/* Full second-order source term and its ratio to GR (Sec. 3, Eqs. full, s1-s4; the
 * diagnostic behind the paper's source-term figure, from which the T1 triangle was chosen).
 * With delta1(k) = D1(k,a) delta0(k) (a = the plan's a_out), phi = delta1/k^2 and
 * psi = delta1/Pi(k,a):
 *   S1 = 4piGrho DFT[phi_,ij IDFT[mu(k) DFT[phi_,ij]]],
 *   S2 = -2piGrho mu(k) DFT[phi_,ii phi_,jj + phi_,ij phi_,ij]   (the printed "-" between the two
 *        products is read as "+": with it S1 + S2 is the GR source at mu = 1 and the sum of the
 *        four terms reproduces Eq. full-d2 for any pair of modes),
 *   S3 = (8piGrho/3)^2 M2/12 (k^2/a^2)/Pi(k) DFT[psi^2],
 *   S4 = -(8piGrho/3) m^2/(2a^2)/Pi(k) DFT[2 phi_,ij psi_,ij + phi_,iij psi_,j],
 * and the GR source S_GR (same delta0, fields evolved with D1_GR(a)).  The per-mode ratio
 * Re(S_MG / S_GR) (modes with |S_GR| below 1e-8 of its rms skipped) is binned in n_bins
 * linear shells of width k_Ny / n_bins, as the P(k) of lpt2_cic_pk.
 *   noise    float[N^3] white noise, or NULL for the plan's Philox noise
 *   mean, sigma  double[n_bins] mean and scatter of the ratio per shell (output)
 *   count    int64[n_bins] modes per shell, conjugate pairs counted twice (output)
 *   t1       double[n_bins] the T1 analytic ratio (D1(k/sqrt2)/D1_GR)^2 [mu(k) - (2/27) 4piGrho
 *            (k^2/a^2) M2 / (Pi(k) Pi(k/sqrt2)^2)] at the shell's mean |k|, or NULL
 *   k_mean   double[n_bins] mean |k| per shell (h/Mpc), or NULL (required when t1 is given)
 *   s_mg, s_gr  complex64 [N][N][N/2] half spectra of S_MG and S_GR (output), or both NULL
 * Device pointers; single-instance plans; needs the workspace (uses most slots); returns
 * LPT2_EINVAL for bad arguments, LPT2_EUNSUPPORTED for multi-instance plans.  Not on the
 * displacement path: about 36 three-pass transforms per call. */
int lpt2_source_ratio(lpt2_plan_t plan, const float* noise, int n_bins, double* mean, double* sigma,
                      int64_t* count, double* t1, double* k_mean, void* s_mg, void* s_gr);

/* The path's three-pass transforms on their own (no counterpart in the paper).
 * lpt2_fft_r2c: forward 3-D transform of a real field (unnormalised,
 * exp(-i k.x)) into the half spectrum; in and out may not alias.
 * lpt2_fft_c2r: inverse (exp(+i k.x), unnormalised: the result is N^3 times the
 * inverse DFT), treating the missing kz = N/2 plane as zero.  `in` is not
 * modified.  Both need the workspace. */
int lpt2_fft_r2c(lpt2_plan_t plan, const float* in, void* out);
int lpt2_fft_c2r(lpt2_plan_t plan, const void* in, float* out);

/* Per-kernel timing (instrumentation; no counterpart in the paper).
 * lpt2_timing(plan, 1) clears the record and brackets each
 * later kernel launch of this plan with CUDA events on the plan's stream (up to
 * 4096 launches); lpt2_timing(plan, 0) stops recording.  lpt2_timing_report
 * waits for the recorded events and aggregates them by kernel name: launches,
 * total device time (ms, from the events) and the algorithmic bytes those
 * launches move (the reads and writes each pass needs at minimum).  Up to `max`
 * entries are written to `out`; *n_out gets their number. */
typedef struct {
  char name[32];
  int64_t launches;
  double total_ms;
  double bytes;
} lpt2_kernel_stat;
int lpt2_timing(lpt2_plan_t plan, int enable);
int lpt2_timing_report(lpt2_plan_t plan, lpt2_kernel_stat* out, int max, int* n_out);

/* lpt2_cic_pk_noalloc: the same CIC density contrast and shell P(k) as
 * lpt2_cic_pk, for callers that are not allowed to allocate GPU memory - for
 * example an application whose device memory is handed to its own pool at
 * start-up, or code running where cudaMalloc is forbidden - and so can create
 * neither a plan nor a workspace.  The paper has no counterpart: this is a
 * deployment variant of one step of the path.
 *   n        grid side, 16, 32, 64 or 128 (larger sizes return LPT2_EUNSUPPORTED)
 *   box      side of the periodic box, Mpc/h (> 0)
 *   pos      device float[3][n^3] particle positions (one particle per cell)
 *   density  device float[n^3] density contrast output, or NULL
 *   pk, k_mean, n_modes, n_shells: as for lpt2_cic_pk
 *   cuda_stream  cudaStream_t to launch on
 * It calls no cudaMalloc/cudaFree and no allocating library routine: all
 * scratch (about 20 MB: density, spectrum, shell partial sums, twiddles) is one
 * static __device__ array inside the library, which every GPU that loads the
 * library keeps until the process exits.  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  All calls share the one array: calls whose
 * kernels overlap on the GPU (different streams, or different host threads on
 * the same device) race and corrupt each other's results - serialise them.
 * Errors as for lpt2_cic_pk; the message is reported by lpt2_last_error(). */
int lpt2_cic_pk_noalloc(int n, double box, const float* pos, float* density, double* pk,
                        double* k_mean, int64_t* n_modes, int n_shells, void* cuda_stream);

/* Test hook for the allocation-failure paths (no counterpart in the paper).  Every device
 * allocation of the library is made by lpt2_plan.  With fail_at = k >= 0 the k-th allocation
 * after this call (counting from 0, over all plans and threads) fails as if the device were out
 * of memory; fail_at = -1 turns the failure off.  *live (if not NULL) receives the number of
 * device allocations of the library that are currently live, so that a test can check that a
 * failed lpt2_plan freed everything it had allocated.  Not for concurrent use with other plans. */
int lpt2_debug_alloc_hook(int fail_at, int64_t* live);

/* Message of the last failing call on this thread ("" if none); error reporting,
 * no counterpart in the paper. */
const char* lpt2_last_error(void);

/* Instrumentation, no counterpart in the paper: the number of kernel launches
 * issued by this plan since creation (counter kept on
 * the host; used to report launch counts). */
int64_t lpt2_launch_count(lpt2_plan_t plan);

/* lpt2_set_wait_budget: the cycle budget of the plan's bounded device-side waits on its
 * bulk-copy rings (default 2e9 SM cycles, about one second), for its later launches.  A
 * CTA whose wait runs out waits (with the default budget) for its own copies in flight,
 * sets the plan's device error word and returns; lpt2_device_status then reports
 * LPT2_ETIMEOUT.  cycles = 0 makes every such wait give up at once without looking at its
 * barrier, which is how the timeout path is exercised (the copies themselves complete).
 * cycles < 0: LPT2_EINVAL.  Failure detection: no counterpart in the paper. */
int lpt2_set_wait_budget(lpt2_plan_t plan, int64_t cycles);

/* Waits for the plan's stream and reads the plan's device error word.  Kernels that
 * stage data with bulk asynchronous copies wait on them with a bounded wait (about
 * one second, lpt2_set_wait_budget); a wait that runs out makes its CTA return early
 * and sets the word.
 * Returns LPT2_OK, or LPT2_ETIMEOUT (the word is then cleared and the outputs of
 * every launch since the previous check are invalid), or LPT2_ECUDA.  Not part of
 * the paper's method: a run-time health check of the asynchronous launches. */
int lpt2_device_status(lpt2_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* LPT2_H */
