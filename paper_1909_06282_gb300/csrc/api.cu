// Host side of the C ABI declared in include/lpt2.h: argument validation, plan
// tables, workspace layout and the launch sequence of each entry point.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>   // header-only: ranges cost a pointer test unless a profiler is attached

#include "../../include/lpt2.h"
#include "boxmuller.cuh"
#include "passes.h"

using namespace lpt2;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

// Every device allocation of the library goes through plan_malloc / plan_free (all of them
// in lpt2_plan).  A test can make the k-th allocation fail (lpt2_debug_alloc_hook) and read
// how many allocations are live, to check that each failure returns LPT2_ENOMEM and frees
// what was already allocated.
std::atomic<int> g_fail_alloc_at{-1};
std::atomic<int> g_alloc_calls{0};
std::atomic<long long> g_alloc_live{0};

cudaError_t plan_malloc(void** ptr, size_t bytes) {
  *ptr = nullptr;
  const int k = g_alloc_calls.fetch_add(1);
  if (g_fail_alloc_at.load() >= 0 && k == g_fail_alloc_at.load()) return cudaErrorMemoryAllocation;
  const cudaError_t e = cudaMalloc(ptr, bytes);
  if (e == cudaSuccess) g_alloc_live.fetch_add(1);
  return e;
}

void plan_free(void* ptr) {
  if (!ptr) return;
  cudaFree(ptr);
  g_alloc_live.fetch_sub(1);
}

bool supported_n(int n) {
  return n == 16 || n == 32 || n == 64 || n == 96 || n == 128 || n == 192 || n == 256 || n == 512 ||
         n == 1024;
}

// Workspace slots, each N^3 floats (= a half spectrum of N^3/2 complex).
// 0-16 serve the forward map; 17-20 hold what the adjoint keeps of it.
enum Slot { S_A = 0, S_DELTA = 1, S_X0 = 2, S_Y0 = 7, S_RHO = 16, S_SHAT = 17, S_POS = 18, N_SLOTS = 21 };
constexpr int kMaxShells = 256;
constexpr int kMaxOutputs = 64;   // output scale factors per plan (lpt2_set_outputs)
constexpr int kMaxRec = 4096;
constexpr long long kDefaultWaitCycles = 2000000000LL;   // about one second at 2 GHz

}  // namespace

// Instances of one grid size run together: every pass kernel covers the whole
// group (grid z = instance).
struct Group {
  int n;
  double box;
  int count;
  int inst0;       // index of the group's first instance in the plan
  float2* tw;      // twiddles exp(-2 pi i m / n)
  size_t off;      // floats before the group's first instance in per-instance real fields
  float4* mt0;     // per-|n|^2 multiplier tables [count][mode_table_len(n)]
  float2* mt1;
  double* geo_k;             // P(k) shell geometry for geo_ns shells: sum of |k| per shell
  unsigned long long* geo_n; // and mode count per shell [kMaxShells]
  int geo_ns;                // 0: not computed yet
  int chunk = 0;             // instances per launch in lpt2_displace / lpt2_cic_pk (0: the whole group)
  int ytile = 0;             // y-pass pencils per CTA (0: build default, 8, 16)
  int xtile = 0;             // x-pass tile path of the delta and adjoint modes (0: default, 1: bulk-tensor, 2: global)
};

struct GraphCache {  // one captured launch sequence per entry point (LPT2_GRAPH)
  const void* key[8];
  cudaGraphExec_t exec;
  int64_t launches;
};

// Device side of lpt2_displace_host: two buffer sets (noise, positions, P(k)) in the
// caller's workspace so that the copies of one realisation overlap the kernels of the
// next, two copy streams and the events that order them (made by lpt2_plan).
struct HostIO {
  float* noise_d[2] = {};
  float* pos_d[2] = {};
  double* pk_d[2] = {};
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t start = nullptr, up_done[2] = {}, in_used[2] = {}, pos_ready[2] = {}, comp_done[2] = {},
              down_done[2] = {};
};

struct lpt2_plan_s {
  // current group (set by set_group): grid side, box, twiddles, batch
  int n;
  double box;
  float2* tw;
  const float4* mt0;
  const float2* mt1;
  int cur_batch, cur_inst0;
  int cur_ytile = 0, cur_xtile = 0;   // tile schedule of the current group
  size_t cur_slot_off = 0;    // bytes into every workspace slot of the current instances (a chunk of a group)
  size_t cur_rho_off = 0;     // floats into the density array of the current instances
  std::vector<Group> groups;
  int n_inst;
  uint64_t* seeds_dev;        // [n_inst]
  double* fr0_dev;            // [n_inst]
  int* dev_err;               // device error word written by bounded waits (0 = ok)
  float4* bm_tab;             // Box-Muller tables of the white noise (boxmuller.cuh)
  long long wait_cycles = kDefaultWaitCycles;   // budget of the bounded consumer waits
  double* gr_tab;             // [4][2] GR growth (D1_GR(a) / D1_GR(1)) for the source diagnostic
  float* gr_tabf;
  size_t slot_sz;             // bytes per workspace slot: max over groups of count n^3 4
  int xb_max;                 // max over groups of count * x-pass blocks
  size_t total_cells;         // sum over instances of n^3
  bool host_io;               // LPT2_HOST_IO: the workspace holds lpt2_displace_host's buffer sets
  bool keep_state;            // LPT2_KEEP_STATE: lpt2_displace keeps what the adjoint needs
  // what the workspace holds of the last forward map (LPT2_KEEP_STATE): fwd = delta(k), S(k),
  // positions and CIC density of lpt2_displace with noise `kept_noise`; spec = also the
  // density spectrum after the z and y passes (a later lpt2_cic_pk of that density)
  bool kept_fwd = false, kept_spec = false;
  const float* kept_noise = nullptr;
  int max_out;                // LPT2_MAX_OUTPUTS(n): room for n output times' tables in the workspace
  bool use_graph;
  GraphCache graphs[2] = {};  // lpt2_displace, lpt2_cic_pk
  uint64_t seed;
  double a_out;
  lpt2_cosmo cosmo;
  int nk;
  double k_min, k_max;
  int n_steps;
  cudaStream_t stream;
  DevCosmo* cosmo_dev;
  double* partials;
  double* tab;    // [n_inst][4][nk]
  float* tabf;    // [n_inst][4][nk]: D1, D2, dD1/dln|fR0|, dD2/dln|fR0| in FP32
  char* ws;
  size_t ws_bytes;
  int64_t launches;
  // per-launch CUDA-event timing (lpt2_timing)
  bool timing_on;
  int n_rec;
  cudaEvent_t* ev;            // 2 * kMaxRec events, created on first enable
  const char* rec_name[kMaxRec];
  double rec_bytes[kMaxRec];
  HostIO* hio = nullptr;      // lpt2_displace_host buffers and streams, made on first use
  // output scale factors of lpt2_displace_outputs (lpt2_set_outputs); per a_j the growth
  // tables [4][nk] (FP64, FP32) and the per-|n|^2 multiplier tables of the plan's grid sit
  // in the workspace (WsLayout::outs)
  int n_out_a = 0;
  std::vector<double> out_a;
};

namespace {

// algorithmic-byte unit of the current group: N^3 times the instances in the launch
double V3(const lpt2_plan_s* p) { return (double)p->n * p->n * p->n * p->cur_batch; }

size_t slot_bytes(const lpt2_plan_s* p) { return p->slot_sz; }

void set_group(lpt2_plan_s* p, int gi) {
  const Group& g = p->groups[gi];
  p->n = g.n;
  p->box = g.box;
  p->tw = g.tw;
  p->mt0 = g.mt0;
  p->mt1 = g.mt1;
  p->cur_batch = g.count;
  p->cur_inst0 = g.inst0;
  p->cur_ytile = g.ytile;
  p->cur_xtile = g.xtile;
  p->cur_slot_off = 0;
  p->cur_rho_off = g.off;
}

// Instances [c0, c0 + cnt) of group gi: the fields of a group's instances are consecutive
// in every workspace slot (one N^3 real field, or half spectrum, per instance), so a chunk
// is the group with offset slots, tables, seeds and density.
void set_chunk(lpt2_plan_s* p, int gi, int c0, int cnt) {
  set_group(p, gi);
  const Group& g = p->groups[gi];
  const size_t n3 = (size_t)g.n * g.n * g.n, len = (size_t)mode_table_len(g.n);
  p->cur_batch = cnt;
  p->cur_inst0 = g.inst0 + c0;
  p->mt0 = g.mt0 + (size_t)c0 * len;
  p->mt1 = g.mt1 + (size_t)c0 * len;
  p->cur_slot_off = (size_t)c0 * n3 * sizeof(float);
  p->cur_rho_off = g.off + (size_t)c0 * n3;
}

int chunk_of(const Group& g) { return g.chunk > 0 && g.chunk < g.count ? g.chunk : g.count; }

int x_blocks(int n) {
  switch (n) {
    case 16: return x_blocks_16();
    case 32: return x_blocks_32();
    case 64: return x_blocks_64();
    case 96: return x_blocks_96();
    case 128: return x_blocks_128();
    case 192: return x_blocks_192();
    case 256: return x_blocks_256();
    case 512: return x_blocks_512();
    default: return x_blocks_1024();
  }
}

// Workspace layout (byte offsets; every region 256-byte aligned):
//   N_SLOTS slots of slot_sz bytes, the CIC density of every instance (sum of n^3 floats),
//   sqrt(P N^3/V) per stored mode of every instance (sum of n^3 / 2 floats; filled by
//   lpt2_set_workspace from the mode tables, read by the x passes of delta(k)), P(k) block partials [xb_max][3][256] doubles, internal pk / k_mean / n_modes [256] each,
//   shell weights [256] floats, dL/dln|fR0| block partials [xb_max] doubles, P(k) per
//   instance [n_inst][256] doubles (lpt2_autotune), then with LPT2_HOST_IO two buffer sets
//   of lpt2_displace_host (noise n^3 floats, positions 3 n^3 floats, P(k) 256 doubles) and
//   with LPT2_MAX_OUTPUTS(m) m output times' tables (growth [4][nk] doubles and floats,
//   multiplier tables [mode_table_len] float4 and float2).
struct WsLayout {
  size_t slot_sz, rho, scf, pk_part, pk, shw, theta, inst_pk, hio, hio_noise, hio_pos, hio_pk, hio_set, outs,
      out_tab, out_tabf, out_mt0, out_mt1, out_each, total;
};
size_t up256(size_t b) { return (b + 255) / 256 * 256; }
WsLayout ws_layout(size_t slot_sz, size_t total_cells, int xb_max, int n_inst, int nk, int n0, bool host_io,
                   int max_out) {
  WsLayout w{};
  w.slot_sz = slot_sz;
  w.rho = N_SLOTS * slot_sz;
  w.scf = up256(w.rho + total_cells * sizeof(float));
  w.pk_part = up256(w.scf + total_cells / 2 * sizeof(float));
  w.pk = up256(w.pk_part + (size_t)xb_max * 3 * kMaxShells * 8);
  w.shw = up256(w.pk + 3 * kMaxShells * 8);
  w.theta = up256(w.shw + kMaxShells * 4);
  w.inst_pk = up256(w.theta + (size_t)xb_max * 8);
  w.hio = up256(w.inst_pk + (size_t)n_inst * kMaxShells * 8);
  const size_t n3 = (size_t)n0 * n0 * n0;
  w.hio_noise = 0;
  w.hio_pos = up256(n3 * sizeof(float));
  w.hio_pk = up256(w.hio_pos + 3 * n3 * sizeof(float));
  w.hio_set = up256(w.hio_pk + kMaxShells * 8);
  w.outs = w.hio + (host_io ? 2 * w.hio_set : 0);
  const size_t len = (size_t)mode_table_len(n0);
  w.out_tab = 0;
  w.out_tabf = up256((size_t)4 * nk * sizeof(double));
  w.out_mt0 = up256(w.out_tabf + (size_t)4 * nk * sizeof(float));
  w.out_mt1 = up256(w.out_mt0 + len * sizeof(float4));
  w.out_each = up256(w.out_mt1 + len * sizeof(float2));
  w.total = w.outs + (size_t)max_out * w.out_each;
  return w;
}
WsLayout ws_layout(const lpt2_plan_s* p) {
  return ws_layout(p->slot_sz, p->total_cells, p->xb_max, p->n_inst, p->nk, p->groups[0].n, p->host_io,
                   p->max_out);
}
size_t rho_all_off(const lpt2_plan_s* p) { return N_SLOTS * slot_bytes(p); }
float* rho_group(const lpt2_plan_s* p) {
  return reinterpret_cast<float*>(p->ws + rho_all_off(p)) + p->cur_rho_off;
}
// sqrt(P N^3/V) per mode of the current instances (the scf field of XArgs)
const float* scf_group(const lpt2_plan_s* p) {
  return reinterpret_cast<const float*>(p->ws + ws_layout(p).scf) + p->cur_rho_off / 2;
}
size_t tail_pk_part(const lpt2_plan_s* p) { return ws_layout(p).pk_part; }
size_t tail_shw(const lpt2_plan_s* p) { return ws_layout(p).shw; }
size_t tail_theta(const lpt2_plan_s* p) { return ws_layout(p).theta; }
size_t ws_need(const lpt2_plan_s* p) { return ws_layout(p).total; }

float2* slot(const lpt2_plan_s* p, int i) {
  return reinterpret_cast<float2*>(p->ws + i * slot_bytes(p) + p->cur_slot_off);
}
double* pk_part(const lpt2_plan_s* p) { return reinterpret_cast<double*>(p->ws + tail_pk_part(p)); }

Geo make_geo(const lpt2_plan_s* p) {
  Geo g{};
  const double n = p->n;
  g.n = p->n;
  g.kf = (float)(2.0 * M_PI / p->box);
  g.box = (float)p->box;
  g.cell = (float)(p->box / n);
  g.inv_cell = (float)(n / p->box);
  g.inv_n3 = (float)(1.0 / (n * n * n));
  g.sqrt_n3_over_v = (float)sqrt(n * n * n / (p->box * p->box * p->box));
  g.kf2n3 = (float)(4.0 * M_PI * M_PI / (p->box * p->box) * n * n * n);
  g.batch = p->cur_batch;
  g.inst0 = p->cur_inst0;
  g.tab_stride = 4 * p->nk;
  g.err = p->dev_err;
  g.wait = p->wait_cycles;
  g.ytile = p->cur_ytile;
  g.xtile = p->cur_xtile;
  return g;
}

GrowthParams growth_params(const lpt2_plan_s* p) {
  GrowthParams g;
  g.omega_m = p->cosmo.omega_m;
  g.omega_l = p->cosmo.omega_l;
  g.omega_b = p->cosmo.omega_b;
  g.h = p->cosmo.h;
  g.n_s = p->cosmo.n_s;
  g.sigma8 = p->cosmo.sigma8;
  g.t_cmb = p->cosmo.t_cmb;
  g.fr0_abs = p->cosmo.fr0_abs;
  g.a_init = p->cosmo.a_init;
  g.a_out = p->a_out;
  g.k_min = p->k_min;
  g.k_max = p->k_max;
  g.nk = p->nk;
  g.n_steps = p->n_steps;
  g.n_inst = p->n_inst;
  g.fr0s = p->fr0_dev;
  g.d2_variant = p->cosmo.d2_variant;
  return g;
}

#define DISPATCH(NAME, n, args, s)          \
  switch (n) {                              \
    case 16: return NAME##_16(args, s);     \
    case 32: return NAME##_32(args, s);     \
    case 64: return NAME##_64(args, s);     \
    case 96: return NAME##_96(args, s);     \
    case 128: return NAME##_128(args, s);   \
    case 192: return NAME##_192(args, s);   \
    case 256: return NAME##_256(args, s);   \
    case 512: return NAME##_512(args, s);   \
    default: return NAME##_1024(args, s);   \
  }

cudaError_t z_r2c(int n, const ZR2CArgs& a, cudaStream_t s) { DISPATCH(launch_z_r2c, n, a, s) }
cudaError_t z_c2r(int n, const ZC2RArgs& a, cudaStream_t s) { DISPATCH(launch_z_c2r, n, a, s) }
cudaError_t z_source(int n, const ZSourceArgs& a, cudaStream_t s) { DISPATCH(launch_z_source, n, a, s) }
cudaError_t z_final(int n, const ZFinalArgs& a, cudaStream_t s) { DISPATCH(launch_z_final, n, a, s) }
cudaError_t y_pass(int n, const YArgs& a, cudaStream_t s) { DISPATCH(launch_y, n, a, s) }
cudaError_t x_pass(int n, const XArgs& a, cudaStream_t s) { DISPATCH(launch_x, n, a, s) }
cudaError_t z_adj_source(int n, const ZAdjSourceArgs& a, cudaStream_t s) { DISPATCH(launch_z_adj_source, n, a, s) }

void timing_begin(lpt2_plan_s* p) {
  if (!p->timing_on || p->n_rec >= kMaxRec) return;
  cudaEventRecord(p->ev[2 * p->n_rec], p->stream);
}

void timing_end(lpt2_plan_s* p, const char* name, double bytes) {
  if (!p->timing_on || p->n_rec >= kMaxRec) return;
  cudaEventRecord(p->ev[2 * p->n_rec + 1], p->stream);
  p->rec_name[p->n_rec] = name;
  p->rec_bytes[p->n_rec] = bytes;
  p->n_rec++;
}

// Every kernel launch goes through LAUNCH(plan, name, algorithmic bytes, call):
// counts it and, when timing is on, brackets it with CUDA events on the plan's stream.
// counts it and, when timing is on, brackets it with CUDA events on the plan's stream; an
// NVTX range named after the pass marks the launch for timeline profilers.
#define LAUNCH(plan, name, bytes, expr)                                               \
  do {                                                                                \
    nvtxRangePushA(name);                                                             \
    timing_begin((plan));                                                             \
    cudaError_t e_ = (expr);                                                          \
    (plan)->launches++;                                                               \
    timing_end((plan), (name), (double)(bytes));                                      \
    nvtxRangePop();                                                                   \
    if (e_ != cudaSuccess)                                                            \
      return fail(LPT2_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));               \
  } while (0)

// NVTX range around one C-ABI call (the whole call, host side).
struct AbiRange {
  explicit AbiRange(const char* name) { nvtxRangePushA(name); }
  ~AbiRange() { nvtxRangePop(); }
};

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

int check_plan_ws(lpt2_plan_t p) {
  if (!p) return fail(LPT2_EINVAL, "null plan");
  if (!p->ws) return fail(LPT2_ENOWORKSPACE, "no workspace attached (lpt2_set_workspace)");
  return LPT2_OK;
}

// forward r2c of a real field (or the Philox noise) into `out`, z -> y -> x (plain)
int forward_zy(lpt2_plan_t p, int src, const float* in, float2* out) {
  ZR2CArgs z{};
  z.g = make_geo(p);
  z.tw = p->tw;
  z.src = src;
  z.in = in;
  z.seed_lo = (uint32_t)p->seed;
  z.seed_hi = (uint32_t)(p->seed >> 32);
  z.seeds = p->seeds_dev;
  z.bm = p->bm_tab;
  z.out = out;
  LAUNCH(p, src == Z_NOISE ? "z_r2c_noise" : (src == Z_DENSITY ? "z_r2c_density" : "z_r2c"),
         (src == Z_NOISE ? 4.0 : 8.0) * V3(p), z_r2c(p->n, z, p->stream));
  YArgs y{};
  y.g = z.g;
  y.tw = p->tw;
  y.inverse = 0;
  y.job.n_in = 1;
  y.job.n_out = 1;
  y.job.in[0] = out;
  y.job.out[0] = out;
  y.job.src[0] = 0;
  y.job.ord[0] = 0;
  LAUNCH(p, "y_fwd", 8.0 * V3(p), y_pass(p->n, y, p->stream));
  return LPT2_OK;
}

int displace_impl(lpt2_plan_t p, const float* noise, float* psi1, float* psi2, float* pos, void* dk,
                  float2* s_keep, float* pos_scratch = nullptr);

// Forgets the forward state kept for the adjoint (a call has overwritten the workspace).
void drop_state(lpt2_plan_t p) {
  p->kept_fwd = false;
  p->kept_spec = false;
}

// Forgets the output times (their tables live in the workspace).
void free_outputs(lpt2_plan_t p) {
  p->n_out_a = 0;
  p->out_a.clear();
}

void free_host_io(lpt2_plan_t p) {
  HostIO* h = p->hio;
  if (!h) return;
  for (int b = 0; b < 2; ++b) {
    for (cudaEvent_t e : {h->up_done[b], h->in_used[b], h->pos_ready[b], h->comp_done[b], h->down_done[b]})
      if (e) cudaEventDestroy(e);
  }
  if (h->start) cudaEventDestroy(h->start);
  if (h->s_in) cudaStreamDestroy(h->s_in);
  if (h->s_out) cudaStreamDestroy(h->s_out);
  delete h;
  p->hio = nullptr;
}

// Streams and events of lpt2_displace_host (plans made with LPT2_HOST_IO; made by lpt2_plan).
int make_host_io(lpt2_plan_t p) {
  p->hio = new HostIO();
  HostIO* h = p->hio;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b)
    for (cudaEvent_t* ev : {&h->up_done[b], &h->in_used[b], &h->pos_ready[b], &h->comp_done[b], &h->down_done[b]})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->start, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    free_host_io(p);
    return fail(LPT2_ECUDA, "host-io streams and events: %s", cudaGetErrorString(e));
  }
  return LPT2_OK;
}

// The two buffer sets of lpt2_displace_host in the workspace.
void host_io_buffers(lpt2_plan_t p) {
  const WsLayout w = ws_layout(p);
  HostIO* h = p->hio;
  for (int b = 0; b < 2; ++b) {
    char* base = p->ws + w.hio + b * w.hio_set;
    h->noise_d[b] = reinterpret_cast<float*>(base + w.hio_noise);
    h->pos_d[b] = reinterpret_cast<float*>(base + w.hio_pos);
    h->pk_d[b] = reinterpret_cast<double*>(base + w.hio_pk);
  }
}

// Shell geometry (mode counts, sum of |k|) of group gi for n_shells shells; made
// once per shell count, outside any graph capture, and reused by every P(k).
int ensure_geometry(lpt2_plan_t p, int gi, int n_shells) {
  Group& gr = p->groups[gi];
  if (gr.geo_ns == n_shells) return LPT2_OK;
  cudaError_t e = cudaMemsetAsync(gr.geo_k, 0, kMaxShells * sizeof(double), p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(gr.geo_n, 0, kMaxShells * sizeof(unsigned long long), p->stream);
  if (e != cudaSuccess) return fail(LPT2_ECUDA, "shell geometry: %s", cudaGetErrorString(e));
  LAUNCH(p, "shell_geometry", 0.0, launch_shell_geometry(gr.n, gr.box, n_shells, gr.geo_k, gr.geo_n, p->stream));
  gr.geo_ns = n_shells;
  return LPT2_OK;
}

// CIC (when positions are given) and P(k) of the current group (geometry made).
int cic_pk_group(lpt2_plan_t p, int gi, const float* pos, float* density, double* pk, double* k_mean,
                 int64_t* n_modes, int n_shells, float2* spec = nullptr) {
  const int n = p->n;
  const Geo g = make_geo(p);
  const size_t cells = (size_t)n * n * n * p->cur_batch;
  float* rho = rho_group(p);
  float2* A = spec ? spec : slot(p, S_A);   // density spectrum scratch
  if (pos) {
    LAUNCH(p, "fill0", 4.0 * V3(p), launch_fill0(rho, cells, p->stream));
    CicArgs c{g, pos, rho};
    LAUNCH(p, "cic", 20.0 * V3(p), launch_cic(c, p->stream));
  }
  int rc = forward_zy(p, Z_DENSITY, rho, A);   // rho - 1 is formed in the z pass; rho is kept
  if (rc) return rc;
  if (density) LAUNCH(p, "contrast", 8.0 * V3(p), launch_contrast(rho, density, cells, p->stream));
  XArgs x{};
  x.g = g;
  x.tw = p->tw;
  x.mode = X_PKP;
  x.in = A;
  x.cosmo = p->cosmo_dev;
  x.pk_part = pk_part(p);
  x.n_shells = n_shells;
  LAUNCH(p, "x_pk", 4.0 * V3(p), x_pass(n, x, p->stream));
  const Group& gr = p->groups[gi];
  LAUNCH(p, "pk_finalize", 0.0,
         launch_pk_finalize_p(pk_part(p), x_blocks(n), n_shells, gr.geo_k, gr.geo_n, pk, k_mean, n_modes,
                              p->stream, p->cur_batch));
  ++p->launches;   // two kernels: row-slice sums, then the shells
  return LPT2_OK;
}

// Runs `body` through a CUDA graph captured on the plan's stream; the graph is
// re-captured when any pointer in `key` changes.
template <class F>
int run_graph(lpt2_plan_t p, int slot_i, const void* const key[8], F body) {
  GraphCache& gc = p->graphs[slot_i];
  bool same = gc.exec != nullptr;
  for (int i = 0; i < 8 && same; ++i) same = (gc.key[i] == key[i]);
  if (!same) {
    const bool timing = p->timing_on;
    p->timing_on = false;
    cudaError_t e = cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
      p->timing_on = timing;
      return fail(LPT2_ECUDA, "stream capture: %s", cudaGetErrorString(e));
    }
    const int64_t l0 = p->launches;
    const int rc = body();
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(p->stream, &graph);
    p->timing_on = timing;
    const int64_t captured = p->launches - l0;
    p->launches = l0;
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return fail(LPT2_ECUDA, "end capture: %s", cudaGetErrorString(e));
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(LPT2_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    if (gc.exec) cudaGraphExecDestroy(gc.exec);
    gc.exec = exec;
    gc.launches = captured;
    for (int i = 0; i < 8; ++i) gc.key[i] = key[i];
  }
  cudaError_t e = cudaGraphLaunch(gc.exec, p->stream);
  if (e != cudaSuccess) return fail(LPT2_ECUDA, "graph launch: %s", cudaGetErrorString(e));
  p->launches += gc.launches;
  return LPT2_OK;
}

// Growth and multiplier tables of output scale factor j, in the workspace.
double* out_tab(lpt2_plan_t p, int j) {
  const WsLayout w = ws_layout(p);
  return reinterpret_cast<double*>(p->ws + w.outs + j * w.out_each + w.out_tab);
}
float* out_tabf(lpt2_plan_t p, int j) {
  const WsLayout w = ws_layout(p);
  return reinterpret_cast<float*>(p->ws + w.outs + j * w.out_each + w.out_tabf);
}
float4* out_mt0(lpt2_plan_t p, int j) {
  const WsLayout w = ws_layout(p);
  return reinterpret_cast<float4*>(p->ws + w.outs + j * w.out_each + w.out_mt0);
}
float2* out_mt1(lpt2_plan_t p, int j) {
  const WsLayout w = ws_layout(p);
  return reinterpret_cast<float2*>(p->ws + w.outs + j * w.out_each + w.out_mt1);
}

// Growth and multiplier tables of every output scale factor (single-instance plan).
int run_output_growth(lpt2_plan_t p) {
  GrowthParams gp = growth_params(p);
  for (int j = 0; j < p->n_out_a; ++j) {
    gp.a_out = p->out_a[j];
    LAUNCH(p, "growth", 0.0, launch_growth(gp, out_tab(p, j), out_tabf(p, j), p->stream));
    LAUNCH(p, "mode_tables", 0.0,
           launch_mode_tables(gp, p->cosmo_dev, out_tab(p, j), 0, 1, p->groups[0].n, p->groups[0].box,
                              out_mt0(p, j), out_mt1(p, j), p->stream));
  }
  return LPT2_OK;
}

int run_growth(lpt2_plan_t p) {
  const GrowthParams gp = growth_params(p);
  LAUNCH(p, "growth", 0.0, launch_growth(gp, p->tab, p->tabf, p->stream));
  for (const Group& g : p->groups)
    LAUNCH(p, "mode_tables", 0.0,
           launch_mode_tables(gp, p->cosmo_dev, p->tab, g.inst0, g.count, g.n, g.box, g.mt0, g.mt1, p->stream));
  return p->n_out_a > 0 ? run_output_growth(p) : LPT2_OK;   // |fR0| changed: output tables too
}

}  // namespace

void lpt2::set_last_error(const char* msg) { g_err = msg; }

extern "C" {

const char* lpt2_last_error(void) { return g_err.c_str(); }

int64_t lpt2_launch_count(lpt2_plan_t plan) { return plan ? plan->launches : -1; }

int lpt2_device_status(lpt2_plan_t p) {
  if (!p) return fail(LPT2_EINVAL, "null plan");
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return fail(LPT2_ECUDA, "stream: %s", cudaGetErrorString(e));
  int code = 0;
  e = cudaMemcpy(&code, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(LPT2_ECUDA, "error word: %s", cudaGetErrorString(e));
  if (code) {
    cudaMemset(p->dev_err, 0, sizeof(int));
    return fail(LPT2_ETIMEOUT, "a bounded device-side wait gave up (kernel code %d); outputs of the "
                "launches since the last check are invalid", code);
  }
  return LPT2_OK;
}

static int check_cosmo(const lpt2_instance* inst) {
  const lpt2_cosmo& c = inst->cosmo;
  if (!supported_n(inst->n)) return fail(LPT2_EUNSUPPORTED, "grid size %d not supported", inst->n);
  if (!(inst->box > 0) || !isfinite(inst->box)) return fail(LPT2_EINVAL, "box must be > 0");
  if (!(c.a_init > 0) || !(inst->a_out > c.a_init) || !(inst->a_out <= 1.0))
    return fail(LPT2_EINVAL, "need 0 < a_init < a_out <= 1");
  if (!(c.omega_m > 0) || !(c.omega_l >= 0) || fabs(c.omega_m + c.omega_l - 1.0) > 1e-6)
    return fail(LPT2_EINVAL, "cosmology must be flat with omega_m > 0");
  if (!(c.h > 0) || !(c.sigma8 > 0) || !(c.omega_b > 0) || !(c.omega_b < c.omega_m) || !(c.t_cmb > 0))
    return fail(LPT2_EINVAL, "bad h / sigma8 / omega_b / t_cmb");
  if (!(c.fr0_abs >= 0) || !isfinite(c.fr0_abs)) return fail(LPT2_EINVAL, "fr0_abs must be >= 0");
  if (c.hs_n != 1) return fail(LPT2_EUNSUPPORTED, "only Hu-Sawicki n = 1 is supported");
  if (c.d2_variant < LPT2_D2_T1 || c.d2_variant > LPT2_D2_LCDM_FIT)
    return fail(LPT2_EUNSUPPORTED, "d2_variant must be one of LPT2_D2_T1 .. LPT2_D2_LCDM_FIT");
  return LPT2_OK;
}

static bool same_background(const lpt2_instance& a, const lpt2_instance& b) {
  const lpt2_cosmo &x = a.cosmo, &y = b.cosmo;
  return x.omega_m == y.omega_m && x.omega_l == y.omega_l && x.omega_b == y.omega_b && x.h == y.h &&
         x.n_s == y.n_s && x.sigma8 == y.sigma8 && x.t_cmb == y.t_cmb && x.a_init == y.a_init &&
         x.hs_n == y.hs_n && x.d2_variant == y.d2_variant && a.a_out == b.a_out;
}

// Host-side checks shared by lpt2_plan and lpt2_workspace_bytes: the instance list, n_k and
// the flags; on success the grid-size groups and the workspace sizes of such a plan.
struct PlanShape {
  std::vector<Group> groups;
  size_t slot_sz = 0, total_cells = 0;
  int xb_max = 0;
  bool host_io = false;
  int max_out = 0;
};
static int plan_shape(const lpt2_instance* inst, int n_inst, int n_k, unsigned flags, PlanShape& ps) {
  if (!inst) return fail(LPT2_EINVAL, "null inst pointer");
  if (n_inst < 1 || n_inst > 65535) return fail(LPT2_EINVAL, "n_inst must be in [1, 65535] (got %d)", n_inst);
  const unsigned known = LPT2_GRAPH | LPT2_HOST_IO | LPT2_KEEP_STATE | LPT2_MAX_OUTPUTS(0xff);
  if (flags & ~known) return fail(LPT2_EINVAL, "unknown flags");
  ps.host_io = (flags & LPT2_HOST_IO) != 0;
  ps.max_out = (int)((flags >> 8) & 0xff);
  if (ps.max_out > kMaxOutputs) return fail(LPT2_EINVAL, "LPT2_MAX_OUTPUTS(n): n must be <= %d", kMaxOutputs);
  if ((ps.host_io || ps.max_out > 0 || (flags & LPT2_KEEP_STATE)) && n_inst != 1)
    return fail(LPT2_EINVAL, "LPT2_HOST_IO, LPT2_KEEP_STATE and LPT2_MAX_OUTPUTS need a single-instance plan");
  if (n_k < 2 || n_k > 4096) return fail(LPT2_EINVAL, "n_k must be in [2, 4096]");
  std::vector<Group>& groups = ps.groups;
  for (int i = 0; i < n_inst; ++i) {
    const int rc = check_cosmo(&inst[i]);
    if (rc) return rc;
    if (!same_background(inst[i], inst[0]))
      return fail(LPT2_EINVAL, "instance %d: all instances must share the background cosmology and a_out "
                               "(only fr0_abs and seed may differ)", i);
    if (groups.empty() || groups.back().n != inst[i].n) {
      for (const Group& g : groups)
        if (g.n == inst[i].n)
          return fail(LPT2_EINVAL, "instances of equal grid size must be contiguous (instance %d)", i);
      groups.push_back(Group{inst[i].n, inst[i].box, 0, i, nullptr});
    }
    if (inst[i].box != groups.back().box)
      return fail(LPT2_EUNSUPPORTED, "instances of one grid size must share the box (instance %d)", i);
    groups.back().count++;
  }
  for (Group& g : groups) {
    g.off = ps.total_cells;
    ps.total_cells += (size_t)g.count * g.n * g.n * g.n;
    const size_t sz = (size_t)g.count * g.n * g.n * g.n * sizeof(float);
    if (sz > ps.slot_sz) ps.slot_sz = sz;
    if (g.count * x_blocks(g.n) > ps.xb_max) ps.xb_max = g.count * x_blocks(g.n);
  }
  return LPT2_OK;
}

int lpt2_set_wait_budget(lpt2_plan_t p, int64_t cycles) {
  if (!p) return fail(LPT2_EINVAL, "null plan");
  if (cycles < 0) return fail(LPT2_EINVAL, "cycles must be >= 0");
  p->wait_cycles = cycles;
  for (auto& gc : p->graphs) {   // captured launches carry the old budget
    if (gc.exec) cudaGraphExecDestroy(gc.exec);
    gc.exec = nullptr;
  }
  return LPT2_OK;
}

int lpt2_debug_alloc_hook(int fail_at, int64_t* live) {
  if (fail_at < -1) return fail(LPT2_EINVAL, "fail_at must be >= -1");
  g_fail_alloc_at.store(fail_at);
  g_alloc_calls.store(0);
  if (live) *live = (int64_t)g_alloc_live.load();
  return LPT2_OK;
}

int lpt2_workspace_bytes(const lpt2_instance* inst, int n_inst, int n_k, unsigned flags, size_t* bytes) {
  if (!bytes) return fail(LPT2_EINVAL, "null bytes pointer");
  PlanShape ps;
  const int rc = plan_shape(inst, n_inst, n_k, flags, ps);
  if (rc) return rc;
  *bytes = ws_layout(ps.slot_sz, ps.total_cells, ps.xb_max, n_inst, n_k, ps.groups[0].n, ps.host_io, ps.max_out)
               .total;
  return LPT2_OK;
}

int lpt2_plan(lpt2_plan_t* out, const lpt2_instance* inst, int n_inst, int n_k, double k_min,
              double k_max, int n_steps, void* cuda_stream, unsigned flags) {
  AbiRange nvtx_range("lpt2_plan");
  g_err.clear();
  if (!out || !inst) return fail(LPT2_EINVAL, "null out/inst pointer");
  *out = nullptr;
  if ((flags & LPT2_GRAPH) && cuda_stream == nullptr)
    return fail(LPT2_EINVAL, "LPT2_GRAPH needs a stream other than the legacy default stream");
  if (!(k_min > 0) || !(k_max > k_min)) return fail(LPT2_EINVAL, "need 0 < k_min < k_max");
  if (n_steps < 1 || n_steps > 2800) return fail(LPT2_EINVAL, "n_steps must be in [1, 2800]");
  PlanShape ps;
  const int prc = plan_shape(inst, n_inst, n_k, flags, ps);
  if (prc) return prc;

  lpt2_plan_s* p = new lpt2_plan_s();
  p->groups = ps.groups;
  p->n_inst = n_inst;
  p->seed = inst[0].seed;
  p->a_out = inst[0].a_out;
  p->cosmo = inst[0].cosmo;
  p->nk = n_k;
  p->k_min = k_min;
  p->k_max = k_max;
  p->n_steps = n_steps;
  p->stream = (cudaStream_t)cuda_stream;
  p->use_graph = (flags & LPT2_GRAPH) != 0;
  p->slot_sz = ps.slot_sz;
  p->xb_max = ps.xb_max;
  p->total_cells = ps.total_cells;
  p->host_io = ps.host_io;
  p->keep_state = (flags & LPT2_KEEP_STATE) != 0;
  p->max_out = ps.max_out;
  cudaError_t e = cudaSuccess;
  for (Group& g : p->groups) {
    if (e == cudaSuccess) e = plan_malloc((void**)&g.tw, g.n * sizeof(float2));
    if (e == cudaSuccess) e = plan_malloc((void**)&g.mt0, (size_t)g.count * mode_table_len(g.n) * sizeof(float4));
    if (e == cudaSuccess) e = plan_malloc((void**)&g.mt1, (size_t)g.count * mode_table_len(g.n) * sizeof(float2));
    if (e == cudaSuccess) e = plan_malloc((void**)&g.geo_k, kMaxShells * sizeof(double));
    if (e == cudaSuccess) e = plan_malloc((void**)&g.geo_n, kMaxShells * sizeof(unsigned long long));
    g.geo_ns = 0;
  }
  if (e == cudaSuccess) e = plan_malloc((void**)&p->cosmo_dev, sizeof(DevCosmo));
  if (e == cudaSuccess) e = plan_malloc((void**)&p->partials, cosmo_partial_blocks() * sizeof(double));
  if (e == cudaSuccess) e = plan_malloc((void**)&p->tab, (size_t)n_inst * 4 * n_k * sizeof(double));
  if (e == cudaSuccess) e = plan_malloc((void**)&p->tabf, (size_t)n_inst * 4 * n_k * sizeof(float));
  if (e == cudaSuccess) e = plan_malloc((void**)&p->seeds_dev, (size_t)n_inst * sizeof(uint64_t));
  if (e == cudaSuccess) e = plan_malloc((void**)&p->fr0_dev, (size_t)n_inst * sizeof(double));
  if (e == cudaSuccess) e = plan_malloc((void**)&p->dev_err, sizeof(int));
  if (e == cudaSuccess) e = plan_malloc((void**)&p->bm_tab, kBmTableLen * sizeof(float4));
  if (e == cudaSuccess) e = plan_malloc((void**)&p->gr_tab, 8 * sizeof(double));
  if (e == cudaSuccess) e = plan_malloc((void**)&p->gr_tabf, 8 * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(p->dev_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    lpt2_plan_destroy(p);
    return fail(e == cudaErrorMemoryAllocation ? LPT2_ENOMEM : LPT2_ECUDA, "plan allocation failed: %s",
                cudaGetErrorString(e));
  }
  // twiddles exp(-2 pi i m / N), FP64 then rounded once
  for (Group& g : p->groups) {
    std::vector<float2> tw(g.n);
    for (int m = 0; m < g.n; ++m) {
      const double ang = 2.0 * M_PI * (double)m / (double)g.n;
      tw[m] = make_float2((float)cos(ang), (float)(-sin(ang)));
    }
    e = cudaMemcpy(g.tw, tw.data(), g.n * sizeof(float2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) break;
  }
  std::vector<uint64_t> seeds(n_inst);
  std::vector<double> fr0s(n_inst);
  for (int i = 0; i < n_inst; ++i) {
    seeds[i] = inst[i].seed;
    fr0s[i] = inst[i].cosmo.fr0_abs;
  }
  std::vector<float4> bm(kBmTableLen);
  bm_table(bm.data());
  if (e == cudaSuccess) e = cudaMemcpy(p->bm_tab, bm.data(), kBmTableLen * sizeof(float4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->seeds_dev, seeds.data(), n_inst * sizeof(uint64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->fr0_dev, fr0s.data(), n_inst * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    lpt2_plan_destroy(p);
    return fail(LPT2_ECUDA, "plan upload: %s", cudaGetErrorString(e));
  }
  set_group(p, 0);
  const GrowthParams gp = growth_params(p);
  e = launch_cosmo_setup(gp, p->partials, p->cosmo_dev, p->stream);
  p->launches += 2;   // partial sums + final
  if (e != cudaSuccess) {
    lpt2_plan_destroy(p);
    return fail(LPT2_ECUDA, "set-up kernels: %s", cudaGetErrorString(e));
  }
  int rc = run_growth(p);   // growth tables, then the per-|n|^2 multiplier tables
  if (!rc && p->host_io) rc = make_host_io(p);
  if (rc) {
    lpt2_plan_destroy(p);
    return rc;
  }
  *out = p;
  return LPT2_OK;
}

int lpt2_plan_destroy(lpt2_plan_t p) {
  if (!p) return LPT2_OK;
  for (Group& g : p->groups) {
    plan_free(g.tw);
    plan_free(g.mt0);
    plan_free(g.mt1);
    plan_free(g.geo_k);
    plan_free(g.geo_n);
  }
  plan_free(p->cosmo_dev);
  plan_free(p->partials);
  plan_free(p->tab);
  plan_free(p->tabf);
  plan_free(p->seeds_dev);
  plan_free(p->fr0_dev);
  plan_free(p->dev_err);
  plan_free(p->bm_tab);
  plan_free(p->gr_tab);
  plan_free(p->gr_tabf);
  for (auto& gc : p->graphs)
    if (gc.exec) cudaGraphExecDestroy(gc.exec);
  if (p->ev) {
    for (int i = 0; i < 2 * kMaxRec; ++i) cudaEventDestroy(p->ev[i]);
    delete[] p->ev;
  }
  free_host_io(p);
  free_outputs(p);
  delete p;
  return LPT2_OK;
}

int lpt2_workspace_size(lpt2_plan_t p, size_t* bytes) {
  if (!p || !bytes) return fail(LPT2_EINVAL, "null argument");
  *bytes = ws_need(p);
  return LPT2_OK;
}

int lpt2_set_workspace(lpt2_plan_t p, void* dev_ptr, size_t bytes) {
  if (p) drop_state(p);   // overwrites the state kept for the adjoint
  if (!p || !dev_ptr) return fail(LPT2_EINVAL, "null argument");
  if (!aligned(dev_ptr, 256)) return fail(LPT2_EINVAL, "workspace must be 256-byte aligned");
  if (bytes < ws_need(p)) return fail(LPT2_ENOWORKSPACE, "workspace too small: %zu < %zu", bytes, ws_need(p));
  p->ws = (char*)dev_ptr;
  p->ws_bytes = bytes;
  // the sqrt(P N^3/V) field of every group (P(k) only: no later call changes it)
  for (const Group& g : p->groups)
    LAUNCH(p, "sc_field", 2.0 * g.n * g.n * (double)g.n * g.count,
           launch_sc_field(g.mt0, g.n, g.count,
                           reinterpret_cast<float*>(p->ws + ws_layout(p).scf) + g.off / 2, p->stream));
  return p->n_out_a > 0 ? run_output_growth(p) : LPT2_OK;   // the output tables live in the workspace
}

int lpt2_growth_tables(lpt2_plan_t p, double* d1, double* d2, double* dd1, double* dd2) {
  if (p) drop_state(p);   // overwrites the state kept for the adjoint
  AbiRange nvtx_range("lpt2_growth_tables");
  if (!p) return fail(LPT2_EINVAL, "null plan");
  int rc = run_growth(p);
  if (rc) return rc;
  double* dst[4] = {d1, d2, dd1, dd2};
  for (int i = 0; i < 4; ++i) {   // plan tables are [n_inst][4][nk]; outputs [n_inst][nk]
    if (!dst[i]) continue;
    cudaError_t e = cudaMemcpy2DAsync(dst[i], p->nk * sizeof(double), p->tab + (size_t)i * p->nk,
                                      4 * p->nk * sizeof(double), p->nk * sizeof(double), p->n_inst,
                                      cudaMemcpyDeviceToDevice, p->stream);
    if (e != cudaSuccess) return fail(LPT2_ECUDA, "table copy: %s", cudaGetErrorString(e));
  }
  return LPT2_OK;
}

int lpt2_white_noise(lpt2_plan_t p, float* noise) {
  if (!p || !noise) return fail(LPT2_EINVAL, "null argument");
  if (p->n_inst != 1) return fail(LPT2_EUNSUPPORTED, "lpt2_white_noise needs a single-instance plan");
  if (!aligned(noise, 4)) return fail(LPT2_EINVAL, "misaligned output");
  LAUNCH(p, "noise", 4.0 * V3(p),
         launch_noise(make_geo(p), (uint32_t)p->seed, (uint32_t)(p->seed >> 32), p->bm_tab, noise, p->stream));
  return LPT2_OK;
}

int lpt2_box_muller(lpt2_plan_t p, const uint32_t* words, int64_t count, float* out) {
  if (!p || (count > 0 && (!words || !out))) return fail(LPT2_EINVAL, "null argument");
  if (count < 0 || count > (1LL << 31)) return fail(LPT2_EINVAL, "count must be in [0, 2^31]");
  if (!aligned(words, 8) || !aligned(out, 8)) return fail(LPT2_EINVAL, "words and out must be 8-byte aligned");
  if (count == 0) return LPT2_OK;
  LAUNCH(p, "box_muller", 16.0 * count, launch_box_muller(words, count, p->bm_tab, out, p->stream));
  return LPT2_OK;
}

int lpt2_philox_words(uint64_t seed, uint64_t first, int64_t count, uint32_t* out, void* stream) {
  if (!out || count < 0 || count > (1LL << 31)) return fail(LPT2_EINVAL, "bad philox arguments");
  if (!aligned(out, 16)) return fail(LPT2_EINVAL, "output must be 16-byte aligned");
  if (count == 0) return LPT2_OK;
  cudaError_t e = launch_philox_words((uint32_t)seed, (uint32_t)(seed >> 32), first, count, out,
                                      (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(LPT2_ECUDA, "philox: %s", cudaGetErrorString(e));
  return LPT2_OK;
}

int lpt2_displace(lpt2_plan_t p, const float* noise, float* psi1, float* psi2, float* pos, void* dk) {
  AbiRange nvtx_range("lpt2_displace");
  int rc = check_plan_ws(p);
  if (rc) return rc;
  if (dk && !aligned(dk, 16)) return fail(LPT2_EINVAL, "dk must be 16-byte aligned");
  drop_state(p);
  // with LPT2_KEEP_STATE a forward to the CIC density only (no Psi, no positions out) also
  // keeps S(k) and the positions in the slots the adjoint reads them from
  const bool keep = p->keep_state && !psi1 && !psi2 && !pos;
  auto body = [&]() -> int {
    for (int gi = 0; gi < (int)p->groups.size(); ++gi) {
      const Group& gr = p->groups[gi];
      const size_t n3 = (size_t)gr.n * gr.n * gr.n;
      for (int c0 = 0; c0 < gr.count; c0 += chunk_of(gr)) {
        set_chunk(p, gi, c0, std::min(chunk_of(gr), gr.count - c0));
        const size_t off = gr.off + (size_t)c0 * n3;   // real elements before the chunk
        const int r = displace_impl(p, noise ? noise + off : nullptr, psi1 ? psi1 + 3 * off : nullptr,
                                    psi2 ? psi2 + 3 * off : nullptr, pos ? pos + 3 * off : nullptr,
                                    dk ? (char*)dk + off * sizeof(float) : nullptr,
                                    keep ? slot(p, S_SHAT) : nullptr,
                                    keep ? reinterpret_cast<float*>(slot(p, S_POS)) : nullptr);
        if (r) return r;
      }
    }
    set_group(p, 0);
    return LPT2_OK;
  };
  const void* key[8] = {noise, psi1, psi2, pos, dk, p->ws, nullptr, nullptr};
  const int r = p->use_graph ? run_graph(p, 0, key, body) : body();
  if (!r && keep) {
    p->kept_fwd = true;
    p->kept_noise = noise;
  }
  return r;
}

}  // extern "C"

namespace {

// The forward map; s_keep (k space, may be null) receives S(k) for the adjoint.
// Slots of the forward path: A (S_A) carries the noise / S spectrum, D (S_DELTA) delta(k),
// X[0..4] the x-pass outputs, Y[0..8] the y-pass outputs.
struct FwdSlots {
  float2* A;
  float2* D;
  float2* X[5];
  float2* Y[9];
  float2* P[6];   // the six phi_ij of the unsplit path (y-pass output order)
};

// Slots of the six phi_ij on the unsplit forward path: none of them is written again by the
// rest of the forward, by lpt2_cic_pk, or by the adjoint before its source transpose, so
// the adjoint reads the forward's phi_ij there instead of recomputing them from delta(k).
constexpr int kPhiSlots[6] = {5, 6, 13, 14, 15, 16};

FwdSlots fwd_slots(lpt2_plan_t p) {
  FwdSlots f;
  f.A = slot(p, S_A);
  f.D = slot(p, S_DELTA);
  for (int i = 0; i < 5; ++i) f.X[i] = slot(p, S_X0 + i);
  for (int i = 0; i < 9; ++i) f.Y[i] = slot(p, S_Y0 + i);
  for (int i = 0; i < 6; ++i) f.P[i] = slot(p, kPhiSlots[i]);
  return f;
}

// Steps that do not depend on the output scale factor: noise -> delta(k) (slot D) and
// the phi potentials (+ Psi1 when split), the six phi_ij, the source term S and its z and
// y forward transforms (slot A).
int displace_prefix(lpt2_plan_t p, const FwdSlots& f, const float* noise, bool split) {
  const int n = p->n;
  const Geo g = make_geo(p);
  // 1. delta(k): noise -> z, y passes; x pass with sqrt(P) and the phi / Psi1 potentials
  int rc = forward_zy(p, noise ? Z_REAL : Z_NOISE, noise, f.A);
  if (rc) return rc;
  XArgs x{};
  x.g = g;
  x.tw = p->tw;
  x.mode = X_DELTA;
  x.split = split;
  x.in = f.A;
  x.scf = scf_group(p);
  x.delta_out = f.D;
  for (int i = 0; i < 5; ++i) x.out[i] = f.X[i];
  x.cosmo = p->cosmo_dev;
  x.mt0 = p->mt0;
  x.mt1 = p->mt1;
  x.d1f = p->tabf;
  x.d2f = p->tabf + p->nk;
  x.t1f = p->tabf + 2 * p->nk;
  x.t2f = p->tabf + 3 * p->nk;
  LAUNCH(p, "x_delta", (split ? 28.0 : 22.0) * V3(p), x_pass(n, x, p->stream));   // + the sqrt(P) field

  // 2. y inverse with y derivatives: the six phi_ij (+ Psi1)
  YArgs y{};
  y.g = g;
  y.tw = p->tw;
  y.inverse = 1;
  y.job.n_in = split ? 5 : 3;
  for (int i = 0; i < 5; ++i) y.job.in[i] = f.X[i];
  const int src[9] = {0, 0, 0, 1, 1, 2, 3, 3, 4};
  const int ord[9] = {0, 1, 2, 0, 1, 0, 0, 1, 0};
  y.job.n_out = split ? 9 : 6;
  for (int o = 0; o < 9; ++o) {
    y.job.out[o] = (split || o >= 6) ? f.Y[o] : f.P[o];   // split: Psi1 parts in Y[6..8]
    y.job.src[o] = src[o];
    y.job.ord[o] = ord[o];
  }
  LAUNCH(p, "y_phi", (split ? 56.0 : 36.0) * V3(p), y_pass(n, y, p->stream));

  // 3. z inverse of phi_ij, source term, z forward of S
  ZSourceArgs zs{};
  zs.g = g;
  zs.tw = p->tw;
  float2* const* ph = split ? f.Y : f.P;
  const float2* phi[6] = {ph[5], ph[2], ph[0], ph[4], ph[3], ph[1]};   // xx yy zz xy xz yz
  const int zord[6] = {0, 0, 2, 0, 1, 1};
  for (int i = 0; i < 6; ++i) {
    zs.in[i] = phi[i];
    zs.ord[i] = zord[i];
  }
  zs.out = f.A;
  LAUNCH(p, "z_source", 28.0 * V3(p), z_source(n, zs, p->stream));
  YArgs yf{};
  yf.g = g;
  yf.tw = p->tw;
  yf.inverse = 0;
  yf.job.n_in = 1;
  yf.job.n_out = 1;
  yf.job.in[0] = f.A;
  yf.job.out[0] = f.A;
  LAUNCH(p, "y_fwd", 8.0 * V3(p), y_pass(n, yf, p->stream));
  return LPT2_OK;
}

// Steps of one output scale factor, whose D1(k, a), D2(k, a) enter through the
// multiplier tables mt0 / mt1 and the growth tables tabf: S(k) -> phi2 (+ phi1 D1),
// Psi, positions, CIC density (slots A and D are read, not written).
int displace_suffix(lpt2_plan_t p, const FwdSlots& f, bool split, float* psi1, float* psi2, float* pos,
                    float2* s_keep, const float4* mt0, const float2* mt1, const float* tabf,
                    float* pos_scratch = nullptr) {
  const int n = p->n;
  const Geo g = make_geo(p);
  float* rho = rho_group(p);
  const size_t cells = (size_t)n * n * n * p->cur_batch;   // real elements of the group

  // 4. x pass: S(k) -> phi2 = -S D2/k^2 (+ D1 delta/k^2 when not split), x inverse
  XArgs xs{};
  xs.g = g;
  xs.tw = p->tw;
  xs.mode = X_SOURCE;
  xs.split = split;
  xs.in = f.A;
  xs.s_out = s_keep;
  xs.delta_out = nullptr;
  xs.delta_in = f.D;
  xs.out[0] = f.X[0];
  xs.out[1] = f.X[1];
  xs.cosmo = p->cosmo_dev;
  xs.mt0 = mt0;
  xs.mt1 = mt1;
  xs.d1f = tabf;
  xs.d2f = tabf + p->nk;
  xs.t1f = tabf + 2 * p->nk;
  xs.t2f = tabf + 3 * p->nk;
  LAUNCH(p, "x_source", (split ? 12.0 : 16.0) * V3(p), x_pass(n, xs, p->stream));

  // 5. y inverse: (x0 y0), (x0 y1), (x1 y0)
  YArgs y2{};
  y2.g = g;
  y2.tw = p->tw;
  y2.inverse = 1;
  y2.job.n_in = 2;
  y2.job.in[0] = f.X[0];
  y2.job.in[1] = f.X[1];
  y2.job.n_out = 3;
  const int src2[3] = {0, 0, 1}, ord2[3] = {0, 1, 0};
  for (int o = 0; o < 3; ++o) {
    y2.job.out[o] = f.Y[o];
    y2.job.src[o] = src2[o];
    y2.job.ord[o] = ord2[o];
  }
  LAUNCH(p, "y_psi", 20.0 * V3(p), y_pass(n, y2, p->stream));

  // 6. z inverse, positions, CIC
  LAUNCH(p, "fill0", 4.0 * V3(p), launch_fill0(rho, cells, p->stream));
  ZFinalArgs zf{};
  zf.g = g;
  zf.tw = p->tw;
  zf.split = split;
  for (int i = 0; i < 3; ++i) {
    zf.a[i] = split ? f.Y[6 + i] : f.Y[i];
    zf.b[i] = f.Y[i];
  }
  zf.psi1 = psi1;
  zf.psi2 = psi2;
  // The CIC deposit runs as its own kernel at full occupancy (atomic throughput
  // needs many warps in flight): z_final writes the positions (to the caller's
  // array, or to dead workspace slots 2-4) and k_cic reads them back.
  float* posw = pos ? pos : (pos_scratch ? pos_scratch : reinterpret_cast<float*>(f.X[0]));
  zf.pos = posw;
  LAUNCH(p, "z_final", ((split ? 24.0 : 12.0) + 12.0 + (psi1 ? 12.0 : 0.0) + (psi2 ? 12.0 : 0.0)) * V3(p),
         z_final(n, zf, p->stream));
  CicArgs ca{g, posw, rho};
  LAUNCH(p, "cic", 20.0 * V3(p), launch_cic(ca, p->stream));
  return LPT2_OK;
}

int displace_impl(lpt2_plan_t p, const float* noise, float* psi1, float* psi2, float* pos, void* dk,
                  float2* s_keep, float* pos_scratch) {
  const bool split = psi1 || psi2;
  const FwdSlots f = fwd_slots(p);
  int rc = displace_prefix(p, f, noise, split);
  if (rc) return rc;
  rc = displace_suffix(p, f, split, psi1, psi2, pos, s_keep, p->mt0, p->mt1, p->tabf, pos_scratch);
  if (rc) return rc;
  if (dk) {
    const size_t cells = (size_t)p->n * p->n * p->n * p->cur_batch;
    cudaError_t e = cudaMemcpyAsync(dk, f.D, cells * sizeof(float), cudaMemcpyDeviceToDevice, p->stream);
    if (e != cudaSuccess) return fail(LPT2_ECUDA, "dk copy: %s", cudaGetErrorString(e));
  }
  return LPT2_OK;
}

}  // namespace

extern "C" {

int lpt2_cic_pk(lpt2_plan_t p, const float* pos, float* density, double* pk, double* k_mean,
                int64_t* n_modes, int n_shells) {
  AbiRange nvtx_range("lpt2_cic_pk");
  int rc = check_plan_ws(p);
  if (rc) return rc;
  if (!pk) return fail(LPT2_EINVAL, "pk must not be null");
  if (n_shells < 1 || n_shells > kMaxShells) return fail(LPT2_EINVAL, "n_shells must be in [1, 256]");
  auto body = [&]() -> int {
    for (int gi = 0; gi < (int)p->groups.size(); ++gi) {
      const Group& gr = p->groups[gi];
      const size_t n3 = (size_t)gr.n * gr.n * gr.n;
      for (int c0 = 0; c0 < gr.count; c0 += chunk_of(gr)) {
        set_chunk(p, gi, c0, std::min(chunk_of(gr), gr.count - c0));
        const size_t off = gr.off + (size_t)c0 * n3;
        const size_t i0 = (size_t)gr.inst0 + c0;
        const int r = cic_pk_group(p, gi, pos ? pos + 3 * off : nullptr, density ? density + off : nullptr,
                                   pk + i0 * n_shells, k_mean ? k_mean + i0 * n_shells : nullptr,
                                   n_modes ? n_modes + i0 * n_shells : nullptr, n_shells);
        if (r) return r;
      }
    }
    set_group(p, 0);
    return LPT2_OK;
  };
  for (int gi = 0; gi < (int)p->groups.size(); ++gi) {
    rc = ensure_geometry(p, gi, n_shells);
    if (rc) return rc;
  }
  if (pos) drop_state(p);   // a new deposit replaces the kept density
  const void* key[8] = {pos, density, pk, k_mean, n_modes, p->ws, (const void*)(intptr_t)n_shells, nullptr};
  const int r = p->use_graph ? run_graph(p, 1, key, body) : body();
  if (!r && !pos && p->kept_fwd) p->kept_spec = true;   // slot A now holds the density spectrum
  return r;
}

// The forward step from and to host memory, pipelined over realisations (see the header).
int lpt2_displace_host(lpt2_plan_t p, int n_real, const float* noise_h, int64_t noise_stride, float* pos_h,
                       int64_t pos_stride, double* pk_h, int64_t pk_stride, int n_shells) {
  if (p) drop_state(p);   // overwrites the state kept for the adjoint
  AbiRange nvtx_range("lpt2_displace_host");
  int rc = check_plan_ws(p);
  if (rc) return rc;
  if (p->n_inst != 1) return fail(LPT2_EUNSUPPORTED, "lpt2_displace_host needs a single-instance plan");
  if (n_real < 1) return fail(LPT2_EINVAL, "n_real must be >= 1");
  if (!pos_h && !pk_h) return fail(LPT2_EINVAL, "pos_h and pk_h are both null: nothing to return");
  if (n_shells < 1 || n_shells > kMaxShells) return fail(LPT2_EINVAL, "n_shells must be in [1, 256]");
  set_group(p, 0);
  const int64_t n3 = (int64_t)p->n * p->n * p->n;
  if ((noise_stride != 0 && noise_stride < n3) || (pos_stride != 0 && pos_stride < 3 * n3) ||
      (pk_stride != 0 && pk_stride < n_shells))
    return fail(LPT2_EINVAL, "a stride must be 0 (one shared buffer) or at least one realisation's size");
  if (!p->host_io || !p->hio)
    return fail(LPT2_EINVAL, "lpt2_displace_host needs a plan made with the LPT2_HOST_IO flag (the workspace "
                             "then holds its two device buffer sets)");
  host_io_buffers(p);
  rc = ensure_geometry(p, 0, n_shells);
  if (rc) return rc;
  HostIO* h = p->hio;
  cudaStream_t cs = p->stream;
  auto ck = [&](cudaError_t e, const char* what) -> int {
    return e == cudaSuccess ? LPT2_OK : fail(LPT2_ECUDA, "lpt2_displace_host %s: %s", what, cudaGetErrorString(e));
  };
  auto body = [&]() -> int {
    // copies start after the work already queued on the plan's stream; both buffer sets start free
    int r0 = ck(cudaEventRecord(h->start, cs), "event");
    if (!r0) r0 = ck(cudaStreamWaitEvent(h->s_in, h->start, 0), "event");
    if (!r0) r0 = ck(cudaStreamWaitEvent(h->s_out, h->start, 0), "event");
    for (int b = 0; b < 2 && !r0; ++b) {
      r0 = ck(cudaEventRecord(h->down_done[b], h->s_out), "event");
      if (!r0) r0 = ck(cudaEventRecord(h->in_used[b], cs), "event");
    }
    if (r0) return r0;
    const size_t nb = (size_t)n3 * sizeof(float);
    if (noise_h) {
      int r1 = ck(cudaMemcpyAsync(h->noise_d[0], noise_h, nb, cudaMemcpyHostToDevice, h->s_in), "upload");
      if (!r1) r1 = ck(cudaEventRecord(h->up_done[0], h->s_in), "event");
      if (r1) return r1;
    }
    for (int r = 0; r < n_real; ++r) {
      const int b = r & 1;
      int e = LPT2_OK;
      if (noise_h && r + 1 < n_real) {   // prefetch the next realisation's noise into the other set
        e = ck(cudaStreamWaitEvent(h->s_in, h->in_used[1 - b], 0), "event");
        if (!e) e = ck(cudaMemcpyAsync(h->noise_d[1 - b], noise_h + (size_t)(r + 1) * noise_stride, nb,
                                       cudaMemcpyHostToDevice, h->s_in), "upload");
        if (!e) e = ck(cudaEventRecord(h->up_done[1 - b], h->s_in), "event");
      }
      if (!e && noise_h) e = ck(cudaStreamWaitEvent(cs, h->up_done[b], 0), "event");
      if (!e) e = ck(cudaStreamWaitEvent(cs, h->down_done[b], 0), "event");   // set b copied out
      if (e) return e;
      e = displace_impl(p, noise_h ? h->noise_d[b] : nullptr, nullptr, nullptr, h->pos_d[b], nullptr, nullptr);
      if (e) return e;
      e = ck(cudaEventRecord(h->in_used[b], cs), "event");
      if (!e) e = ck(cudaEventRecord(h->pos_ready[b], cs), "event");
      if (e) return e;
      // P(k) of the density that lpt2_displace deposited
      e = cic_pk_group(p, 0, nullptr, nullptr, h->pk_d[b], nullptr, nullptr, n_shells);
      if (e) return e;
      e = ck(cudaEventRecord(h->comp_done[b], cs), "event");
      if (!e && pos_h) {
        e = ck(cudaStreamWaitEvent(h->s_out, h->pos_ready[b], 0), "event");
        if (!e) e = ck(cudaMemcpyAsync(pos_h + (size_t)r * pos_stride, h->pos_d[b], 3 * nb, cudaMemcpyDeviceToHost,
                                       h->s_out), "download");
      }
      if (!e && pk_h) {
        e = ck(cudaStreamWaitEvent(h->s_out, h->comp_done[b], 0), "event");
        if (!e) e = ck(cudaMemcpyAsync(pk_h + (size_t)r * pk_stride, h->pk_d[b], n_shells * sizeof(double),
                                       cudaMemcpyDeviceToHost, h->s_out), "download");
      }
      if (!e) e = ck(cudaEventRecord(h->down_done[b], h->s_out), "event");
      if (e) return e;
    }
    return LPT2_OK;
  };
  const int rb = body();
  // wait for everything queued (also after an error, so no copy is left in flight)
  const cudaError_t e1 = cudaStreamSynchronize(h->s_out);
  const cudaError_t e2 = cudaStreamSynchronize(h->s_in);
  const cudaError_t e3 = cudaStreamSynchronize(cs);
  if (rb) return rb;
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
    return fail(LPT2_ECUDA, "lpt2_displace_host: %s",
                cudaGetErrorString(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3)));
  return LPT2_OK;
}

// Output scale factors of lpt2_displace_outputs: growth and multiplier tables per a_j.
int lpt2_set_outputs(lpt2_plan_t p, int n_a, const double* a_out) {
  AbiRange nvtx_range("lpt2_set_outputs");
  if (!p) return fail(LPT2_EINVAL, "null plan");
  if (p->n_inst != 1) return fail(LPT2_EUNSUPPORTED, "lpt2_set_outputs needs a single-instance plan");
  if (n_a < 1 || n_a > kMaxOutputs || !a_out) return fail(LPT2_EINVAL, "need 1 <= n_a <= %d and an a_out array", kMaxOutputs);
  for (int j = 0; j < n_a; ++j)
    if (!(a_out[j] > p->cosmo.a_init) || !(a_out[j] <= 1.0))
      return fail(LPT2_EINVAL, "a_out[%d] = %g: need a_init < a_out <= 1", j, a_out[j]);
  if (n_a > p->max_out)
    return fail(LPT2_EINVAL, "n_a = %d output times, the plan has room for %d: make it with LPT2_MAX_OUTPUTS(n_a)",
                n_a, p->max_out);
  if (!p->ws) return fail(LPT2_ENOWORKSPACE, "no workspace attached (the output tables live in it)");
  set_group(p, 0);
  free_outputs(p);
  p->out_a.assign(a_out, a_out + n_a);
  p->n_out_a = n_a;
  const int rc = run_output_growth(p);
  if (rc) free_outputs(p);
  return rc;
}

// One realisation at every output scale factor: the a-independent prefix once, then per
// a_j the multipliers, positions, CIC and P(k) (see the header).
int lpt2_displace_outputs(lpt2_plan_t p, const float* noise, float* pos, double* pk, double* k_mean,
                          int64_t* n_modes, int n_shells) {
  if (p) drop_state(p);   // overwrites the state kept for the adjoint
  AbiRange nvtx_range("lpt2_displace_outputs");
  int rc = check_plan_ws(p);
  if (rc) return rc;
  if (p->n_inst != 1) return fail(LPT2_EUNSUPPORTED, "lpt2_displace_outputs needs a single-instance plan");
  if (p->n_out_a < 1) return fail(LPT2_EINVAL, "no output scale factors: call lpt2_set_outputs first");
  if (!pk) return fail(LPT2_EINVAL, "pk must not be null");
  if (n_shells < 1 || n_shells > kMaxShells) return fail(LPT2_EINVAL, "n_shells must be in [1, 256]");
  set_group(p, 0);
  rc = ensure_geometry(p, 0, n_shells);
  if (rc) return rc;
  const FwdSlots f = fwd_slots(p);
  rc = displace_prefix(p, f, noise, false);
  if (rc) return rc;
  const size_t n3 = (size_t)p->n * p->n * p->n;
  for (int j = 0; j < p->n_out_a; ++j) {
    rc = displace_suffix(p, f, false, nullptr, nullptr, pos ? pos + j * 3 * n3 : nullptr, nullptr,
                         out_mt0(p, j), out_mt1(p, j), out_tabf(p, j));
    if (rc) return rc;
    // the density spectrum goes to a slot the suffix does not use (A and D stay intact)
    rc = cic_pk_group(p, 0, nullptr, nullptr, pk + (size_t)j * n_shells, j == 0 ? k_mean : nullptr,
                      j == 0 ? n_modes : nullptr, n_shells, f.Y[3]);
    if (rc) return rc;
  }
  return LPT2_OK;
}

// ------------------------------------------------------------ launch schedule
int lpt2_schedule(lpt2_plan_t p, int* chunk, int max_groups, int* n_groups) {
  if (!p || !n_groups) return fail(LPT2_EINVAL, "null argument");
  *n_groups = (int)p->groups.size();
  for (int gi = 0; gi < (int)p->groups.size() && gi < max_groups && chunk; ++gi) chunk[gi] = chunk_of(p->groups[gi]);
  return LPT2_OK;
}

namespace {
void drop_graphs(lpt2_plan_t p) {
  for (auto& gc : p->graphs) {
    if (gc.exec) cudaGraphExecDestroy(gc.exec);
    gc.exec = nullptr;
  }
}
}  // namespace

int lpt2_set_schedule(lpt2_plan_t p, const int* chunk, int n_groups) {
  if (!p || !chunk) return fail(LPT2_EINVAL, "null argument");
  if (n_groups != (int)p->groups.size())
    return fail(LPT2_EINVAL, "n_groups = %d, the plan has %d grid-size groups", n_groups, (int)p->groups.size());
  for (int gi = 0; gi < n_groups; ++gi)
    if (chunk[gi] < 1) return fail(LPT2_EINVAL, "chunk[%d] = %d: need >= 1", gi, chunk[gi]);
  for (int gi = 0; gi < n_groups; ++gi) p->groups[gi].chunk = std::min(chunk[gi], p->groups[gi].count);
  drop_graphs(p);
  return LPT2_OK;
}

namespace {
// y-pass pencils per CTA a group of grid size n can take: the build default (0), or 8 and
// 16 where they tile the n/2 kz of the half spectrum (n >= 32; at n = 16 only the default 8)
bool valid_ytile(int n, int v) { return v == 0 || v == 8 || (v == 16 && n >= 32); }
}  // namespace

int lpt2_tiles(lpt2_plan_t p, int* ytile, int* xtile, int max_groups, int* n_groups) {
  if (!p || !n_groups) return fail(LPT2_EINVAL, "null argument");
  *n_groups = (int)p->groups.size();
  for (int gi = 0; gi < (int)p->groups.size() && gi < max_groups; ++gi) {
    if (ytile) ytile[gi] = p->groups[gi].ytile;
    if (xtile) xtile[gi] = p->groups[gi].xtile;
  }
  return LPT2_OK;
}

int lpt2_set_tiles(lpt2_plan_t p, const int* ytile, const int* xtile, int n_groups) {
  if (!p || !ytile || !xtile) return fail(LPT2_EINVAL, "null argument");
  if (n_groups != (int)p->groups.size())
    return fail(LPT2_EINVAL, "n_groups = %d, the plan has %d grid-size groups", n_groups, (int)p->groups.size());
  for (int gi = 0; gi < n_groups; ++gi) {
    if (!valid_ytile(p->groups[gi].n, ytile[gi]))
      return fail(LPT2_EINVAL, "ytile[%d] = %d: need 0, 8 or 16 (16 needs N >= 32)", gi, ytile[gi]);
    if (xtile[gi] < 0 || xtile[gi] > 2) return fail(LPT2_EINVAL, "xtile[%d] = %d: need 0, 1 or 2", gi, xtile[gi]);
  }
  for (int gi = 0; gi < n_groups; ++gi) {
    p->groups[gi].ytile = ytile[gi];
    p->groups[gi].xtile = xtile[gi];
  }
  drop_graphs(p);
  return LPT2_OK;
}

// Times every group's forward step (Philox noise, positions, CIC, P(k)) at chunk sizes
// count, ceil(count/2), ceil(count/4), ..., 1 and keeps the fastest per group; then, at
// that chunk size, the y-pass pencils per CTA (8, 16) and the x-pass tile path of the
// delta and adjoint modes (bulk-tensor, global loads), one after the other.
int lpt2_autotune(lpt2_plan_t p, int n_shells, int reps) {
  if (p) drop_state(p);   // overwrites the state kept for the adjoint
  AbiRange nvtx_range("lpt2_autotune");
  int rc = check_plan_ws(p);
  if (rc) return rc;
  if (n_shells < 1 || n_shells > kMaxShells) return fail(LPT2_EINVAL, "n_shells must be in [1, 256]");
  if (reps < 1 || reps > 100) return fail(LPT2_EINVAL, "reps must be in [1, 100]");
  double* pk = reinterpret_cast<double*>(p->ws + ws_layout(p).inst_pk);   // [n_inst][n_shells]
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  auto cleanup = [&]() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    set_group(p, 0);
  };
  if (e != cudaSuccess) {
    cleanup();
    return fail(LPT2_ECUDA, "autotune events: %s", cudaGetErrorString(e));
  }
  for (int gi = 0; gi < (int)p->groups.size() && !rc; ++gi) rc = ensure_geometry(p, gi, n_shells);
  drop_graphs(p);
  for (int gi = 0; gi < (int)p->groups.size() && !rc; ++gi) {
    Group& gr = p->groups[gi];
    auto step = [&]() -> int {
      for (int c0 = 0; c0 < gr.count; c0 += chunk_of(gr)) {
        set_chunk(p, gi, c0, std::min(chunk_of(gr), gr.count - c0));
        int r = displace_impl(p, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
        if (!r) r = cic_pk_group(p, gi, nullptr, nullptr, pk + ((size_t)gr.inst0 + c0) * n_shells, nullptr, nullptr,
                                 n_shells);
        if (r) return r;
      }
      return LPT2_OK;
    };
    auto timed = [&](float& ms) -> int {   // one warm-up, then reps timed steps
      int r = step();
      if (r) return r;
      e = cudaEventRecord(e0, p->stream);
      for (int k = 0; k < reps && !r && e == cudaSuccess; ++k) r = step();
      if (r) return r;
      if (e == cudaSuccess) e = cudaEventRecord(e1, p->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) return fail(LPT2_ECUDA, "autotune timing: %s", cudaGetErrorString(e));
      return LPT2_OK;
    };
    int best = gr.count;
    float best_ms = 0.f;
    for (int c = gr.count, prev = 0; c != prev && !rc; prev = c, c = (c + 1) / 2) {
      gr.chunk = c;
      float ms = 0.f;
      if ((rc = timed(ms))) break;
      if (best_ms == 0.f || ms < best_ms) {
        best_ms = ms;
        best = c;
      }
      if (c == 1) break;
    }
    gr.chunk = best;
    for (int yt : {8, 16}) {   // y-pass pencils per CTA
      if (rc || !valid_ytile(gr.n, yt)) continue;
      const int keep = gr.ytile;
      gr.ytile = yt;
      float ms = 0.f;
      if ((rc = timed(ms))) break;
      if (ms < best_ms) best_ms = ms;
      else gr.ytile = keep;
    }
    for (int xt : {1, 2}) {    // x-pass tile path of the delta and adjoint modes
      if (rc) break;
      const int keep = gr.xtile;
      gr.xtile = xt;
      float ms = 0.f;
      if ((rc = timed(ms))) break;
      if (ms < best_ms) best_ms = ms;
      else gr.xtile = keep;
    }
  }
  cleanup();
  return rc;
}

// P(k) estimator refinements: CIC window deconvolution and interlacing (see the header).
int lpt2_cic_pk_est(lpt2_plan_t p, const float* pos, float* density, double* pk, double* k_mean, int64_t* n_modes,
                    int n_shells, unsigned flags) {
  if (p) drop_state(p);   // overwrites the state kept for the adjoint
  AbiRange nvtx_range("lpt2_cic_pk_est");
  int rc = check_plan_ws(p);
  if (rc) return rc;
  if (!pk) return fail(LPT2_EINVAL, "pk must not be null");
  if (n_shells < 1 || n_shells > kMaxShells) return fail(LPT2_EINVAL, "n_shells must be in [1, 256]");
  if (flags & ~(unsigned)(LPT2_PK_DECONVOLVE | LPT2_PK_INTERLACE)) return fail(LPT2_EINVAL, "unknown flags");
  const bool inter = flags & LPT2_PK_INTERLACE;
  if (inter && !pos) return fail(LPT2_EINVAL, "interlacing needs the positions (pos must not be null)");
  for (int gi = 0; gi < (int)p->groups.size(); ++gi) {
    rc = ensure_geometry(p, gi, n_shells);
    if (rc) return rc;
  }
  for (int gi = 0; gi < (int)p->groups.size(); ++gi) {
    set_group(p, gi);
    const Group& gr = p->groups[gi];
    const int n = p->n;
    const Geo g = make_geo(p);
    const size_t cells = (size_t)n * n * n * p->cur_batch;
    const float* gpos = pos ? pos + 3 * gr.off : nullptr;
    float* rho = rho_group(p);
    float2* A = slot(p, S_A);
    if (gpos) {
      LAUNCH(p, "fill0", 4.0 * V3(p), launch_fill0(rho, cells, p->stream));
      CicArgs c{g, gpos, rho, 0.f};
      LAUNCH(p, "cic", 20.0 * V3(p), launch_cic(c, p->stream));
    }
    if ((rc = forward_zy(p, Z_DENSITY, rho, A))) return rc;
    if (density)
      LAUNCH(p, "contrast", 8.0 * V3(p), launch_contrast(rho, density + gr.off, cells, p->stream));
    float2* B = slot(p, S_Y0);
    if (inter) {   // second grid: the particles shifted by +h/2 along every axis
      float* rho2 = reinterpret_cast<float*>(slot(p, S_X0));
      LAUNCH(p, "fill0", 4.0 * V3(p), launch_fill0(rho2, cells, p->stream));
      CicArgs c{g, gpos, rho2, 0.5f};
      LAUNCH(p, "cic", 20.0 * V3(p), launch_cic(c, p->stream));
      if ((rc = forward_zy(p, Z_DENSITY, rho2, B))) return rc;
    }
    XArgs x{};
    x.g = g;
    x.tw = p->tw;
    x.mode = inter ? X_PKI : X_PKP;
    x.in = A;
    x.in2[0] = B;
    x.cosmo = p->cosmo_dev;
    x.pk_part = pk_part(p);
    x.n_shells = n_shells;
    x.pk_deconv = (flags & LPT2_PK_DECONVOLVE) ? 1 : 0;
    LAUNCH(p, "x_pk", (inter ? 8.0 : 4.0) * V3(p), x_pass(n, x, p->stream));
    LAUNCH(p, "pk_finalize", 0.0,
           launch_pk_finalize_p(pk_part(p), x_blocks(n), n_shells, gr.geo_k, gr.geo_n, pk + (size_t)gr.inst0 * n_shells,
                                k_mean ? k_mean + (size_t)gr.inst0 * n_shells : nullptr,
                                n_modes ? n_modes + (size_t)gr.inst0 * n_shells : nullptr, p->stream, p->cur_batch));
    ++p->launches;   // two kernels: row-slice sums, then the shells
  }
  return LPT2_OK;
}

// ------------------------------------------------------------ full-source diagnostic
int lpt2_source_ratio(lpt2_plan_t p, const float* noise, int n_bins, double* mean, double* sigma, int64_t* count,
                      double* t1, double* k_mean, void* s_mg, void* s_gr) {
  if (p) drop_state(p);   // overwrites the state kept for the adjoint
  AbiRange nvtx_range("lpt2_source_ratio");
  int rc = check_plan_ws(p);
  if (rc) return rc;
  if (p->n_inst != 1) return fail(LPT2_EUNSUPPORTED, "lpt2_source_ratio needs a single-instance plan");
  if (n_bins < 1 || n_bins > kMaxShells) return fail(LPT2_EINVAL, "n_bins must be in [1, 256]");
  if (!mean || !sigma || !count) return fail(LPT2_EINVAL, "mean, sigma and count must not be null");
  if ((s_mg == nullptr) != (s_gr == nullptr)) return fail(LPT2_EINVAL, "give both s_mg and s_gr or neither");
  if ((s_mg && !aligned(s_mg, 16)) || (s_gr && !aligned(s_gr, 16))) return fail(LPT2_EINVAL, "misaligned spectra");
  set_group(p, 0);
  const int n = p->n;
  const Geo g = make_geo(p);
  const size_t cells = (size_t)n * n * n;
  rc = ensure_geometry(p, 0, n_bins);
  if (rc) return rc;

  // background at a (FP64 on the host): 4 pi G rho, m^2, M2 (Sec. 2.4, n = 1)
  const double a = p->a_out, H0c = 1.0 / 2997.92458;
  const double om = p->cosmo.omega_m, ol = p->cosmo.omega_l, fr0 = p->cosmo.fr0_abs;
  const double fpg = 1.5 * om / (a * a * a) * H0c * H0c;
  const double xa = om / (a * a * a) + 4.0 * ol, x0 = om + 4.0 * ol;
  const double m2a = fr0 > 0 ? 0.5 * H0c * H0c * xa * xa * xa / (fr0 * x0 * x0) : 0.0;
  const double M2a = fr0 > 0 ? 2.25 * H0c * H0c * pow(xa, 5) / (fr0 * fr0 * pow(x0, 4)) : 0.0;

  // D1_GR(a) / D1_GR(1): the growth integration with |fR0| = 0 on two dummy k nodes
  GrowthParams gp = growth_params(p);
  gp.fr0_abs = 0.0;
  gp.fr0s = nullptr;
  gp.n_inst = 1;
  gp.nk = 2;
  gp.k_min = 1e-3;
  gp.k_max = 2e-3;
  LAUNCH(p, "growth_gr", 0.0, launch_growth(gp, p->gr_tab, p->gr_tabf, p->stream));
  double d1gr_h = 0.0;
  cudaError_t ce = cudaMemcpyAsync(&d1gr_h, p->gr_tab, sizeof(double), cudaMemcpyDeviceToHost, p->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(p->stream);
  if (ce != cudaSuccess) return fail(LPT2_ECUDA, "GR growth: %s", cudaGetErrorString(ce));

  // slots: 0 temporary spectrum, 1 delta0(k), 2-5 real temporaries, 6-11 accumulators,
  // 12 psi / s3, 13-17 spectra of s1, s2, s3, s4, s_GR
  float2* T = slot(p, S_A);
  float2* D = slot(p, S_DELTA);
  auto real = [&](int i) { return reinterpret_cast<float*>(slot(p, i)); };
  float *P = real(2), *Q = real(3), *R = real(4), *P0 = real(5);
  SrcAccum acc{real(6), real(7), real(8), real(9), real(10), real(11)};
  float* PS = real(12);
  float2* F[5] = {slot(p, 13), slot(p, 14), slot(p, 15), slot(p, 16), slot(p, 17)};
  for (int i = 6; i <= 11; ++i) {
    ce = cudaMemsetAsync(real(i), 0, cells * sizeof(float), p->stream);
    if (ce != cudaSuccess) return fail(LPT2_ECUDA, "clear: %s", cudaGetErrorString(ce));
  }

  // delta0(k) (the x pass of the forward path writes it; its potential outputs are scratch)
  rc = forward_zy(p, noise ? Z_REAL : Z_NOISE, noise, T);
  if (rc) return rc;
  {
    XArgs x{};
    x.g = g;
    x.tw = p->tw;
    x.mode = X_DELTA;
    x.in = T;
    x.scf = scf_group(p);
    x.delta_out = D;
    for (int i = 0; i < 3; ++i) x.out[i] = F[i];
    x.cosmo = p->cosmo_dev;
    x.mt0 = p->mt0;
    x.mt1 = p->mt1;
    x.d1f = p->tabf;
    x.d2f = p->tabf + p->nk;
    x.t1f = p->tabf + 2 * p->nk;
    x.t2f = p->tabf + 3 * p->nk;
    LAUNCH(p, "x_delta", 22.0 * V3(p), x_pass(n, x, p->stream));   // + the sqrt(P) field
  }
  // one real field: IDFT[(i k)^ord g(|k|) delta0(k)]
  auto field = [&](int gk, int ox, int oy, int oz, float* out) -> int {
    XArgs x{};
    x.g = g;
    x.tw = p->tw;
    x.mode = X_MUL;
    x.in = D;
    x.out[0] = T;
    x.mt0 = p->mt0;
    x.mul_g = gk;
    x.mul_ord[0] = ox;
    x.mul_ord[1] = oy;
    x.mul_ord[2] = oz;
    x.mul_m2a = (float)m2a;
    x.mul_inv_a2 = (float)(1.0 / (a * a));
    x.mul_d1gr = (float)d1gr_h;
    LAUNCH(p, "x_mul", 8.0 * V3(p), x_pass(n, x, p->stream));
    YArgs y{};
    y.g = g;
    y.tw = p->tw;
    y.inverse = 1;
    y.job.n_in = 1;
    y.job.n_out = 1;
    y.job.in[0] = T;
    y.job.out[0] = T;
    LAUNCH(p, "y_inv", 8.0 * V3(p), y_pass(n, y, p->stream));
    ZC2RArgs z{g, p->tw, T, out, nullptr};
    LAUNCH(p, "z_c2r", 8.0 * V3(p), z_c2r(n, z, p->stream));
    return LPT2_OK;
  };
  static const int pairs[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
  for (const auto& ij : pairs) {
    int o[3] = {0, 0, 0};
    ++o[ij[0]];
    ++o[ij[1]];
    if ((rc = field(G_POT, o[0], o[1], o[2], P)) || (rc = field(G_MUPOT, o[0], o[1], o[2], Q)) ||
        (rc = field(G_PSI, o[0], o[1], o[2], R)) || (rc = field(G_POT0, o[0], o[1], o[2], P0)))
      return rc;
    const bool diag = ij[0] == ij[1];
    LAUNCH(p, "src_pair", 40.0 * V3(p),
           launch_src_pair(cells, P, Q, R, P0, diag ? 1.f : 2.f, diag ? 1 : 0, acc, p->stream));
  }
  for (int j = 0; j < 3; ++j) {
    int o[3] = {0, 0, 0};
    o[j] = 1;
    if ((rc = field(G_D1, o[0], o[1], o[2], P)) || (rc = field(G_PSI, o[0], o[1], o[2], Q))) return rc;
    LAUNCH(p, "src_grad", 16.0 * V3(p), launch_src_grad(cells, P, Q, acc.s4, p->stream));
  }
  if ((rc = field(G_PSI, 0, 0, 0, PS))) return rc;
  LAUNCH(p, "src_final", 28.0 * V3(p), launch_src_final(cells, acc, PS, p->stream));

  // forward transforms of s1, s2, s3, s4, s_GR
  const float* src[5] = {acc.s1, acc.s2, PS, acc.s4, acc.sg};
  for (int i = 0; i < 5; ++i) {
    if ((rc = forward_zy(p, Z_REAL, src[i], F[i]))) return rc;
    XArgs x{};
    x.g = g;
    x.tw = p->tw;
    x.mode = X_FWD;
    x.in = F[i];
    x.out[0] = F[i];
    LAUNCH(p, "x_fwd", 8.0 * V3(p), x_pass(n, x, p->stream));
  }
  // per-mode ratio, shell mean and scatter
  SrcRatioArgs ra{};
  ra.n = n;
  ra.n_bins = n_bins;
  ra.kf = g.kf;
  ra.fpg = (float)fpg;
  ra.e3 = (float)(2.0 / 3.0 * fpg);
  ra.m2a = (float)m2a;
  ra.inv_a2 = (float)(1.0 / (a * a));
  ra.M2a = (float)M2a;
  ra.fr0 = (float)fr0;
  ra.f1 = F[0];
  ra.f2 = F[1];
  ra.f3 = F[2];
  ra.f4 = F[3];
  ra.fg = F[4];
  ra.smg = reinterpret_cast<float2*>(s_mg);
  ra.sgr = reinterpret_cast<float2*>(s_gr);
  const int nblk = src_ratio_blocks(n);
  double* part0 = pk_part(p);                          // [nblk][2]
  double* part1 = part0 + (size_t)2 * nblk;            // [nblk][3][n_bins]
  ra.part = part0;
  LAUNCH(p, "src_ratio0", 20.0 * V3(p), launch_src_ratio(ra, 0, nullptr, p->stream));
  ra.part = part1;
  LAUNCH(p, "src_ratio1", 20.0 * V3(p), launch_src_ratio(ra, 1, part0, p->stream));
  LAUNCH(p, "src_finalize", 0.0, launch_src_finalize(part1, nblk, n_bins, mean, sigma, count, p->stream));
  if (t1 && !k_mean) return fail(LPT2_EINVAL, "t1 needs k_mean");
  if (k_mean) {
    const Group& gr = p->groups[0];
    LAUNCH(p, "src_t1", 0.0,
           launch_src_t1(n_bins, gr.geo_k, gr.geo_n, k_mean, p->tab, p->nk, p->k_min, p->k_max, p->gr_tab, a, m2a,
                         M2a, fpg, fr0 > 0 ? 0 : 1, t1, p->stream));
  }
  return LPT2_OK;
}

int lpt2_fft_r2c(lpt2_plan_t p, const float* in, void* out) {
  AbiRange nvtx_range("lpt2_fft_r2c");
  int rc = check_plan_ws(p);
  if (rc) return rc;
  if (p->n_inst != 1) return fail(LPT2_EUNSUPPORTED, "lpt2_fft_r2c needs a single-instance plan");
  set_group(p, 0);
  if (!in || !out || !aligned(out, 16)) return fail(LPT2_EINVAL, "bad in/out");
  float2* o = reinterpret_cast<float2*>(out);
  rc = forward_zy(p, Z_REAL, in, o);
  if (rc) return rc;
  XArgs x{};
  x.g = make_geo(p);
  x.tw = p->tw;
  x.mode = X_FWD;
  x.in = o;
  x.out[0] = o;
  LAUNCH(p, "x_fwd", 8.0 * V3(p), x_pass(p->n, x, p->stream));
  return LPT2_OK;
}

int lpt2_fft_c2r(lpt2_plan_t p, const void* in, float* out) {
  if (p) p->kept_spec = false;   // slot A is overwritten
  AbiRange nvtx_range("lpt2_fft_c2r");
  int rc = check_plan_ws(p);
  if (rc) return rc;
  if (p->n_inst != 1) return fail(LPT2_EUNSUPPORTED, "lpt2_fft_c2r needs a single-instance plan");
  set_group(p, 0);
  if (!in || !out || !aligned(in, 16)) return fail(LPT2_EINVAL, "bad in/out");
  const Geo g = make_geo(p);
  float2* A = slot(p, S_A);
  XArgs x{};
  x.g = g;
  x.tw = p->tw;
  x.mode = X_INV;
  x.in = reinterpret_cast<const float2*>(in);
  x.out[0] = A;
  LAUNCH(p, "x_inv", 8.0 * V3(p), x_pass(p->n, x, p->stream));
  YArgs y{};
  y.g = g;
  y.tw = p->tw;
  y.inverse = 1;
  y.job.n_in = 1;
  y.job.n_out = 1;
  y.job.in[0] = A;
  y.job.out[0] = A;
  LAUNCH(p, "y_inv", 8.0 * V3(p), y_pass(p->n, y, p->stream));
  ZC2RArgs z{g, p->tw, A, out, nullptr};
  LAUNCH(p, "z_c2r", 8.0 * V3(p), z_c2r(p->n, z, p->stream));
  return LPT2_OK;
}

int lpt2_set_fr0(lpt2_plan_t p, double fr0_abs) {
  if (p) drop_state(p);   // overwrites the state kept for the adjoint
  if (!p) return fail(LPT2_EINVAL, "null plan");
  if (p->n_inst != 1) return fail(LPT2_EUNSUPPORTED, "lpt2_set_fr0 needs a single-instance plan");
  if (!(fr0_abs >= 0) || !isfinite(fr0_abs)) return fail(LPT2_EINVAL, "fr0_abs must be >= 0");
  p->cosmo.fr0_abs = fr0_abs;
  cudaError_t e = cudaMemcpyAsync(p->fr0_dev, &p->cosmo.fr0_abs, sizeof(double), cudaMemcpyHostToDevice, p->stream);
  if (e != cudaSuccess) return fail(LPT2_ECUDA, "fr0 upload: %s", cudaGetErrorString(e));
  e = cudaStreamSynchronize(p->stream);   // the host value must outlive the copy
  if (e != cudaSuccess) return fail(LPT2_ECUDA, "fr0 upload: %s", cudaGetErrorString(e));
  return run_growth(p);
}

int lpt2_displace_vjp(lpt2_plan_t p, const float* noise, const float* g_pos, const float* g_density,
                      const double* g_pk, int n_shells, float* g_noise, double* g_log_fr0) {
  AbiRange nvtx_range("lpt2_displace_vjp");
  int rc = check_plan_ws(p);
  if (rc) return rc;
  if (p->n_inst != 1) return fail(LPT2_EUNSUPPORTED, "lpt2_displace_vjp needs a single-instance plan");
  set_group(p, 0);
  if (n_shells < 1 || n_shells > kMaxShells) return fail(LPT2_EINVAL, "n_shells must be in [1, 256]");
  const int n = p->n;
  const Geo g = make_geo(p);
  float2* S[N_SLOTS];
  for (int i = 0; i < N_SLOTS; ++i) S[i] = slot(p, i);
  float* pos = reinterpret_cast<float*>(S[S_POS]);            // 3 consecutive slots
  float* rho = rho_group(p);
  float* shw = reinterpret_cast<float*>(p->ws + tail_shw(p));
  double* thp = reinterpret_cast<double*>(p->ws + tail_theta(p));
  const double V3d = (double)n * n * n;

  // The forward map, keeping delta(k) (slot 1), S(k), positions and the CIC density, unless
  // the last lpt2_displace of a LPT2_KEEP_STATE plan left them for this noise; then the
  // delta_rho spectrum after the z and y passes, unless a later lpt2_cic_pk left it in slot A.
  const bool reuse = p->keep_state && p->kept_fwd && p->kept_noise == noise;
  const bool reuse_spec = reuse && p->kept_spec;
  drop_state(p);   // this call overwrites the kept slots
  if (!reuse) {
    rc = displace_impl(p, noise, nullptr, nullptr, nullptr, nullptr, S[S_SHAT], pos);
    if (rc) return rc;
  }
  if (!reuse_spec) {
    rc = forward_zy(p, Z_DENSITY, rho, S[S_A]);
    if (rc) return rc;
  }
  // the P(k) transpose needs the mode count per shell (cached geometry), not P(k) itself
  rc = ensure_geometry(p, 0, n_shells);
  if (rc) return rc;
  static_assert(sizeof(unsigned long long) == sizeof(int64_t), "mode counts are 64-bit");
  const int64_t* nmodes = reinterpret_cast<const int64_t*>(p->groups[0].geo_n);
  XArgs xp{};
  xp.g = g;
  xp.tw = p->tw;
  xp.in = S[S_A];
  xp.cosmo = p->cosmo_dev;
  xp.pk_part = pk_part(p);
  xp.n_shells = n_shells;

  // 1. density cotangent: g_density + IDFT[w_b delta_rho(k)]
  const double v_over_n6 = p->box * p->box * p->box / (V3d * V3d);
  LAUNCH(p, "pk_adj_w", 0.0, launch_pk_adj_weights(g_pk, nmodes, n_shells, v_over_n6, shw, p->stream));
  XArgs xa = xp;
  xa.mode = X_PKADJ;
  xa.shell_w = shw;
  xa.out[0] = S[S_A];
  LAUNCH(p, "x_pkadj", 8.0 * V3(p), x_pass(n, xa, p->stream));
  YArgs yi{};
  yi.g = g;
  yi.tw = p->tw;
  yi.inverse = 1;
  yi.job.n_in = 1;
  yi.job.n_out = 1;
  yi.job.in[0] = S[S_A];
  yi.job.out[0] = S[S_A];
  LAUNCH(p, "y_inv", 8.0 * V3(p), y_pass(n, yi, p->stream));
  float* grho = reinterpret_cast<float*>(S[2]);
  ZC2RArgs zc{g, p->tw, S[S_A], grho, g_density};
  LAUNCH(p, "z_c2r_grho", (g_density ? 12.0 : 8.0) * V3(p), z_c2r(n, zc, p->stream));

  // 2-3. CIC transpose (tiled gather) into real g_Psi fields (slots 10-12), then their
  // forward z transforms: slots 7 (z; its conj(i k_z) is applied in the y pass), 8 (y), 9 (x)
  float* gps[3] = {reinterpret_cast<float*>(S[12]), reinterpret_cast<float*>(S[11]),
                   reinterpret_cast<float*>(S[10])};   // x, y, z
  CicGradArgs cg{g, grho, pos, g_pos, gps[0], gps[1], gps[2]};
  LAUNCH(p, "cic_grad", (g_pos ? 40.0 : 28.0) * V3(p), launch_cic_grad(cg, p->stream));
  ZR2CArgs zp{};
  zp.g = g;
  zp.tw = p->tw;
  zp.src = Z_REAL;
  for (int c = 0; c < 3; ++c) {   // z, y, x
    zp.in = gps[2 - c];
    zp.out = S[7 + c];
    LAUNCH(p, "z_r2c_gpsi", 8.0 * V3(p), z_r2c(n, zp, p->stream));
  }
  // 4. y transpose: x-order 0 group = Psi_z (y0) + Psi_y (y1); x-order 1 = Psi_x
  YArgs ys{};
  ys.g = g;
  ys.tw = p->tw;
  ys.job.sum = 1;
  ys.job.n_in = 3;
  ys.job.n_out = 2;
  ys.job.in[0] = S[7];
  ys.job.in[1] = S[8];
  ys.job.in[2] = S[9];
  ys.job.dst[0] = 0; ys.job.ord[0] = 0; ys.job.zord[0] = 1;
  ys.job.dst[1] = 0; ys.job.ord[1] = 1;
  ys.job.dst[2] = 1; ys.job.ord[2] = 0;
  ys.job.out[0] = S[10];
  ys.job.out[1] = S[11];
  LAUNCH(p, "y_adj_psi", 20.0 * V3(p), y_pass(n, ys, p->stream));
  // 5-6. x transpose of the source step: h_Psi (slot 12), inverse x of h_S (slot 3), theta
  // partials; then h_S to real space (g_S, in the position slot: the positions are dead after
  // the CIC transpose)
  XArgs xs{};
  xs.g = g;
  xs.tw = p->tw;
  xs.mode = X_ADJ_SOURCE;
  xs.in2[0] = S[10];
  xs.in2[1] = S[11];
  xs.delta_in = S[S_DELTA];
  xs.s_in = S[S_SHAT];
  xs.hpsi_out = S[12];
  xs.out[0] = S[3];
  xs.cosmo = p->cosmo_dev;
  xs.mt0 = p->mt0;
  xs.mt1 = p->mt1;
  xs.d1f = p->tabf;
  xs.d2f = p->tabf + p->nk;
  xs.t1f = p->tabf + 2 * p->nk;
  xs.t2f = p->tabf + 3 * p->nk;
  xs.theta_part = thp;
  LAUNCH(p, "x_adj_source", 28.0 * V3(p), x_pass(n, xs, p->stream));
  YArgs yh = yi;
  yh.job.in[0] = S[3];
  yh.job.out[0] = S[3];
  LAUNCH(p, "y_inv", 8.0 * V3(p), y_pass(n, yh, p->stream));
  float* gsr = reinterpret_cast<float*>(S[S_POS]);
  ZC2RArgs zg{g, p->tw, S[3], gsr, nullptr};
  LAUNCH(p, "z_c2r_gs", 8.0 * V3(p), z_c2r(n, zg, p->stream));
  // 7-8. z transpose of the source term: the six phi_ij are the forward's (checkpointed in
  // their slots: the forward above, or the kept one, wrote them and nothing since has);
  // outputs xx yy zz xy xz yz
  ZAdjSourceArgs za{};
  za.g = g;
  za.tw = p->tw;
  za.gs = gsr;
  const FwdSlots fs = fwd_slots(p);
  const float2* phi[6] = {fs.P[5], fs.P[2], fs.P[0], fs.P[4], fs.P[3], fs.P[1]};   // xx yy zz xy xz yz
  const int zord[6] = {0, 0, 2, 0, 1, 1};
  float2* gout[6] = {S[0], S[2], S[4], S[7], S[8], S[9]};
  for (int i = 0; i < 6; ++i) {
    za.in[i] = phi[i];
    za.ord[i] = zord[i];
    za.out[i] = gout[i];
  }
  LAUNCH(p, "z_adj_source", 52.0 * V3(p), z_adj_source(n, za, p->stream));
  // 9. y transpose: x-order 0 <- zz (y0) + yz (y1) + yy (y2); x-order 1 <- xz (y0) + xy (y1); 2 <- xx
  YArgs y6{};
  y6.g = g;
  y6.tw = p->tw;
  y6.job.sum = 1;
  y6.job.n_in = 6;
  y6.job.n_out = 3;
  const int gdst[6] = {2, 0, 0, 1, 1, 0}, gord[6] = {0, 2, 0, 1, 0, 1};   // xx yy zz xy xz yz
  for (int i = 0; i < 6; ++i) {
    y6.job.in[i] = gout[i];
    y6.job.dst[i] = gdst[i];
    y6.job.ord[i] = gord[i];
  }
  y6.job.out[0] = S[15];
  y6.job.out[1] = S[16];
  y6.job.out[2] = S[5];
  LAUNCH(p, "y_adj_phi", 36.0 * V3(p), y_pass(n, y6, p->stream));
  // 10. x transpose of the delta step: s(k) (h_Psi + h_phi) -> inverse x (slot 6)
  XArgs xd{};
  xd.g = g;
  xd.tw = p->tw;
  xd.mode = X_ADJ_DELTA;
  xd.scf = scf_group(p);
  xd.in2[0] = S[15];
  xd.in2[1] = S[16];
  xd.in2[2] = S[5];
  xd.hpsi_in = S[12];
  xd.out[0] = S[6];
  xd.cosmo = p->cosmo_dev;
  xd.mt0 = p->mt0;
  xd.mt1 = p->mt1;
  LAUNCH(p, "x_adj_delta", 22.0 * V3(p), x_pass(n, xd, p->stream));   // + the sqrt(P) field
  YArgs yg = yi;
  yg.job.in[0] = S[6];
  yg.job.out[0] = S[6];
  LAUNCH(p, "y_inv", 8.0 * V3(p), y_pass(n, yg, p->stream));
  if (g_noise) {
    ZC2RArgs zn{g, p->tw, S[6], g_noise, nullptr};
    LAUNCH(p, "z_c2r", 8.0 * V3(p), z_c2r(n, zn, p->stream));
  }
  if (g_log_fr0) LAUNCH(p, "theta_sum", 0.0, launch_sum_partials(thp, x_blocks(n), g_log_fr0, p->stream));
  return LPT2_OK;
}

int lpt2_timing(lpt2_plan_t p, int enable) {
  if (!p) return fail(LPT2_EINVAL, "null plan");
  if (enable && !p->ev) {
    p->ev = new cudaEvent_t[2 * kMaxRec];
    for (int i = 0; i < 2 * kMaxRec; ++i) {
      cudaError_t e = cudaEventCreate(&p->ev[i]);
      if (e != cudaSuccess) return fail(LPT2_ECUDA, "event create: %s", cudaGetErrorString(e));
    }
  }
  p->timing_on = enable != 0;
  if (enable) p->n_rec = 0;
  return LPT2_OK;
}

int lpt2_timing_report(lpt2_plan_t p, lpt2_kernel_stat* out, int max, int* n_out) {
  if (!p || !n_out || (max > 0 && !out)) return fail(LPT2_EINVAL, "null argument");
  *n_out = 0;
  if (p->n_rec == 0) return LPT2_OK;
  cudaError_t e = cudaEventSynchronize(p->ev[2 * p->n_rec - 1]);
  if (e != cudaSuccess) return fail(LPT2_ECUDA, "event sync: %s", cudaGetErrorString(e));
  int n = 0;
  for (int r = 0; r < p->n_rec; ++r) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, p->ev[2 * r], p->ev[2 * r + 1]);
    if (e != cudaSuccess) return fail(LPT2_ECUDA, "event time: %s", cudaGetErrorString(e));
    int j = 0;
    while (j < n && strcmp(out[j].name, p->rec_name[r]) != 0) ++j;
    if (j == n) {
      if (n >= max) continue;
      memset(&out[n], 0, sizeof(out[n]));
      strncpy(out[n].name, p->rec_name[r], sizeof(out[n].name) - 1);
      ++n;
    }
    out[j].launches += 1;
    out[j].total_ms += ms;
    out[j].bytes += p->rec_bytes[r];
  }
  *n_out = n;
  return LPT2_OK;
}

}  // extern "C"
