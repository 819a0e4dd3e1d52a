// lpt2_cic_pk_noalloc: CIC density and shell P(k) for callers that cannot
// allocate device memory.  All scratch lives in one file-scope __device__ array
// of fixed size (grids up to kNoAllocMaxN per side); the caller passes only
// inputs and outputs.  The array is part of the library image, so every GPU
// that loads the library holds it until the process exits.
#include <cuda.h>   // CUcontext / CUresult types only; the driver calls are resolved at run time
#include <math.h>

#include <mutex>
#include <string>

#include "../../include/lpt2.h"
#include "passes.cuh"

using namespace lpt2;

namespace {

constexpr int kNoAllocMaxN = 128;
constexpr int kMaxShells = 256;
constexpr size_t kGrid = (size_t)kNoAllocMaxN * kNoAllocMaxN * kNoAllocMaxN;
// x-pass blocks of a grid: (N/2 kz / W kz per block) * N, with W the pencils per CTA of this
// build (a tuning macro); the partial-sum region is sized for the largest of the four grids
template <int N> constexpr size_t xblocks_of() { return (size_t)(PassCfg<N>::H / PassCfg<N>::W) * N; }
constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kMaxXBlocks =
    cmax(cmax(xblocks_of<16>(), xblocks_of<32>()), cmax(xblocks_of<64>(), xblocks_of<128>()));
constexpr size_t kRhoOff = 0;                                        // float[N^3]
constexpr size_t kSpecOff = kRhoOff + kGrid * sizeof(float);         // float2[N^3/2]
constexpr size_t kPartOff = kSpecOff + kGrid * sizeof(float);        // double[blocks][3][256]
constexpr size_t kTwOff = kPartOff + kMaxXBlocks * 3 * kMaxShells * sizeof(double);
constexpr size_t kCosmoOff = kTwOff + kNoAllocMaxN * sizeof(float2);
constexpr size_t kScratchBytes = kCosmoOff + 256;
static_assert(kSpecOff % 256 == 0 && kPartOff % 256 == 0 && kTwOff % 256 == 0 && kCosmoOff % 256 == 0,
              "scratch sub-arrays must stay 256-byte aligned");

}  // namespace

// The scratch array (about 20 MB).  Host code must not take its address
// directly: the symbol's device address is fetched with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_lpt2_noalloc_scratch[kScratchBytes];

namespace {

// Device address of the scratch per device ordinal, valid for the context it was looked up
// in: after cudaDeviceReset (or a release of the primary context) the library image is loaded
// again into a new context and the address must be looked up again, so each entry records
// the unique id of its context.
struct ScratchAddr {
  unsigned long long ctx_id = 0;
  void* ptr = nullptr;
};
std::mutex g_mu;
ScratchAddr g_addr[128];

typedef CUresult (*PfnCtxGetCurrent)(CUcontext*);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long*);

// Unique id of the calling thread's current context (0 if none is current yet).
int current_ctx_id(unsigned long long* id) {
  static PfnCtxGetCurrent get_current = nullptr;
  static PfnCtxGetId get_id = nullptr;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return -1;
    get_current = (PfnCtxGetCurrent)f1;
    get_id = (PfnCtxGetId)f2;
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS) return -1;
  *id = 0;
  if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return -1;
  return 0;
}

int fail(int code, const std::string& msg) {
  set_last_error(msg);   // reported by lpt2_last_error()
  return code;
}

// Twiddles exp(-2 pi i m / n) in FP64, rounded once to FP32.
__global__ void k_noalloc_twiddles(float2* tw, int n) {
  for (int m = threadIdx.x; m < n; m += blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)m / (double)n, &s, &c);
    tw[m] = make_float2((float)c, (float)(-s));
  }
}

cudaError_t z_r2c_n(int n, const ZR2CArgs& a, cudaStream_t s) {
  switch (n) {
    case 16: return launch_z_r2c_16(a, s);
    case 32: return launch_z_r2c_32(a, s);
    case 64: return launch_z_r2c_64(a, s);
    default: return launch_z_r2c_128(a, s);
  }
}
cudaError_t y_n(int n, const YArgs& a, cudaStream_t s) {
  switch (n) {
    case 16: return launch_y_16(a, s);
    case 32: return launch_y_32(a, s);
    case 64: return launch_y_64(a, s);
    default: return launch_y_128(a, s);
  }
}
cudaError_t x_n(int n, const XArgs& a, cudaStream_t s) {
  switch (n) {
    case 16: return launch_x_16(a, s);
    case 32: return launch_x_32(a, s);
    case 64: return launch_x_64(a, s);
    default: return launch_x_128(a, s);
  }
}
int xblocks_n(int n) {
  switch (n) {
    case 16: return x_blocks_16();
    case 32: return x_blocks_32();
    case 64: return x_blocks_64();
    default: return x_blocks_128();
  }
}

}  // namespace

extern "C" int lpt2_cic_pk_noalloc(int n, double box, const float* pos, float* density, double* pk,
                                   double* k_mean, int64_t* n_modes, int n_shells, void* cuda_stream) {
  if (!(n == 16 || n == 32 || n == 64 || n == 128))
    return fail(LPT2_EUNSUPPORTED, "lpt2_cic_pk_noalloc: grid side must be 16, 32, 64 or 128 "
                                   "(static scratch holds at most 128^3)");
  if (!(box > 0) || !isfinite(box)) return fail(LPT2_EINVAL, "lpt2_cic_pk_noalloc: box must be > 0");
  if (!pos || !pk) return fail(LPT2_EINVAL, "lpt2_cic_pk_noalloc: pos and pk must not be null");
  if (n_shells < 1 || n_shells > kMaxShells)
    return fail(LPT2_EINVAL, "lpt2_cic_pk_noalloc: n_shells must be in [1, 256]");
  if ((uintptr_t)pos % 4 || (density && (uintptr_t)density % 4))
    return fail(LPT2_EINVAL, "lpt2_cic_pk_noalloc: misaligned pointer");
  cudaStream_t s = (cudaStream_t)cuda_stream;

  // the shell partial sums of the P(k) pass must fit their region of the scratch
  if ((size_t)xblocks_n(n) * 3 * n_shells > kMaxXBlocks * 3 * kMaxShells)
    return fail(LPT2_EUNSUPPORTED, "lpt2_cic_pk_noalloc: shell partial sums exceed the static scratch");

  // Set-up once per device (and again if the device's context was re-created): the
  // scratch symbol's device address, looked up with that device current.
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(LPT2_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 128) return fail(LPT2_EUNSUPPORTED, "device ordinal >= 128");
  char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    unsigned long long ctx = 0;
    if (current_ctx_id(&ctx)) return fail(LPT2_ECUDA, "lpt2_cic_pk_noalloc: cannot read the current context");
    if (!g_addr[dev].ptr || ctx == 0 || ctx != g_addr[dev].ctx_id) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_lpt2_noalloc_scratch);   // makes the device's context current
      if (e != cudaSuccess)
        return fail(LPT2_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      if (current_ctx_id(&ctx) || ctx == 0)
        return fail(LPT2_ECUDA, "lpt2_cic_pk_noalloc: no current context after the set-up");
      g_addr[dev].ptr = p;
      g_addr[dev].ctx_id = ctx;
    }
    base = (char*)g_addr[dev].ptr;
  }
  float* rho = reinterpret_cast<float*>(base + kRhoOff);
  float2* spec = reinterpret_cast<float2*>(base + kSpecOff);
  double* part = reinterpret_cast<double*>(base + kPartOff);
  float2* tw = reinterpret_cast<float2*>(base + kTwOff);
  const DevCosmo* cosmo = reinterpret_cast<const DevCosmo*>(base + kCosmoOff);

  Geo g{};
  const double nd = n;
  g.n = n;
  g.kf = (float)(2.0 * M_PI / box);
  g.box = (float)box;
  g.cell = (float)(box / nd);
  g.inv_cell = (float)(nd / box);
  g.inv_n3 = (float)(1.0 / (nd * nd * nd));
  g.sqrt_n3_over_v = (float)sqrt(nd * nd * nd / (box * box * box));
  g.batch = 1;        // one grid per call
  g.inst0 = 0;
  g.tab_stride = 0;
  g.wait = LPT2_WAIT_CYCLES;   // none of these passes waits on a barrier
  const size_t n3 = (size_t)n * n * n;

#define NA_CHECK(expr)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess) return fail(LPT2_ECUDA, std::string(#expr ": ") + cudaGetErrorString(e_)); \
  } while (0)

  k_noalloc_twiddles<<<1, 128, 0, s>>>(tw, n);
  NA_CHECK(cudaGetLastError());
  NA_CHECK(launch_fill0(rho, n3, s));               // the deposit accumulates: start from zero
  CicArgs c{g, pos, rho};
  NA_CHECK(launch_cic(c, s));
  ZR2CArgs z{};
  z.g = g;
  z.tw = tw;
  z.src = Z_DENSITY;
  z.in = rho;
  z.out = spec;
  NA_CHECK(z_r2c_n(n, z, s));
  YArgs y{};
  y.g = g;
  y.tw = tw;
  y.inverse = 0;
  y.job.n_in = 1;
  y.job.n_out = 1;
  y.job.in[0] = spec;
  y.job.out[0] = spec;
  NA_CHECK(y_n(n, y, s));
  XArgs x{};
  x.g = g;
  x.tw = tw;
  x.mode = X_PK;
  x.in = spec;
  x.cosmo = cosmo;
  x.pk_part = part;
  x.n_shells = n_shells;
  NA_CHECK(x_n(n, x, s));
  NA_CHECK(launch_pk_finalize(part, xblocks_n(n), n_shells, pk, k_mean, n_modes, s));
  if (density) NA_CHECK(launch_contrast(rho, density, n3, s));
#undef NA_CHECK
  return LPT2_OK;
}
