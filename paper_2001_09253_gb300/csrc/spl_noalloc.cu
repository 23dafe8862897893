// spl_fit_eval_noalloc: the mixed-precision fit (one refinement step) and evaluation of one
// instance for callers that cannot allocate device memory.  Everything the two kernels need
// beyond the caller's inputs and outputs lives in one fixed array compiled into this file.
#include <mutex>

#include "../../include/spl.h"
#include "spl_internal.h"

namespace {

constexpr unsigned long long kMaxN = SPL_NOALLOC_MAX_N;
constexpr size_t kInstOff = 0;      // the instance descriptor
constexpr size_t kStatusOff = 256;  // its status word and two tile counters (cleared by every call)
constexpr size_t kZOff = 512;       // binary32 y'' of the first pass, kMaxN floats
constexpr size_t kScratchBytes = kZOff + 4 * kMaxN;
static_assert(sizeof(spl::Inst) <= kStatusOff, "the descriptor fits below the status words");

// The scratch.  Every GPU that loads this library holds these 4 MiB + 512 B until the
// process exits.  Host code must not use this name as an address: it is a host-side stand-in;
// the device address comes from cudaGetSymbolAddress (see setup_device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// The array's device address, looked up once per CUDA context.  A context is recognised by its
// process-unique ID (cuCtxGetId), not by the device ordinal: a device reset destroys the primary
// context and the module with it, so the context that replaces it (whatever its handle) gets its
// own look-up instead of a stale address.  The driver calls are fetched through the runtime, so
// the library needs no link-time dependency on the driver library.
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);

constexpr int kMaxContexts = 64;
struct AddrEntry {
  unsigned long long ctx_id;
  unsigned char *addr;
  int sms;
};
std::mutex g_mu;
AddrEntry g_cache[kMaxContexts];
int g_cached = 0;
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

spl_status driver_fns() {
  if (g_ctx_current && g_ctx_id) return SPL_OK;
  void *f1 = nullptr, *f2 = nullptr;
  cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
      q1 != cudaDriverEntryPointSuccess || !f1)
    return SPL_ERR_CUDA;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
      q2 != cudaDriverEntryPointSuccess || !f2)
    return SPL_ERR_CUDA;
  g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f1);
  g_ctx_id = reinterpret_cast<CtxGetIdFn>(f2);
  return SPL_OK;
}

// With the caller's device current: the array's device address in the current context (looked
// up with cudaGetSymbolAddress on the first call in each context) and the device's SM count.
spl_status setup_device(int dev, unsigned char **addr, int *sms) {
  std::lock_guard<std::mutex> lk(g_mu);
  spl_status s = driver_fns();
  if (s != SPL_OK) return s;
  void *ctx = nullptr;
  if (g_ctx_current(&ctx) != 0) return SPL_ERR_CUDA;
  if (!ctx) {  // no context bound to this thread yet: cudaSetDevice binds the device's primary one
    if (cudaSetDevice(dev) != cudaSuccess || g_ctx_current(&ctx) != 0 || !ctx) return SPL_ERR_CUDA;
  }
  unsigned long long id = 0;
  if (g_ctx_id(ctx, &id) != 0) return SPL_ERR_CUDA;
  for (int i = 0; i < g_cached; ++i) {
    if (g_cache[i].ctx_id == id) {
      *addr = g_cache[i].addr;
      *sms = g_cache[i].sms;
      return SPL_OK;
    }
  }
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SPL_ERR_CUDA;
  int n_sm = 0;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SPL_ERR_CUDA;
  // a full table keeps serving by looking the address up again on each call
  if (g_cached < kMaxContexts) g_cache[g_cached++] = AddrEntry{id, static_cast<unsigned char *>(p), n_sm};
  *addr = static_cast<unsigned char *>(p);
  *sms = n_sm;
  return SPL_OK;
}

// Writes the descriptor into the scratch and clears the status word and the tile counters,
// so that no host buffer has to be copied.
__global__ void noalloc_prepare(spl::Inst I, spl::Inst *dst, unsigned *status, unsigned long long *counters) {
  *dst = I;
  *status = 0u;
  counters[0] = 0ull;
  counters[1] = 0ull;
}

bool slope_valid(double s) { return !(s != s) && !(s < -1.7976931348623157e308); }

}  // namespace

extern "C" spl_status spl_fit_eval_noalloc(const double *x, const double *y, uint64_t n, double yp1, double ypn,
                                           uint64_t m, double *ypp_out, double *yq_out, void *stream,
                                           int32_t *status_out) {
  if (status_out) *status_out = SPL_PENDING;
  if (n < 3 || !x || !y || (m > 0 && !yq_out) || m > (1ull << 40)) return SPL_ERR_INVALID_ARG;
  if (!slope_valid(yp1) || !slope_valid(ypn)) return SPL_ERR_INVALID_ARG;
  if (n > kMaxN) return SPL_ERR_BUDGET;  // beyond the fixed scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPL_ERR_CUDA;
  unsigned char *base = nullptr;
  int sms = 0;
  spl_status s = setup_device(dev, &base, &sms);
  if (s != SPL_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  spl::Inst I{};
  I.x = x; I.y = y; I.ypp = ypp_out; I.yq = yq_out; I.jq = nullptr;
  I.n = (long long)n; I.m = (long long)m;
  I.yp1 = yp1; I.ypn = ypn;
  // the warp-cooperative kernel and the runtime's tile rule for one binary32 instance
  const long long L = spl::scan_mixed_tile_rows((long long)n, sms, 1);
  I.tile_rows = (int)L;
  I.ntiles = ((long long)n + L - 1) / L;
  I.tile_begin = 0;
  I.status = reinterpret_cast<unsigned *>(base + kStatusOff);
  I.z = reinterpret_cast<float *>(base + kZOff);
  spl::Inst *d_inst = reinterpret_cast<spl::Inst *>(base + kInstOff);

  unsigned long long *counters = reinterpret_cast<unsigned long long *>(base + kStatusOff + 16);
  noalloc_prepare<<<1, 1, 0, st>>>(I, d_inst, I.status, counters);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = spl::launch_scan_mixed(d_inst, nullptr, 1, I.ntiles, sms, counters, st, 1);
  if (e == cudaSuccess) e = spl::launch_scan_mixed(d_inst, nullptr, 1, I.ntiles, sms, counters + 1, st, 2);
  if (e != cudaSuccess) return SPL_ERR_CUDA;
  if (status_out) {
    unsigned bits = 0;
    // device -> pageable host: returns once the copy (and all earlier work on st) is done
    if (cudaMemcpyAsync(&bits, I.status, sizeof(bits), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return SPL_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SPL_ERR_CUDA;
    *status_out = (bits & spl::kStNonFinite) ? SPL_ERR_NONFINITE
                  : (bits & spl::kStNotIncreasing) ? SPL_ERR_NOT_INCREASING : SPL_OK;
  }
  return SPL_OK;
}
