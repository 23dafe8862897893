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

// The scratch.  Every GPU that loads this library holds these 4 MiB + 512 B until the
// process exits.  Host code must not use this name as an address: it is a host-side stand-in;
// the device address comes from cudaGetSymbolAddress (see setup_device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 128;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices];  // device address of g_noalloc_scratch, per device
int g_sms[kMaxDevices];

// Once per device, with that device current: look up the array's device address.
spl_status setup_device(int dev, unsigned char **addr, int *sms) {
  if (dev < 0 || dev >= kMaxDevices) return SPL_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SPL_ERR_CUDA;
    int s = 0;
    if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SPL_ERR_CUDA;
    g_sms[dev] = s;
    g_addr[dev] = static_cast<unsigned char *>(p);
  }
  *addr = g_addr[dev];
  *sms = g_sms[dev];
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
  long long target = (long long)sms * spl::mixed_threads_per_sm();  // one tile per thread of one wave
  long long L = ((long long)n + target - 1) / target;
  L = L < 128 ? 128 : L;
  I.tile_rows = (int)L;
  I.ntiles = ((long long)n + L - 1) / L;
  I.tile_begin = 0;
  I.status = reinterpret_cast<unsigned *>(base + kStatusOff);
  I.z = reinterpret_cast<float *>(base + kZOff);
  spl::Inst *d_inst = reinterpret_cast<spl::Inst *>(base + kInstOff);

  unsigned long long *counters = reinterpret_cast<unsigned long long *>(base + kStatusOff + 16);
  noalloc_prepare<<<1, 1, 0, st>>>(I, d_inst, I.status, counters);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = spl::launch_fused_mixed(d_inst, 1, I.ntiles, sms, counters, st, true);
  if (e == cudaSuccess) e = spl::launch_refine_mixed(d_inst, 1, I.ntiles, sms, counters + 1, st);
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
