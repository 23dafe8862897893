// Self-tests of the plain FP64 kernel's arithmetic: its division replacement, and the rate at which
// this part's FP64 pipe retires a pure DFMA stream (the ceiling of an FP64-bound kernel).
//
// The fused FP64 kernel forms the slopes s_j = (y_{j+1} - y_j) / h_j of eq. (init_val) and the
// reciprocals it multiplies by with spl::rcp64 (a MUFU seed and one third-order Newton step) and
// spl::quot64 (a Markstein correction of num * rcp64(den)) instead of IEEE divisions.  This entry
// point runs those two routines and CUDA's correctly rounded __drcp_rn / __ddiv_rn on the same
// operands, so a test can compare them bit for bit over any operand set.
#include "../../include/spl.h"
#include "spl_device.cuh"

namespace {

__global__ void div64_kernel(const double *__restrict__ num, const double *__restrict__ den, long long count,
                             double *__restrict__ q_fast, double *__restrict__ r_fast,
                             double *__restrict__ q_ieee, double *__restrict__ r_ieee) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    const double a = num[i], d = den[i];
    const double r = spl::rcp64(d);
    r_fast[i] = r;
    q_fast[i] = spl::quot64(a, d, r);
    r_ieee[i] = __drcp_rn(d);
    q_ieee[i] = __ddiv_rn(a, d);
  }
}

// kChains independent DFMA recurrences a <- a * mul + add per thread (kUnroll iterations per loop
// trip, so the loop's own integer work is a small share of the issue slots).  With mul < 1 the
// recurrences converge to add / (1 - mul): values stay bounded for any iteration count.
constexpr int kChains = 4;
constexpr int kUnroll = 16;

__global__ void dfma_kernel(long long trips, double mul, double add, double *__restrict__ sink) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = (double)(threadIdx.x & 31) * 0.001 + c;
  for (long long t = 0; t < trips; ++t) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = __fma_rn(a[c], mul, add);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  sink[tid] = s;
}

}  // namespace

extern "C" spl_status spl_selftest_dfma(uint64_t trips, int32_t warps_per_sm, double mul, double add, double *sink,
                                        uint64_t sink_count, uint64_t *lane_ops, void *stream) {
  if (warps_per_sm < 1 || warps_per_sm > 32 || trips > (1ull << 40)) return SPL_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPL_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SPL_ERR_CUDA;
  const uint64_t threads = (uint64_t)sms * (uint64_t)warps_per_sm * 32ull;
  if (!sink || sink_count < threads) return SPL_ERR_INVALID_ARG;
  if (lane_ops) *lane_ops = threads * trips * (uint64_t)(kUnroll * kChains);
  dfma_kernel<<<sms, warps_per_sm * 32, 0, static_cast<cudaStream_t>(stream)>>>((long long)trips, mul, add, sink);
  return cudaGetLastError() == cudaSuccess ? SPL_OK : SPL_ERR_CUDA;
}

extern "C" spl_status spl_selftest_div64(const double *num, const double *den, uint64_t count, double *q_fast,
                                         double *r_fast, double *q_ieee, double *r_ieee, void *stream) {
  if (count == 0) return SPL_OK;
  if (!num || !den || !q_fast || !r_fast || !q_ieee || !r_ieee || count > (1ull << 40)) return SPL_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPL_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SPL_ERR_CUDA;
  const long long blocks_needed = ((long long)count + 255) / 256;
  const int blocks = (int)(blocks_needed < 4LL * sms ? blocks_needed : 4LL * sms);
  div64_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(num, den, (long long)count, q_fast, r_fast,
                                                                      q_ieee, r_ieee);
  return cudaGetLastError() == cudaSuccess ? SPL_OK : SPL_ERR_CUDA;
}
