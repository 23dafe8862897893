// Self-test of the FP64 division replacement of the plain FP64 kernel.
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

}  // namespace

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
