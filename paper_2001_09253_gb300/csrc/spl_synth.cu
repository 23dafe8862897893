// Device copy of the benchmark-curve generator (the host copy is synth.py).
// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) used counter-style; knots are the exact
// integer prefix sum of (top 27 bits + 1) scaled by 2^-27, so a parallel scan reproduces
// the sequential sum bit for bit.
#include "spl_internal.h"

namespace spl {
namespace {

constexpr unsigned long long kGolden = 0x9E3779B97F4A7C15ULL;
constexpr unsigned long long kInst = 0xD1B54A32D192ED03ULL;
constexpr int kBlock = 256;
constexpr int kPer = 16;                  // elements per thread
constexpr int kChunk = kBlock * kPer;     // elements per block

__host__ __device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

unsigned long long stream_key(unsigned long long seed, unsigned long long inst, unsigned long long stream) {
  unsigned long long k = mix64(seed + kGolden);
  return mix64(k + inst * kInst + stream);
}

// increment of knot i (i >= 1): draw i-1 of the x stream, top 27 bits, plus one
__device__ __forceinline__ long long increment(unsigned long long kx, long long i) {
  unsigned long long r = mix64(kx + (unsigned long long)i * kGolden);
  return (long long)(r >> 37) + 1;
}

__device__ long long block_sum(long long v) {
  __shared__ long long warp_sums[kBlock / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = v;
  __syncthreads();
  long long t = 0;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < kBlock / 32) ? warp_sums[threadIdx.x] : 0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;  // valid in thread 0
}

// exclusive block scan of one value per thread
__device__ long long block_exscan(long long v, long long *total) {
  __shared__ long long warp_tot[kBlock / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    long long u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    long long t = (lane < kBlock / 32) ? warp_tot[lane] : 0;
    long long ti = t;
    for (int o = 1; o < 32; o <<= 1) {
      long long u = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += u;
    }
    if (lane < kBlock / 32) warp_tot[lane] = ti - t;  // exclusive warp offsets
    if (lane == kBlock / 32 - 1) *total = ti;
  }
  __syncthreads();
  long long r = warp_tot[w] + inc - v;
  __syncthreads();
  return r;
}

// phase 1: per-block sums of the increments of knots [1 + b*kChunk, ...)
__global__ void gen_sums(unsigned long long kx, long long n, long long *sums) {
  const long long base = 1 + (long long)blockIdx.x * kChunk;
  long long v = 0;
  for (int e = 0; e < kPer; ++e) {
    long long i = base + (long long)threadIdx.x * kPer + e;
    if (i < n) v += increment(kx, i);
  }
  long long s = block_sum(v);
  if (threadIdx.x == 0) sums[blockIdx.x] = s;
}

// phase 2: exclusive scan of the block sums, one block
__global__ void gen_scan_sums(long long *sums, int nb) {
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int off = 0; off < nb; off += kBlock) {
    int i = off + threadIdx.x;
    long long v = (i < nb) ? sums[i] : 0;
    long long tot = 0;
    __shared__ long long tot_s;
    long long ex = block_exscan(v, &tot_s);
    tot = tot_s;
    if (i < nb) sums[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
}

// phase 3: knots from the scanned sums, values from the y stream
__global__ void gen_write(unsigned long long kx, unsigned long long ky, long long n, const long long *sums,
                          double *x, double *y) {
  const long long base = 1 + (long long)blockIdx.x * kChunk;
  long long loc[kPer];
  long long v = 0;
  for (int e = 0; e < kPer; ++e) {
    long long i = base + (long long)threadIdx.x * kPer + e;
    loc[e] = (i < n) ? increment(kx, i) : 0;
    v += loc[e];
  }
  __shared__ long long tot;
  long long pre = block_exscan(v, &tot) + sums[blockIdx.x];
  for (int e = 0; e < kPer; ++e) {
    long long i = base + (long long)threadIdx.x * kPer + e;
    pre += loc[e];
    if (i < n) x[i] = (double)pre * 0x1p-27;
  }
  // values: this block also writes y for the same index range, and y[0]/x[0] in block 0
  for (int e = 0; e < kPer; ++e) {
    long long i = base + (long long)threadIdx.x * kPer + e;
    if (i < n) y[i] = (double)(mix64(ky + (unsigned long long)(i + 1) * kGolden) >> 11) * 0x1p-53;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    x[0] = 0.0;
    y[0] = (double)(mix64(ky + kGolden) >> 11) * 0x1p-53;
  }
}

}  // namespace

size_t generate_scratch_bytes(long long n) {
  long long nb = (n > 1) ? (n - 1 + kChunk - 1) / kChunk : 1;
  return (size_t)nb * sizeof(long long);
}

cudaError_t launch_generate_curve(uint64_t seed, uint64_t instance, long long n, double *x, double *y,
                                  void *scratch, cudaStream_t stream, int *launches) {
  const unsigned long long kx = stream_key(seed, instance, 0), ky = stream_key(seed, instance, 1);
  long long nb = (n > 1) ? (n - 1 + kChunk - 1) / kChunk : 1;
  long long *sums = static_cast<long long *>(scratch);
  gen_sums<<<(unsigned)nb, kBlock, 0, stream>>>(kx, n, sums);
  gen_scan_sums<<<1, kBlock, 0, stream>>>(sums, (int)nb);
  gen_write<<<(unsigned)nb, kBlock, 0, stream>>>(kx, ky, n, sums, x, y);
  if (launches) *launches += 3;
  return cudaGetLastError();
}

}  // namespace spl
