// Device-side pieces shared by the spline kernels: the instance descriptor, the tile
// geometry, order-preserving keys for exact bracketing, the uniform query grid and a
// reciprocal that keeps the FP64 pipe free of the full IEEE division.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace spl {

// Status bits a tile ORs into its instance's status word (device memory).  kStBadTile: a tile
// longer than the kernel's scratch holds (the host never launches one; the tile is skipped).
enum : unsigned { kStNonFinite = 1u, kStNotIncreasing = 2u, kStBadTile = 4u, kStWaitTimeout = 8u };

// One instance as the kernels see it (built by the host runtime, lives in device memory
// or in the kernel parameter block).
struct Inst {
  const double *x;      // knots, n
  const double *y;      // values, n
  double *ypp;          // y'' out, n (may be null)
  double *yq;           // S(x_k) out, m (null when m == 0)
  int32_t *jq;          // bracket index out, m (may be null)
  long long n, m;
  double yp1, ypn;      // end slopes (natural when > 0.99e30)
  long long tile_begin; // global index of this instance's first tile
  long long ntiles;     // tiles of this instance
  int tile_rows;        // knots per tile (the last tile of an instance is ragged)
  int pad;              // bit 0: grouped tile geometry (FP64 kernel); bit 1: served with refinement
  unsigned *status;     // device word, OR of kSt* bits
  float *z;             // mixed path with refinement: binary32 y'' of the first pass (n), scratch
  const double *xq;     // separate evaluation: explicit query positions (mq), or null for the grid
  long long mq;         // separate evaluation: queries (the fused kernels see m = 0 then)
  long long q_begin;    // separate evaluation: global index of this instance's first query
  const long long *ktab;// separate evaluation of explicit positions: keys of every kCoarseKeys-th
                        // knot (spl_internal.h; the coarse level of the bisection), or null
};

// Inst::pad bit of a served request with one refinement step (two passes over its tiles).
constexpr int kServeRefined = 2;

// One request appended by the host to the serving ring (mapped host memory).
struct ServeEntry {
  Inst inst;
  unsigned long long first_tile;  // global tile ticket of the request's first tile
  unsigned slot, seq;
};

// Arguments of the persistent serving kernel.
struct ServeArgs {
  unsigned long long *published, *claimed, *consumed;  // device counters
  unsigned *stop, *err;                                  // device flags
  Inst *slot_inst;                                       // per slot
  unsigned long long *slot_first;
  unsigned *slot_done, *slot_status, *slot_seq;
  unsigned *tile_slot;                                   // tile ticket % tile_cap -> slot
  unsigned long long tile_cap;
  const volatile unsigned long long *h_tail;             // mapped host memory, written by the host
  const volatile unsigned *h_stop;
  const ServeEntry *h_ring;
  unsigned long long rcap;
  volatile unsigned long long *h_consumed;               // mapped host memory, written by the device
  volatile unsigned *h_alive;
  volatile unsigned *h_done;                             // per slot: status, seq
  unsigned long long idle_ns, deadline_ns;
  unsigned fault_flags;                                  // tests: bit 0, the scheduler leaves at once
};

// Natural end condition: section "Start and End Derivatives" (slope > 0.99e30).
__device__ __forceinline__ bool is_natural(double slope) { return slope > 0.99e30; }

// Order-preserving signed key of a double (with -0 folded onto +0): for non-NaN a, b,
// a < b exactly when key(a) < key(b).  Compares run on the integer pipe instead of the
// (scarce) FP64 pipe and are exact, which keeps the bracket indices bit-identical to a
// sequential FP64 sweep.
__device__ __forceinline__ long long dkey(double v) {
  long long b = __double_as_longlong(v);
  b = (b == (long long)0x8000000000000000ULL) ? 0LL : b;
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}

// True for one element of each kPfBlock-byte aligned block of a stream walked one element at a time
// (in either direction): a software prefetch per block instead of one per element, since every
// prefetch instruction of a lane is a memory request of its own.
constexpr unsigned kPfBlock = 32;
template <typename T>
__device__ __forceinline__ bool first_in_block(const T *p) {
  return ((unsigned)(size_t)p & (kPfBlock - 1u)) < (unsigned)sizeof(T);
}

__device__ __forceinline__ bool finite64(double v) {
  return ((unsigned long long)__double_as_longlong(v) & 0x7FF0000000000000ULL) != 0x7FF0000000000000ULL;
}

// Biased binary64 exponent field of v (integer pipe).
__device__ __forceinline__ unsigned exp_field64(double v) { return ((unsigned)__double2hiint(v) >> 20) & 0x7FFu; }

// Correctly rounded IEEE forms, out of line so that the rare operands outside the fast routines'
// domain never put them on the common path.
static __device__ __noinline__ double rcp64_ieee(double d) { return __drcp_rn(d); }
static __device__ __noinline__ double quot64_ieee(double a, double b) { return __ddiv_rn(a, b); }

// 1/d: the MUFU seed (rcp.approx.ftz.f64, ~2^-22 relative) refined by one third-order
// Newton-Raphson step, r' = r + r(e + e^2) with e = 1 - d r (error ~ e^3 before the final
// rounding): three DFMAs instead of a full IEEE division.  The result is within one ulp of 1/d
// (correctly rounded in all but ~3 of 10^4 random operands, measured against __drcp_rn).  The seed
// flushes subnormals, so |d| outside [2^-1022, 2^1022) (and zero, infinities, NaN) takes the IEEE
// reciprocal instead.
__device__ __forceinline__ double rcp64(double d) {
  if (exp_field64(d) - 1u > 2043u) return rcp64_ieee(d);
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  double e = fma(-d, r, 1.0);
  double e2 = fma(e, e, e);
  return fma(r, e2, r);
}

// num/den from r = rcp64(den): q = num*r, then one Markstein correction q + (num - den*q)*r with
// the remainder formed exactly by the FMA.  Slopes s_j = (y_{j+1}-y_j)/h_j feed the cancelling
// difference s_j - s_{j-1}, where a one-ulp difference would be amplified, so they must equal the
// IEEE quotient: on GB300 this routine matched __ddiv_rn bit for bit on every operand tested
// (random, dyadic, continuous and 8-decade widths, powers of two and their neighbours, all-ones
// significands; the self-test entry point spl_selftest_div64) even where r itself was one ulp
// off.  The remainder is exact and the quotient normal only while neither operand nor the
// quotient approaches the ends of the exponent range, so operands outside 2^-963 <= |num| <
// 2^977, |den| within rcp64's domain and |num/den| within 2^+-1000 take the IEEE division (a zero
// numerator gives num * r, the correctly signed zero).
__device__ __forceinline__ double quot64(double num, double den, double r) {
  const int ea = (int)exp_field64(num), eb = (int)exp_field64(den);
  if (ea < 60 || ea > 2000 || (unsigned)(eb - 1) > 2043u || ea - eb > 1000 || eb - ea > 1000) {
    if (ea == 0 && (((unsigned long long)__double_as_longlong(num) << 1) == 0ull) && (unsigned)(eb - 1) <= 2043u)
      return num * r;
    return quot64_ieee(num, den);
  }
  double q = num * r;
  double rem = fma(-den, q, num);
  return fma(rem, r, q);
}

// Same seed and step for binary32 (MUFU rcp has ~1 ulp; one second-order step suffices).
// The MUFU binary32 reciprocal alone (~1 ulp).
__device__ __forceinline__ float rcp_approx32(float d) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  return r;
}

__device__ __forceinline__ float rcp32(float d) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  float e = fmaf(-d, r, 1.0f);
  return fmaf(r, e, r);
}

// Exact conversion of 0 <= k < 2^53 to double built with integer operations (the
// hardware int->f64 conversion runs at the FP64-pipe rate on this part).
__device__ __forceinline__ double i2d_exact(long long k) {
  if (k == 0) return 0.0;
  int lz = __clzll(k);                 // k has 64 - lz significant bits
  int e = 63 - lz;                     // floor(log2 k)
  unsigned long long mant = (((unsigned long long)k << lz) << 1) >> 12;  // drop the leading 1
  unsigned long long bits = ((unsigned long long)(1023 + e) << 52) | mant;
  return __longlong_as_double((long long)bits);
}

// Uniform query grid: x_k = x_0 + k*step with separately rounded product and sum, the
// last point forced to x_{n-1}; m == 1 gives x_0 (numpy linspace semantics).
struct Grid {
  double x0, xl, step;
  long long m;
  __device__ __forceinline__ double at(long long k) const {
    if (m == 1) return x0;
    if (k == m - 1) return xl;
    return __dadd_rn(__dmul_rn(i2d_exact(k), step), x0);
  }
};

__device__ __forceinline__ Grid make_grid(const double *x, long long n, long long m) {
  Grid g;
  g.x0 = x[0];
  g.xl = x[n - 1];
  g.m = m;
  g.step = (m >= 2) ? __ddiv_rn(__dsub_rn(g.xl, g.x0), (double)(m - 1)) : 0.0;
  return g;
}

// First query whose bracket index is >= s: k = 0 for s == 0, else the least k with
// x_k > x_s (queries are non-decreasing), found by bisection over [0, m].
__device__ __forceinline__ long long first_query(const Grid &g, const double *x, long long s) {
  if (s == 0 || g.m == 0) return 0;
  const long long ks = dkey(x[s]);
  long long lo = 0, hi = g.m;
  while (lo < hi) {
    long long mid = lo + ((hi - lo) >> 1);
    if (dkey(g.at(mid)) > ks) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// Instance owning global tile t (binary search over tile_begin).
__device__ __forceinline__ int find_inst(const Inst *insts, int ninst, long long t) {
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (insts[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Input checks of row j (section "Generating Second Derivatives" takes strictly increasing
// knots; finite values are required on top), made while a forward sweep passes the row.
__device__ __forceinline__ unsigned row_check(double xj, double yj, bool has_next, double xj1) {
  unsigned bad = (!finite64(xj) || !finite64(yj)) ? kStNonFinite : 0u;
  if (has_next && !(dkey(xj1) > dkey(xj))) bad |= kStNotIncreasing;
  return bad;
}

}  // namespace spl
