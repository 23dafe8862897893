// Host-side declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "spl_device.cuh"

namespace spl {

// Persistent-grid geometry: at most one CTA of max_threads per SM; when the tiles would not fill
// that, the CTAs shrink (to whole warps) so that the tiles spread over all SMs instead of
// crowding a few.
inline void spread_grid(int sm_count, long long tiles, int max_threads, int *blocks, int *block_threads) {
  const long long per_sm = (tiles + sm_count - 1) / sm_count;
  long long bt = (per_sm + 31) / 32 * 32;
  bt = bt < 32 ? 32 : (bt > max_threads ? max_threads : bt);
  long long b = (tiles + bt - 1) / bt;
  b = b < 1 ? 1 : (b > sm_count ? sm_count : b);
  *blocks = (int)b;
  *block_threads = (int)bt;
}

// FP64 fused fit + evaluation (spl_fused_f64.cu).  `threads` (threads_f64) sizes the scratch; `scratch`
// must hold ring_bytes_f64(threads, tile_rows) bytes, tile_rows being the longest tile of the
// launch; `counter` (8 bytes of device memory) must be zero when the kernel starts.
size_t ring_bytes_f64(long long threads, int tile_rows);
long long threads_f64(int sm_count, long long total_tiles);
int overhang_rows_f64();  // rows past a tile that start its back substitution
int lane0_short_rows_f64();  // rows the first tile of an FP64 warp group gives up for its halo
int f64_threads_per_sm();  // resident threads of the FP64 kernel per SM
cudaError_t launch_fused_f64(const Inst *d_insts, int ninst, long long total_tiles, double *scratch,
                             int tile_rows, int sm_count, unsigned long long *counter, cudaStream_t stream);

// FP64 fit + evaluation of small instances, one CTA per instance (spl_small_f64.cu): for
// instances of at most small_f64_max_rows() knots (latency path; no scratch beyond the CTA's
// shared memory).
int small_f64_max_rows();
cudaError_t launch_small_f64(const Inst *d_insts, int ninst, cudaStream_t stream);
// FP64 fit + evaluation of one mid-size instance on a cooperative grid of CTAs (spl_mid_f64.cu):
// mid_f64_cta_rows gives the rows per CTA for n points (0: beyond the path, n > SMs x 9600);
// the descriptor is *d_inst in device memory or, with d_inst null, *h_inst passed by value;
// `exchange` (mid_f64_exchange_bytes) carries the CTAs' maps: zeroed before the launch with
// launch = 0, else an area reserved for such launches and given a new launch number > 0 each time
// (never cleared); fault bit 0 makes the last CTA withhold its maps (failure-detection tests: the
// others' waits run out).
uint64_t mid_f64_exchange_bytes();
long long mid_f64_cta_rows(long long n, int sm_count);
cudaError_t launch_mid_f64(const Inst *d_inst, const Inst *h_inst, long long n, void *exchange,
                           unsigned long long launch, int sm_count, unsigned fault, cudaStream_t stream);

// Persistent serving loop (spl_mixed_scan.cu): a cooperative launch of one CTA per SM; its
// workers solve tiles of serve_tile_rows(tile_rows) rows (at most serve_tile_max()) with the
// warp-cooperative kernel's solver, each in its own shared memory.
cudaError_t launch_serve(const ServeArgs &args, int sm_count, cudaStream_t stream);
int serve_tile_rows(int tile_rows);
int serve_tile_max();

// Warp-cooperative binary32 fit + evaluation (spl_mixed_scan.cu): one warp per tile of
// scan_mixed_tile_rows rows (a multiple of 32, at most scan_mixed_tile_max()), its scratch in
// shared memory.  mode 0: fit + eval; 1: fit only into Inst::z (binary32), the refined path's
// first pass; 2: refinement of Inst::z + eval.  The descriptors are d_insts in device memory or,
// with d_insts null, the one instance *h_one passed by value.  Warps fetch tiles from `counter`,
// which must be zero when the kernel starts; the kernel leaves it at zero when it ends.
int scan_mixed_threads_per_sm();
int scan_mixed_tile_max();
int scan_mixed_tile_rows(long long total_points, int sm_count, int count);
long long threads_scan_mixed(int sm_count, long long total_tiles);
cudaError_t launch_scan_mixed(const Inst *d_insts, const Inst *h_one, int ninst, long long total_tiles, int sm_count,
                              unsigned long long *counter, cudaStream_t stream, int mode);

// Knots per entry of the coarse key table of the explicit-position evaluation (every 16th knot),
// and the entries of an instance's table: knots 0, 16, 32, ... up to n - 2.
constexpr int kCoarseKeys = 16;
__host__ __device__ __forceinline__ long long coarse_key_entries(long long n) {
  return (n - 1 + kCoarseKeys - 1) / kCoarseKeys;
}

// Separate evaluation (spl_eval.cu): queries q_begin .. q_begin+mq-1 of each instance, explicit
// (Inst::xq) or on the uniform grid, with the y'' in Inst::ypp; variant = spl_eval_variant; f32:
// the binary32 form of the mixed-precision plans.
// uniform: no instance of the launch has explicit positions (the queries ascend).
// max_coarse_entries: the largest coarse key table of the launch (Inst::ktab), 0 when none; the
// tables are filled by a kernel launched first.
cudaError_t launch_eval(const Inst *d_insts, int ninst, long long total_q, int variant, bool f32, bool uniform,
                        long long max_coarse_entries, int sm_count, cudaStream_t stream);

}  // namespace spl

// Context services for the other host translation units (defined in spl_runtime.cu; each
// takes the context's lock).
struct spl_ctx;
int spl_ctx_device(spl_ctx *c);
int spl_ctx_sms(spl_ctx *c);
char *spl_ctx_arena_base(spl_ctx *c);
bool spl_ctx_arena_alloc(spl_ctx *c, uint64_t bytes, uint64_t *off);
void spl_ctx_arena_release(spl_ctx *c, uint64_t off, uint64_t bytes);
void spl_ctx_count_launch(spl_ctx *c, int n);

namespace spl {

// Device curve generator (spl_synth.cu).
size_t generate_scratch_bytes(long long n);
cudaError_t launch_generate_curve(uint64_t seed, uint64_t instance, long long n, double *x, double *y,
                                  void *scratch, cudaStream_t stream, int *launches);

}  // namespace spl
