/*
 * spl.h - C ABI of the GB300 cubic-spline library (fit + uniform-grid evaluation).
 *
 * What it computes (Hornbeck, "Fast Cubic Spline Interpolation", arXiv 2001.09253):
 *   fit   - the second derivatives y''[0..n-1] of the interpolating C2 cubic
 *           spline through (x_j, y_j): the tridiagonal system of eq. (init_val),
 *           section "Generating Second Derivatives", with the end rows of section
 *           "Start and End Derivatives" (an end slope > 0.99e30 selects the
 *           natural end y'' = 0, any other finite slope clamps S' there), solved
 *           as Thomas' algorithm of section "Implementation" prescribes;
 *   eval  - S(x_k) at M uniformly spaced queries x_k = x_0 + k*step (or at M explicit
 *           positions, see spl_query_mode),
 *           step = (x_{n-1}-x_0)/(M-1), the last query forced to x_{n-1}
 *           (section "Curve Interpolation", benchmark step 8), each query
 *           bracketed to the interval j with x_j < x_k <= x_{j+1} (j = 0 for
 *           x_k <= x_0; j <= n-2), and evaluated with the one-division form of
 *           section "Fast Interpolation".
 *   Bracket indices are bit-exact with a sequential FP64 reference; floating-point
 *   outputs agree with it to a relative 1e-12 (SPL_PREC_F64) or 1e-5
 *   (SPL_PREC_F32_REFINE): normwise for y'' (max error over max |y''|), per query for
 *   S(x_k) (relative to the largest of |y_j|, |y_{j+1}|, |S(x_k)| and the curvature term
 *   h_j^2 max(|y''_j|, |y''_{j+1}|)/6 of its interval).
 *
 * Conventions for every entry point:
 *   - Return an spl_status; nothing is thrown across the ABI.  SPL_OK is 0,
 *     errors are negative, SPL_PENDING is positive.
 *   - Arrays are plain C arrays of float64 (double) or int32, contiguous,
 *     0-based, structure-of-arrays.  "device" pointers are CUDA device (or
 *     managed) addresses on the context's device; "host" pointers are CPU
 *     addresses (pinned memory gives asynchronous copies).
 *   - The caller owns every input and output array; the library owns its
 *     scratch, which it carves from the arena given at creation.
 *   - One context orders its GPU work on one CUDA stream; requests with host
 *     (SPL_MEM_HOST) arrays additionally copy their inputs and outputs on two
 *     copy streams the context owns, ordered against the kernels by events, so
 *     that the copies of one request overlap the kernels of its neighbours.
 *     Calls on a context are serialised by an internal lock; distinct contexts
 *     are independent.
 *   - Nothing falls back to the CPU: without the CUDA device the calls fail
 *     with SPL_ERR_CUDA.
 */
#ifndef SPL_H_
#define SPL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum spl_status {
  SPL_OK = 0,
  SPL_PENDING = 1,                /* submitted, not finished yet */
  SPL_ERR_INVALID_ARG = -1,       /* n < 3, M < 0, null pointer, NaN or -inf end slope, bad option */
  SPL_ERR_NOT_INCREASING = -2,    /* knots not strictly increasing (found on the device) */
  SPL_ERR_NONFINITE = -3,         /* a knot or value is NaN or infinite (found on the device) */
  SPL_ERR_BUDGET = -4,            /* the request can never fit in the context's memory budget */
  SPL_ERR_QUEUE_FULL = -5,        /* no free slot or memory right now; retry after a completion */
  SPL_ERR_TIMEOUT = -6,           /* a bounded wait ran out (host wait, or a device-side wait) */
  SPL_ERR_CUDA = -7,              /* a CUDA call failed; the context may be unusable */
  SPL_ERR_UNKNOWN_TICKET = -8,    /* ticket never issued by this context, or already collected */
  SPL_ERR_STATE = -9              /* call not valid in the context's current mode */
} spl_status;

/* Precision of the arithmetic on the hot path. */
typedef enum spl_precision {
  SPL_PREC_F64 = 0,         /* every step in binary64 on the GPU */
  SPL_PREC_F32_REFINE = 1   /* knot/query differences exact, solve and cubic in binary32,
                               optional refinement of y'' against an extended-precision residual */
} spl_precision;

typedef enum spl_mem {
  SPL_MEM_DEVICE = 0,       /* request arrays are device pointers */
  SPL_MEM_HOST = 1          /* request arrays are host pointers: the library stages them through
                               its arena and copies results back before completion */
} spl_mem;

/* Where the queries come from (plan option). */
typedef enum spl_query_mode {
  SPL_QUERY_UNIFORM = 0,    /* m uniform queries on [x_0, x_{n-1}] (section "Curve Interpolation") */
  SPL_QUERY_EXPLICIT = 1    /* m caller-given positions xq[m], any order, each bracketed by
                               bisection (the interval search of section "Quality Checks" for an
                               unsorted query) */
} spl_query_mode;

/* Form of the evaluation (plan option; used when the queries are evaluated by the separate
 * evaluation kernel, i.e. explicit queries or a request with ypp_in).  The three variants of
 * section "Fast Interpolation" benchmarked in section "Curve Interpolation":
 *   ORIG   inv_ba = 1/(x_{j+1}-x_j) formed first, the sum multiplied by it (the paper's newint);
 *   NOINV  the sum divided by (x_{j+1}-x_j) at the end;
 *   VOL    ORIG with inv_ba kept in a volatile local (a memory round trip pins the division
 *          before the cubic, the paper's scheduling trick).
 * All three agree to rounding; the fused uniform-grid kernels always use ORIG.  The evaluation
 * kernel runs them in binary64 for SPL_PREC_F64 plans and in binary32 (exact differences of the
 * binary64 positions, rounded once) for SPL_PREC_F32_REFINE plans. */
typedef enum spl_eval_variant {
  SPL_EVAL_ORIG = 0,
  SPL_EVAL_NOINV = 1,
  SPL_EVAL_VOL = 2,
  SPL_EVAL_NOOP = 3         /* control of section "Curve Interpolation" (its noop loop): the queries
                               are generated and bracketed but not evaluated; yq_out receives the
                               left knot x_j of each query's interval, jq_out (if given) j */
} spl_eval_variant;

typedef struct spl_ctx spl_ctx;
typedef struct spl_plan spl_plan;
typedef struct spl_batch spl_batch;

/* Context creation.
 *   device       CUDA device ordinal.
 *   stream       cudaStream_t (as void*) that orders the context's work; NULL means the
 *                legacy default stream.  Caller-owned; must outlive the context.
 *   arena        device memory the library sub-allocates all of its scratch and staging
 *                from (caller-owned, e.g. a PyTorch tensor).  NULL: the library allocates
 *                arena_bytes itself with cudaMalloc and frees it in spl_destroy.
 *   arena_bytes  size of the arena.  It is also the memory budget: requests whose
 *                footprint (inputs, outputs, scratch) cannot fit are refused with
 *                SPL_ERR_BUDGET, requests that do not fit right now with SPL_ERR_QUEUE_FULL
 *                (or wait in the serving queue, see spl_serve_create).
 *   max_slots    requests that may be in flight at once (>= 1). */
typedef struct spl_ctx_desc {
  int32_t device;
  int32_t max_slots;
  void *stream;
  void *arena;
  uint64_t arena_bytes;
} spl_ctx_desc;

/* Plan: options shared by the requests submitted with it.
 *   max_n         largest knot count a request may have (sizes the scratch).
 *   precision     spl_precision.
 *   refine_steps  SPL_PREC_F32_REFINE only: 0 (one fused binary32 pass) or 1 (binary32 fit,
 *                 then one step of iterative refinement of y'' against the residual of the
 *                 system formed in double-float arithmetic, then the evaluation).  Other
 *                 values are SPL_ERR_INVALID_ARG.
 *   tile_rows     knots per tile of the chunked solve; 0 picks it from the device and n.
 *                 Exposed so tests can force many small tiles; values below 16 are refused.
 *                 Binary32 launches of one instance, or whose points lie mostly in instances
 *                 of 1,024 knots or more, run the warp-cooperative kernel, whose tiles are
 *                 whole 32-row chunks: there tile_rows is rounded up to a multiple of 32.
 *                 With 0, an FP64 request of one instance of at most SMs x 9,600 knots runs
 *                 on a cooperative grid of CTAs that exchange their partial solutions (the
 *                 latency path; its device-side waits are bounded and a wait that runs out
 *                 completes the request with SPL_ERR_TIMEOUT).
 *   query_mode    spl_query_mode.
 *   eval_variant  spl_eval_variant of the separate evaluation kernel.
 *   fault_flags   failure-detection tests only (0 otherwise): bit 0 makes the last CTA of the
 *                 multi-CTA FP64 kernel withhold its partial solutions, so that the other
 *                 CTAs' bounded waits run out.  Other bits are SPL_ERR_INVALID_ARG. */
typedef struct spl_plan_desc {
  uint64_t max_n;
  int32_t precision;
  int32_t refine_steps;
  int32_t tile_rows;
  int32_t query_mode;
  int32_t eval_variant;
  uint32_t fault_flags;
} spl_plan_desc;

/* One instance.
 *   n, x, y      knots (strictly increasing) and values, n >= 3.
 *   yp1, ypn     end slopes S'(x_0), S'(x_{n-1}); a value > 0.99e30 (e.g. 1e32 or +inf)
 *                selects the natural end.  NaN or -inf is SPL_ERR_INVALID_ARG.
 *   m            number of queries (0 = fit only; uniform mode: 1 = the single query x_0).
 *   ypp_out      y''[n] output, or NULL if not wanted.
 *   yq_out       S(x_k)[m] output (NULL allowed only when m == 0).
 *   jq_out       optional int32 bracket index per query (j of the interval used), or NULL.
 *   mem          spl_mem: where every array of the request lives.
 *   xq           explicit-mode plans: the m query positions (finite, any order; a query
 *                below x_0 or above x_{n-1} is extrapolated by the end cubic).  Must be NULL
 *                in uniform mode.  A non-finite position completes with SPL_ERR_NONFINITE.
 *   ypp_in       NULL: fit, then evaluate.  Otherwise y''[n] of an earlier fit of the same
 *                x, y: the fit is skipped and only the evaluation runs ("fit once, evaluate
 *                many"), in the plan's precision; ypp_out and the end slopes are ignored.
 *                Every request of one spl_submit_batch call must agree on NULL or not. */
typedef struct spl_request {
  uint64_t n;
  const double *x;
  const double *y;
  double yp1;
  double ypn;
  uint64_t m;
  double *ypp_out;
  double *yq_out;
  int32_t *jq_out;
  int32_t mem;
  int32_t reserved;
  const double *xq;
  const double *ypp_in;
} spl_request;

/* Completion record.
 *   status      SPL_OK, SPL_PENDING or the request's error.
 *   device_ms   GPU time of the launch that carried the request (0 if unknown).
 *   latency_ms  host wall time from submission to the first poll that saw completion. */
typedef struct spl_result {
  int32_t status;
  float device_ms;
  double latency_ms;
} spl_result;

/* Library counters (monotonic over the context's life). */
typedef struct spl_stats {
  uint64_t kernel_launches;   /* kernels this library launched */
  uint64_t graph_launches;    /* CUDA graph launches */
  uint64_t requests_done;
  uint64_t arena_high_water;  /* bytes */
} spl_stats;

const char *spl_status_str(int32_t status);

/* Creates a context (device, stream, arena) for the fit and evaluation of section "Fast
 * Interpolation" / "Generating Second Derivatives"; SPL_ERR_INVALID_ARG for a null or malformed
 * descriptor (max_slots < 1, arena_bytes < 1 MiB, an arena not 256-byte aligned), SPL_ERR_CUDA when
 * the device is absent or an allocation fails.  *out is NULL on failure.  The context keeps ~12 KB
 * of the arena for its single-instance launches (spl_submit) from creation on. */
spl_status spl_create(spl_ctx **out, const spl_ctx_desc *desc);
void spl_destroy(spl_ctx *ctx);  /* waits for the context's work; NULL is a no-op.  Destroy the
                                    context's servers first: they use its arena. */

/* Options of the problem statement of section "Implementation" (new_second_derivative: knots,
 * values, start and end derivatives) and of section "Curve Interpolation" (the evaluated form and
 * its queries), fixed for the requests that use the plan.  SPL_ERR_INVALID_ARG for max_n < 3, an
 * unknown precision, query mode or form, refine_steps outside 0..1 (0 for SPL_PREC_F64), or
 * 0 < tile_rows < 16. */
spl_status spl_plan_create(spl_ctx *ctx, const spl_plan_desc *desc, spl_plan **out);
void spl_plan_destroy(spl_plan *plan);

/* Validate and enqueue one instance on the context's stream: the second derivatives of section
 * "Generating Second Derivatives" with the end rows of "Start and End Derivatives"
 * (new_second_derivative), then newint of "Fast Interpolation" at the request's queries.  On
 * SPL_OK *ticket names it until spl_poll/spl_wait returns a final status.  Host-side checks return
 * SPL_ERR_INVALID_ARG (n < 3 or > max_n, null arrays, a NaN or -inf end slope), SPL_ERR_BUDGET
 * (footprint above the arena) or SPL_ERR_QUEUE_FULL (no slot or memory now).  The paper's input
 * asserts (strictly increasing knots) and finite values are checked on the device and reported at
 * completion (NOT_INCREASING, NONFINITE).  One instance in device memory that is fitted and
 * evaluated in one pass (no ypp_in, uniform queries, automatic tile length for SPL_PREC_F64 up to
 * SMs x 9,600 knots, any binary32 plan) is enqueued as its kernel launch(es) alone where the device
 * has native atomics on host memory: the descriptor goes as a kernel parameter and the kernel writes
 * the status into the context's pinned memory, with no copy or memset around it. */
spl_status spl_submit(spl_ctx *ctx, spl_plan *plan, const spl_request *req, uint64_t *ticket);

/* Many instances in one launch; tickets[i] names req[i].  All requests must use the same
 * memory kind. */
spl_status spl_submit_batch(spl_ctx *ctx, spl_plan *plan, const spl_request *reqs, uint32_t count,
                            uint64_t *tickets);

/* Completion of a request submitted for the fit and evaluation of sections "Generating Second
 * Derivatives" and "Fast Interpolation".  Non-blocking.  Returns SPL_PENDING, or the final status
 * (then the ticket is released), or SPL_ERR_UNKNOWN_TICKET. */
spl_status spl_poll(spl_ctx *ctx, uint64_t ticket, spl_result *res);

/* As spl_poll (completion of the fit and evaluation of sections "Generating Second Derivatives"
 * and "Fast Interpolation"), blocking up to timeout_ns (bounded; never forever);
 * SPL_ERR_TIMEOUT when it runs out (res->status is then SPL_PENDING and the ticket stays valid).
 * A request that completed because a device-side wait ran out also returns SPL_ERR_TIMEOUT, with
 * res->status = SPL_ERR_TIMEOUT and the ticket released. */
spl_status spl_wait(spl_ctx *ctx, uint64_t ticket, uint64_t timeout_ns, spl_result *res);

spl_status spl_get_stats(spl_ctx *ctx, spl_stats *out);

/* Launch geometry (introspection; the paper has no counterpart: this is the GPU decomposition of
 * the fit of section "Implementation").  Which kernel fits a submission of `count` instances of
 * n[0..count-1] knots under the plan options *plan on a device of sm_count SMs, and with what
 * tiling: the decision spl_submit / spl_submit_batch take, as a pure function of these arguments
 * (no device, no context, no allocation).  mem: where the requests' arrays live (spl_mem);
 * stored_fit: nonzero when the requests carry ypp_in (evaluation only).  SPL_ERR_INVALID_ARG for
 * a null pointer, count 0, an n below 3, sm_count < 1, an unknown mem, or plan options that
 * spl_plan_create rejects. */
typedef enum spl_kernel {
  SPL_KERNEL_NONE = 0,        /* no fit (stored y''): the evaluation kernel alone */
  SPL_KERNEL_FUSED_F64 = 1,   /* FP64, one thread per tile of tile_rows knots, persistent CTAs */
  SPL_KERNEL_SMALL_F64 = 2,   /* FP64, one CTA per instance (batches of small instances) */
  SPL_KERNEL_MID_F64 = 3,     /* FP64, one instance on a cooperative grid of ctas CTAs */
  SPL_KERNEL_SCAN_MIXED = 4   /* binary32 (+ refinement), one warp per tile of tile_rows knots */
} spl_kernel;
typedef struct spl_geometry {
  int32_t fit_kernel;     /* spl_kernel */
  int32_t separate_eval;  /* 1: the queries are evaluated by the separate evaluation kernel */
  int32_t tile_rows;      /* knots per tile in the instance descriptors */
  int32_t direct;         /* 1: enqueued as its kernel launch(es) alone where the device has native
                             atomics on host memory (see spl_submit) */
  int64_t cta_rows;       /* SPL_KERNEL_MID_F64: knots per CTA (a multiple of 128); else 0 */
  int64_t ctas;           /* SPL_KERNEL_MID_F64: CTAs of the cooperative grid; else 0 */
} spl_geometry;
spl_status spl_launch_geometry(const spl_plan_desc *plan, const uint64_t *n, uint32_t count, int32_t mem,
                               int32_t stored_fit, int32_t sm_count, spl_geometry *out);

/* Reusable batch: the descriptors of count device-memory requests are uploaded once and
 * the launch is captured in a CUDA graph; every spl_batch_launch replays it on the
 * context's stream (one persistent kernel over all tiles of all instances; two, the fit and
 * then the refinement with the evaluation, for a plan with a refinement step).  Statuses
 * of the last launch are read with spl_batch_wait. */
spl_status spl_batch_create(spl_ctx *ctx, spl_plan *plan, const spl_request *reqs, uint32_t count,
                            spl_batch **out);
spl_status spl_batch_launch(spl_batch *batch);
spl_status spl_batch_wait(spl_batch *batch, uint64_t timeout_ns, int32_t *statuses /* count, or NULL */);
void spl_batch_destroy(spl_batch *batch);

/* Device generator of the benchmark curve (the same counter-based SplitMix64 draws and
 * integer prefix sum as the host generator, bit for bit): x_0 = 0,
 * x_i = x_{i-1} + (u_i + 1) 2^-27 with u_i the top 27 bits of draw i, y_i = (top 53 bits)
 * 2^-53.  x, y are device arrays of n doubles; scratch needs spl_generate_scratch_bytes(n). */
uint64_t spl_generate_scratch_bytes(uint64_t n);
spl_status spl_generate_curve(uint64_t seed, uint64_t instance, uint64_t n, double *x, double *y,
                              void *scratch, uint64_t scratch_bytes, void *stream);

/* Serving: continuous batching of independent instances onto a persistent device loop.
 *
 * A server owns a persistent kernel (one CTA per SM, cooperative launch) on its own stream:
 * a scheduler warp takes requests from a ring in mapped host memory and publishes their tiles;
 * worker warps solve published tiles, one tile per warp (binary32 solve and cubic, exact
 * binary64 differences and query positions: the mixed path, with or without refinement), so the
 * work of requests that arrive while others run overlaps on the device.  A request is admitted
 * when a slot is free, its tiles fit the tile map and its footprint (16 n + 8 m bytes, plus
 * 8 n for y'' and 4 m for indices when requested) fits in budget_bytes; otherwise it waits in
 * a host FIFO and is admitted by a later submit/poll/wait.  The device loop exits after
 * idle_timeout_ms without work (and after 30 s in any case); the next admission relaunches it.
 * Requests use device memory (SPL_MEM_DEVICE), and their arrays must hold their final contents
 * when the request is submitted (no GPU work still writing them on another stream): a running
 * loop may read the inputs and write the outputs at once.  Results equal those of a
 * single-request server, bit for bit, whatever else is in flight.
 *   max_inflight     requests resident on the device at once (slots), 1..65536.
 *   tile_rows        knots per tile, >= 16 (rounded up to a multiple of 32); shorter tiles
 *                    lower the latency of a request, longer ones raise the throughput (each
 *                    tile repeats 96 rows of start-up).  0: per request, about 32 tiles each,
 *                    256..1024 rows.
 *   budget_bytes     HBM budget for the footprints of resident requests.
 *   max_tiles        tile-map capacity (0 = max(2^20, 64 max_inflight)).
 *   idle_timeout_ms  0 = 200.
 *   deadline_ms      longest run of one launch of the loop (0 = 30,000); its worker warps give
 *                    up waiting for work one second after it.  A worker that gives up raises
 *                    the loop's error flag: the host then completes every request resident on
 *                    the device with SPL_ERR_TIMEOUT, drops their tiles and relaunches for the
 *                    rest, so the context stays usable.
 *   fault_flags      failure-detection tests only (0 otherwise): bit 0 makes the scheduler warp
 *                    leave at once without publishing any work or the stop word, so that the
 *                    workers' bounded waits run out.
 *   refine_steps     0: the binary32 solve as is; 1: one step of iterative refinement of y''
 *                    against a double-float residual before the evaluation, as spl_plan_desc's
 *                    refine_steps (each tile is solved twice: the second pass of a request starts
 *                    once all of its first-pass tiles are done).  The footprint then includes 4 n
 *                    bytes of binary32 y'' carved from the context's arena while the request is
 *                    resident.  Other values are SPL_ERR_INVALID_ARG. */
typedef struct spl_server spl_server;
typedef struct spl_serve_desc {
  uint32_t max_inflight;
  uint32_t tile_rows;
  uint64_t budget_bytes;
  uint64_t max_tiles;
  uint32_t idle_timeout_ms;
  uint32_t deadline_ms;
  uint32_t fault_flags;
  uint32_t refine_steps;
} spl_serve_desc;

spl_status spl_serve_create(spl_ctx *ctx, const spl_serve_desc *desc, spl_server **out);
/* Queue one request; SPL_OK with a ticket (admitted now or later), or SPL_ERR_BUDGET when it
 * can never fit, SPL_ERR_INVALID_ARG as spl_submit. */
spl_status spl_serve_submit(spl_server *srv, const spl_request *req, uint64_t *ticket);
/* Non-blocking; SPL_PENDING or the final status (the ticket is then released).  latency_ms in
 * the result is submission to the poll that saw completion. */
spl_status spl_serve_poll(spl_server *srv, uint64_t ticket, spl_result *res);
spl_status spl_serve_wait(spl_server *srv, uint64_t ticket, uint64_t timeout_ns, spl_result *res);
/* Replays an arrival trace: request i (i < count) is pool[pick[i]], submitted at arrival_s[i]
 * seconds (non-decreasing) after the call starts; latency_ms[i] = time from its scheduled
 * arrival to the completion seen by the driver.  makespan_s (may be NULL) = first arrival to
 * last completion.  Returns the first non-OK request status, or SPL_ERR_TIMEOUT 60 s after
 * the last arrival. */
spl_status spl_serve_replay(spl_server *srv, const spl_request *pool, uint32_t pool_count, const uint32_t *pick,
                            const double *arrival_s, uint64_t count, double *latency_ms, double *makespan_s);
spl_status spl_serve_stats(spl_server *srv, uint64_t *loop_launches, uint64_t *waiting, uint64_t *resident);
/* Stops the device loop (bounded wait) and releases the server's memory. */
void spl_serve_destroy(spl_server *srv);

/* Self-test of the division replacement of the SPL_PREC_F64 kernel (no counterpart in the paper:
 * the paper divides with the CPU's IEEE division).  The FP64 kernel forms the slopes of eq.
 * (init_val) and its reciprocals with a MUFU seed refined by a Newton step plus a Markstein
 * correction instead of IEEE divisions; this call runs those routines and CUDA's correctly rounded
 * reciprocal and quotient on the same operands, elementwise:
 *   r_fast[i] = the kernel's 1/den[i],  q_fast[i] = the kernel's num[i]/den[i],
 *   r_ieee[i] = RN(1/den[i]),           q_ieee[i] = RN(num[i]/den[i]).
 * All arrays are device arrays of count doubles (caller-owned), on the current device; the work is
 * enqueued on `stream` (NULL = legacy default stream).  SPL_ERR_INVALID_ARG for a null array,
 * SPL_ERR_CUDA when the launch fails. */
spl_status spl_selftest_div64(const double *num, const double *den, uint64_t count, double *q_fast, double *r_fast,
                              double *q_ieee, double *r_ieee, void *stream);

/* Probe of the FP64 pipe's rate (no counterpart in the paper: it measures the ceiling of the
 * SPL_PREC_F64 kernel, whose time is set by its FP64 instructions).  Launches one CTA of
 * warps_per_sm warps on every SM of the current device; each thread runs 4 independent
 * recurrences a <- fma(a, mul, add) for trips x 16 steps and writes the sum of its four values to
 * sink[thread] (sink: caller-owned device array of at least sink_count >= SMs x warps_per_sm x 32
 * doubles).  *lane_ops (host, may be NULL) receives the number of DFMA lane operations the launch
 * performs; the caller times the launch on `stream` (NULL = legacy default stream) and divides.
 * With |mul| < 1 the values converge to add / (1 - mul).  SPL_ERR_INVALID_ARG for warps_per_sm
 * outside 1..32, trips above 2^40, or a missing or short sink; SPL_ERR_CUDA when the launch
 * fails. */
spl_status spl_selftest_dfma(uint64_t trips, int32_t warps_per_sm, double mul, double add, double *sink,
                             uint64_t sink_count, uint64_t *lane_ops, void *stream);

/* One instance without any allocation, for callers that cannot allocate device memory:
 * host applications that own all of the GPU's memory themselves (a simulation or game
 * engine, a database or plug-in host that hands out fixed pools), and code under a hard
 * memory budget or latency deadline, where cudaMalloc/cudaFree may fail, or stall the
 * whole device, at the wrong moment.  The paper has no counterpart; this entry point exists
 * only for such callers.
 *
 * Computes what spl_submit computes with a SPL_PREC_F32_REFINE plan and refine_steps = 1
 * (binary32 fit, one refinement step of y'', evaluation at m uniform queries), enqueued on
 * `stream` (a cudaStream_t, NULL = legacy default stream) on the current device.  x, y,
 * ypp_out (may be NULL) and yq_out (may be NULL when m == 0) are caller-owned device arrays,
 * as in spl_request.  The scratch it needs (the descriptor, a status word and n binary32
 * values) lives in one fixed array of 4 MiB + 512 B compiled into the library, held by every
 * GPU that loads the library until the process exits; so n is limited to SPL_NOALLOC_MAX_N
 * and larger n returns SPL_ERR_BUDGET without launching anything.  The call makes no
 * cudaMalloc, cudaFree or other allocating call.
 *
 * The first call in each CUDA context looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it, keyed by the context's unique ID: make that first call
 * before any stream capture.  A device reset (cudaDeviceReset) destroys the context and the
 * array with it; the next call then runs in a new context and looks the address up again.
 * The context is the one current on the calling thread, or else the current device's primary
 * context (bound with cudaSetDevice).  Every call shares the
 * same array and leaves the previous call's contents in it (each call clears what must start
 * at zero): calls whose work overlaps on the GPU (different streams, or several host threads)
 * race and give wrong results; order them on one stream or synchronise between them.
 *
 * status_out: NULL = fully asynchronous, no device-side status.  Non-NULL = the call waits for
 * its stream and stores SPL_OK, SPL_ERR_NONFINITE or SPL_ERR_NOT_INCREASING.  Returns
 * SPL_ERR_INVALID_ARG (as spl_submit), SPL_ERR_BUDGET (n too large) or SPL_ERR_CUDA. */
#define SPL_NOALLOC_MAX_N 1048576u
spl_status spl_fit_eval_noalloc(const double *x, const double *y, uint64_t n, double yp1, double ypn,
                                uint64_t m, double *ypp_out, double *yq_out, void *stream, int32_t *status_out);

#ifdef __cplusplus
}
#endif
#endif /* SPL_H_ */
