/*
 * pr.h -- C ABI of the GB300 (sm_103a) parallel-reduction library libpr.so.
 *
 * A reduction computes x_0 (x) x_1 (x) ... (x) x_{n-1} for an associative
 * combiner (x) (Section 1.1, "Problem Definition").  The library implements it
 * as one persistent kernel launch per call: grid-stride vector loads into
 * several independent per-thread accumulators (the loop unrolling of
 * Section 3, "Unrolling the step 1", on the persistent grid of Section 2.5),
 * warp and block combines (Sections 2.2-2.3), and the second stage of the
 * two-stage scheme (Section 2.3) fused into the same launch by a
 * last-block-done counter, combined in a fixed order so that results are
 * bitwise identical from run to run for a given launch configuration.
 *
 * Conventions for every entry point:
 *   - Data pointers (x, offsets, out, argidx, aux, grad_*) are DEVICE memory
 *     owned by the caller, except where a name says "host".  Nothing is freed
 *     or retained by the library.
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL is the
 *     legacy default stream) on the CURRENT device.  No host synchronisation
 *     happens unless stated.
 *   - The library owns a small workspace per (device, stream): block partials,
 *     completion counters and an error word.  It is created on the first call
 *     for that pair, or by pr_prepare(); after that, calls allocate nothing and
 *     may be captured into a CUDA graph.  A first call made while the stream is
 *     capturing fails with PR_ERR_INVALID.  Calls issued concurrently on ONE
 *     stream from several host threads are serialised by the stream itself.
 *   - Arguments are validated on the host before anything is enqueued: a
 *     non-OK status means nothing was launched.  pr_last_error_message() gives
 *     the reason.  Asynchronous device-side errors are reported by
 *     pr_last_device_error().
 *   - Integer / bitwise / max / min results are exact (bit-identical to the
 *     sequential loop).  Floating-point sums and products depend on the
 *     association order (Section 1.1, footnote on reordering); for a fixed
 *     configuration (pr_config) the order, and so the result, is fixed.
 *   - F64 PROD keeps a separate integer exponent, so no partial product
 *     overflows or underflows; half of each vector's factors multiply on the
 *     fp64 pipe (rounded to nearest), half as 64-bit integer significands
 *     (truncated, under 2^-61 each).  Of the n - 1 merges of partial
 *     products at most n / 2 round to nearest, the others truncate, and the
 *     conversion to double rounds once: within max(n - 1, 2) 2^-53 relative.
 *
 * Result types (pr_out_dtype):
 *   F32 -> F32;  F16/BF16: SUM,PROD -> F32, MAX,MIN -> same type;  F64 -> F64;
 *   I32: SUM -> I64 (exact), others -> I32 (PROD wraps mod 2^32);
 *   U32 -> U32 (SUM, PROD wrap mod 2^32);  I64 -> I64 (SUM, PROD wrap mod 2^64).
 *   AND/OR/XOR are defined on integer types only (PR_ERR_UNSUPPORTED on floats).
 * Empty input (n == 0, or an empty segment) yields the identity: SUM 0, PROD 1,
 * MAX -inf / INT_MIN / 0, MIN +inf / INT_MAX / UINT_MAX, AND all ones, OR/XOR 0.
 * Float MAX/MIN propagate NaN and order -0 below +0.
 */
#ifndef PR_H
#define PR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* pr_stream_t; /* identical to cudaStream_t */

typedef enum {
    PR_F32 = 0, PR_F16 = 1, PR_BF16 = 2, PR_F64 = 3, PR_I32 = 4, PR_U32 = 5, PR_I64 = 6
} pr_dtype;

/* The combiners of Section 1.1 (set intersection / union are AND / OR on
 * bitset words). */
typedef enum {
    PR_SUM = 0, PR_PROD = 1, PR_MAX = 2, PR_MIN = 3, PR_AND = 4, PR_OR = 5, PR_XOR = 6
} pr_op;

typedef enum {
    PR_OK = 0,
    PR_ERR_INVALID = 1,      /* bad pointer / size / enum / state */
    PR_ERR_UNSUPPORTED = 2,  /* (dtype, op, precision) combination not defined */
    PR_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    PR_ERR_TIMEOUT = 4,      /* a bounded device-side wait ran out */
    PR_ERR_NOMEM = 5         /* workspace allocation failed */
} pr_status;

/* Precision of floating-point SUM (Section 1.1, second footnote: use double
 * precision or Kahan-style compensation to cut the accumulated error).
 *   PLAIN          per-thread fp32 accumulators, fp32 combines (fp64 input: fp64).
 *   COMPENSATED    per-thread fp32 (sum, compensation) pairs, each element added
 *                  with its exact rounding error (TwoSum); pairs combined within
 *                  and across blocks with Neumaier's algorithm in fp32; the final
 *                  s + c rounded once.
 *   FP64_COMBINE   per-thread fp32 accumulators, fp64 warp/block/grid combine. */
typedef enum {
    PR_PREC_PLAIN = 0, PR_PREC_COMPENSATED = 1, PR_PREC_FP64_COMBINE = 2
} pr_precision;

/* Launch configuration of one kernel family (chosen by the autotuner).
 * Plain reductions of at most 64 KiB ignore it: they run as one block of
 * (up to) 1024 threads with two 32-byte vectors a thread, which finishes
 * without the cross-block ticket.
 *   block          threads per block (multiple of 32, 64..1024)
 *   blocks_per_sm  persistent blocks per SM (clamped to the occupancy limit)
 *   unroll         independent accumulators / vectors in flight per thread (1,2,4,8)
 *   vec_bytes      bytes per vector load (16 or 32) */
typedef struct {
    int32_t block;
    int32_t blocks_per_sm;
    int32_t unroll;
    int32_t vec_bytes;
} pr_config;

/* Kernel families with their own configurations: REDUCE (pr_reduce*),
 * SEGMENTED (pr_segmented_reduce*, and rows that do not fit ROWS), BACKWARD
 * (pr_reduce_backward), ROWS (pr_reduce_rows when cols is a whole number of
 * vectors and x is aligned to the vector width; bucketed by rows*cols), AXIS
 * (pr_reduce_axis with inner > 1; bucketed by outer*n*inner: block and
 * blocks_per_sm size the warps in flight, unroll the rows in flight per lane,
 * vec_bytes the column vectors when a row is a whole number of them). */
typedef enum {
    PR_KIND_REDUCE = 0, PR_KIND_SEGMENTED = 1, PR_KIND_BACKWARD = 2, PR_KIND_ROWS = 3, PR_KIND_AXIS = 4
} pr_kind;

/* Line-search methods (pr_line_search). */
typedef enum { PR_SEARCH_GOLDEN = 0, PR_SEARCH_FIBONACCI = 1 } pr_search;

/* Per-segment state that the product's gradient needs. */
typedef struct {
    double p_nz;          /* product of the non-zero elements (as double) */
    int64_t zero_count;   /* number of elements equal to +-0 */
    int64_t first_zero;   /* index (within the segment) of the first zero, -1 if none */
} pr_prod_aux;

/* ---------------------------------------------------------------------- */
/* Plain reduction                                                          */
/* ---------------------------------------------------------------------- */

/* out[0] = x[0] (x) ... (x) x[n-1]                (Section 1.1; Sections 2.3, 3)
 * x: n elements of `dtype` (any alignment of the element type).  n >= 0;
 * x may be NULL only if n == 0.  out: one element of pr_out_dtype(dtype, op).
 * Inputs of 768 MiB and more keep the grid-stride loop for about nine tenths
 * of their vectors; blocks claim the rest in tiles from a counter, so that
 * SMs that stream faster take more of the end.  A tile's partial is stored
 * by tile index and all partials are combined in a fixed order, so the result
 * still depends only on the configuration, n and x's alignment, not on which
 * block took which tile. */
pr_status pr_reduce(const void* x, int64_t n, pr_dtype dtype, pr_op op, void* out,
                    pr_stream_t stream);

/* As pr_reduce, with a precision mode for float SUM and a choice of output
 * type: out_dtype is pr_out_dtype(dtype, op), or PR_F64 for a float SUM under
 * COMPENSATED / FP64_COMBINE (the combined value in fp64, before the final
 * rounding to fp32).  Non-PLAIN precision with any other (dtype, op):
 * PR_ERR_UNSUPPORTED.                          (Section 1.1, second footnote) */
pr_status pr_reduce_ex(const void* x, int64_t n, pr_dtype dtype, pr_op op,
                       pr_precision precision, pr_dtype out_dtype, void* out,
                       pr_stream_t stream);

/* (out[0], idx[0]) = (MAX or MIN of x[0..n), index of its first occurrence):
 * argmax / argmin of a whole array, in one launch like pr_reduce.  Float
 * inputs follow the MAX/MIN rules above (NaN is the extremum, its first
 * occurrence wins; -0 < +0).  out: one element of pr_out_dtype(dtype, op);
 * idx: one int64, -1 for n == 0.  Other ops: PR_ERR_UNSUPPORTED.
 *                         (Section 1.1's combiner on (value, index) pairs) */
pr_status pr_reduce_arg(const void* x, int64_t n, pr_dtype dtype, pr_op op, void* out,
                        int64_t* idx, pr_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Segmented reduction: many independent reductions in one launch           */
/* ---------------------------------------------------------------------- */

/* out[s] = reduction of x[offsets[s] .. offsets[s+1]) for s in [0, nseg).
 * offsets: nseg+1 int64 in device memory, non-decreasing, offsets[0] >= 0 and
 * offsets[nseg] <= the length of x (the caller's contract; checked on the
 * device, a violation sets PR_ERR_INVALID in the device error word and the
 * affected outputs are unspecified).  nseg >= 0.  out: nseg elements of
 * pr_out_dtype(dtype, op).  Empty segments get the identity.
 * The result of each segment is independent of the others' lengths only up to
 * float association order, which is fixed for a fixed configuration.
 *                                             (Section 1.1 applied per segment) */
pr_status pr_segmented_reduce(const void* x, const int64_t* offsets, int64_t nseg,
                              pr_dtype dtype, pr_op op, void* out, pr_stream_t stream);

/* As pr_segmented_reduce, plus optional outputs (pass NULL to skip):
 *   argidx (MAX/MIN only): int64 per segment, index WITHIN the segment of the
 *           first element attaining the extremum (-1 for an empty segment);
 *   aux (PROD, F32/F64 only): pr_prod_aux per segment.
 * precision applies to float SUM as in pr_reduce_ex (out type unchanged). */
pr_status pr_segmented_reduce_aux(const void* x, const int64_t* offsets, int64_t nseg,
                                  pr_dtype dtype, pr_op op, pr_precision precision,
                                  void* out, int64_t* argidx, pr_prod_aux* aux,
                                  pr_stream_t stream);

/* Row reduction of a contiguous row-major [rows, cols] array along its last
 * dimension: segments of equal length without an offsets array.  Outputs as in
 * pr_segmented_reduce_aux, one per row.  rows, cols >= 0. */
pr_status pr_reduce_rows(const void* x, int64_t rows, int64_t cols, pr_dtype dtype, pr_op op,
                         pr_precision precision, void* out, int64_t* argidx,
                         pr_prod_aux* aux, pr_stream_t stream);

/* Reduction along one axis of a contiguous row-major [outer, n, inner] array:
 *   out[p*inner + q] = reduction over i in [0, n) of x[(p*n + i)*inner + q]
 * for p < outer, q < inner (Section 1.1 applied to every column of every
 * [n, inner] slab).  Any single axis of a contiguous tensor of shape S reduces
 * with outer = S[0]*...*S[d-1], n = S[d], inner = S[d+1]*...; inner == 1 is
 * pr_reduce_rows.  Optional outputs as in pr_segmented_reduce_aux, one per
 * output element: argidx (MAX/MIN) is the index i along the axis of the first
 * extremum; aux (PROD, F32/F64) the product state.  n == 0 gives identities.
 * outer, n, inner >= 0 (PR_ERR_INVALID otherwise or when outer*n*inner
 * exceeds 2^62).  x is read, out (outer*inner elements of pr_out_dtype) written;
 * all device memory of the caller.  Shapes with many rows per output use a
 * per-stream partials buffer grown on first use (outside graph capture:
 * PR_ERR_INVALID if a captured call would need to grow it).  The result is
 * deterministic for a fixed configuration. */
pr_status pr_reduce_axis(const void* x, int64_t outer, int64_t n, int64_t inner, pr_dtype dtype,
                         pr_op op, pr_precision precision, void* out, int64_t* argidx,
                         pr_prod_aux* aux, pr_stream_t stream);

/* Prefix scan in one pass (the prefix counterpart of Section 1.1's reduction;
 * the paper names stream compaction and counting / radix sort as its users):
 *   inclusive (exclusive == 0): y[i] = x[0] op x[1] op ... op x[i]
 *   exclusive (exclusive != 0): y[0] = identity, y[i] = x[0] op ... op x[i-1]
 * for the combiners whose result is exact: every integer / bitwise combiner
 * (sums and products wrap in the output type, an I32 sum widens to I64 as in
 * pr_out_dtype) and MAX / MIN of F32, F64, BF16 and F16 (NaN propagates,
 * -0 < +0).  Float SUM / PROD: PR_ERR_UNSUPPORTED.  x: n elements, y: n
 * elements of pr_out_dtype(dtype, op), device memory of the caller, not
 * overlapping.  Bitwise deterministic.  Uses a per-stream tile-state buffer
 * grown on first use (outside graph capture: PR_ERR_INVALID if a captured
 * call would need to grow it).  Every wait is bounded (tile states: 2^18
 * polls; shared-memory barriers: 250 ms): one that runs out (not expected)
 * leaves PR_ERR_TIMEOUT for pr_last_device_error and y unspecified.
 * Alignment: x and y 16-byte aligned take the staged path (bulk copies into
 * shared memory); otherwise every tile is read from x directly. */
pr_status pr_scan(const void* x, int64_t n, pr_dtype dtype, pr_op op, int32_t exclusive, void* y,
                  pr_stream_t stream);

/* Self-check of the bounded waits pr_scan relies on: enqueues, in one
 * thread, a wait of `polls` polls (>= 1; each at least 64 ns after the first
 * 16) on a tile state that nothing publishes (in both status layouts), then
 * a wait of `polls` microseconds on a shared-memory barrier phase that
 * nothing completes.  Each wait gives up and sets PR_ERR_TIMEOUT in the
 * stream's device error word (read it with pr_last_device_error); the
 * context stays usable. */
pr_status pr_check_bounded_wait(int32_t polls, pr_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Line search with the reduction as its inner step                        */
/* ---------------------------------------------------------------------- */

/* The Beckmann objective of BPR link costs along a direction, the function
 * the golden-ratio step of Section 5's traffic assignment minimises (each
 * evaluation one reduction over all links):
 *   phi(alpha) = sum_i t0[i] (v_i + beta cap[i] / (power + 1) (v_i / cap[i])^(power + 1)),
 *   v_i = x[i] + alpha d[i].
 * x (flows), d (direction), t0 (free-flow times), cap (capacities > 0): n
 * float32 each, device memory, 4-byte aligned (16-byte aligned: vector
 * loads).  beta >= 0, power in [1, 16].  Terms are evaluated in float32, a
 * thread's links summed pairwise per point into a Kahan (sum, compensation)
 * pair, then combined in float64 in a fixed order: deterministic.  Error,
 * with u = 2^-24, counted from the operations (first order): each term's
 * linear part t0 v within 3 u, its power part within c u (c = 24 for power
 * 4, else 4 power + 7), the sums within 5 u of sum |term|; so phi is within
 * u (8 sum |t0 v_i| + (c + 5) sum |power part_i|) <= (c + 5) u sum |term|
 * of the exact sum of the exact terms at float32(alpha) and beta.
 *
 * pr_beckmann: out[k] = phi(alphas[k]) for k < m, m in [1, 16], in one pass
 * over the links (alphas and out: device, 8-byte aligned; alphas rounded to
 * float32 for the evaluation).
 *
 * pr_line_search: minimises phi on [lo, hi] (finite, lo < hi).
 *   PR_SEARCH_GOLDEN: golden-section search (points b - r (b - a) and
 *     a + r (b - a), r = (sqrt 5 - 1) / 2) with `count` iterations in
 *     [0, 200] after the first two evaluations: the bracket ends
 *     (hi - lo) r^count wide.
 *   PR_SEARCH_FIBONACCI: Fibonacci search with `count` evaluations in
 *     [3, 78]: points a_j + F_{N-j-1} u and a_j + F_{N-j} u, u = (hi - lo) /
 *     F_N (F_0 = F_1 = 1), the last one a tenth of u from the retained point;
 *     the bracket ends u or 1.1 u wide.
 * Each iteration keeps [a, x2] when phi(x1) < phi(x2), else [x1, b] (ties),
 * and evaluates one new point; the points are placed in float64 with the
 * expressions above evaluated left to right.  `depth` in [1, 3]: one pass
 * over the links evaluates every point the next `depth` iterations could
 * need (2^(depth+1) - 2 of them), so a search costs about count / depth
 * passes; the sequence of points is that of the one-by-one search.  The
 * state lives on the device (a per-stream buffer made on first use, outside
 * graph capture): nothing is synchronised, and result (device, 4 doubles:
 * final a, b, the better of the last two points, its phi) is written by the
 * last kernel of the call.  A search of P passes is P + 1 launches; each
 * pass is launched as a programmatic dependent of the launch before it (it
 * starts streaming links while that one finishes, and waits for it before
 * reading the points it placed), so the link arrays must not be written by
 * other work while a search runs on them. */
pr_status pr_beckmann(const float* x, const float* d, const float* t0, const float* cap, int64_t n, float beta,
                      int32_t power, const double* alphas, int32_t m, double* out, pr_stream_t stream);

/* Golden-section iterations for a tolerance: *count = the smallest K >= 0
 * with (hi - lo) r^K <= tol, r = (sqrt 5 - 1) / 2 (each iteration keeps r of
 * the bracket), evaluated in double as (hi - lo) * pow(r, K).  Host only, no
 * GPU needed.  lo < hi finite, tol > 0 finite; PR_ERR_INVALID otherwise or
 * when K would exceed pr_line_search's limit of 200.  (Golden-section search,
 * one of the reduction's consumers named in Section 1.) */
pr_status pr_golden_iterations(double lo, double hi, double tol, int32_t* count);
pr_status pr_line_search(const float* x, const float* d, const float* t0, const float* cap, int64_t n, float beta,
                         int32_t power, double lo, double hi, pr_search method, int32_t count, int32_t depth,
                         double* result, pr_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Differentiation of a row reduction (F32 and F64)                         */
/* ---------------------------------------------------------------------- */

/* The derivative of Section 1.1's reduction x_0 (x) ... (x) x_{n-1} with
 * respect to each x_i, for the differentiable combiners (the paper gives no
 * gradient: these are the combiners' own partial derivatives, with the
 * derivative of MAX / MIN taken at the first arg-extremum and the product's
 * prod_{j != i} x_j formed from the forward's zero count).
 * grad_in[r, c] = d out[r] / d x[r, c] * grad_out[r]  for a [rows, cols] x:
 *   SUM:      grad_out[r]
 *   MAX/MIN:  grad_out[r] at c == argidx[r] (first arg-extremum), 0 elsewhere
 *   PROD:     zero_count 0: grad_out[r] * p_nz[r] / x[r,c];
 *             zero_count 1: grad_out[r] * p_nz[r] at c == first_zero, 0 elsewhere;
 *             zero_count >= 2: 0
 * x is read only for PROD (may be NULL otherwise); argidx only for MAX/MIN;
 * aux only for PROD (both from pr_reduce_rows).  grad_out: rows elements,
 * grad_in: rows*cols elements, both of `dtype`. */
pr_status pr_reduce_backward(pr_op op, pr_dtype dtype, const void* x, int64_t rows, int64_t cols,
                             const void* grad_out, const int64_t* argidx,
                             const pr_prod_aux* aux, void* grad_in, pr_stream_t stream);

/* Gradient of pr_reduce_axis (the partial derivatives above, for Section
 * 1.1's reduction applied to every column of every [n, inner] slab):
 * grad_in[p, i, q] = d out[p, q] / d x[p, i, q] *
 * grad_out[p, q], with the rules of pr_reduce_backward per output element
 * (argidx / aux as written by pr_reduce_axis).  grad_in: [outer, n, inner];
 * grad_out: [outer, inner]; x read only for PROD.  inner == 1 is
 * pr_reduce_backward.  Status codes as for pr_reduce_backward. */
pr_status pr_reduce_axis_backward(pr_op op, pr_dtype dtype, const void* x, int64_t outer, int64_t n,
                                  int64_t inner, const void* grad_out, const int64_t* argidx,
                                  const pr_prod_aux* aux, void* grad_in, pr_stream_t stream);

/* ---------------------------------------------------------------------- */
/* End to end from host memory                                              */
/* ---------------------------------------------------------------------- */

/* Section 1.1's reduction of a vector held in host memory, with the two
 * stages of Section 2.3 split across chunks: stage 1 reduces each chunk on
 * the device as it arrives, stage 2 combines the chunk partials.
 * host_out[0] = reduction of host_x[0..n): the input is streamed to the device
 * in chunks (copies overlapped with the reduction of the previous chunk) and
 * the result copied back; returns after host_out is written.  host_x should be
 * pinned (cudaHostAlloc / cudaHostRegister) for full copy bandwidth.  Chunk
 * partials are combined in chunk order, so the result is deterministic for a
 * fixed n, but a float SUM may differ in the last bits from pr_reduce. */
pr_status pr_reduce_host(const void* host_x, int64_t n, pr_dtype dtype, pr_op op,
                         void* host_out, pr_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Plain reduction without any library allocation                          */
/* ---------------------------------------------------------------------- */

/* out[0] = x[0] (x) ... (x) x[n-1], like pr_reduce (PLAIN precision), for
 * callers that cannot allocate device memory when they reduce -- code inside
 * a memory pool or arena that owns every allocation, allocation-free
 * real-time paths, or hosts that forbid pr_reduce's implicit first-use
 * workspace allocation.  The paper has no counterpart: this is a deployment
 * variant of the same kernel.  Its scratch (1024 block partials of 64 bytes
 * and a ticket counter, 64.25 KiB) is a static array in device memory that
 * every GPU loading libpr.so holds until the process exits; the entry point
 * calls no cudaMalloc / cudaFree.  The caller passes x and out as for
 * pr_reduce.
 *   - A launch needing more than 1024 block partials is rejected with
 *     PR_ERR_UNSUPPORTED (GB300 uses 304).
 *   - All calls share the one array: calls whose kernels overlap on the GPU
 *     (e.g. on different streams) race; serialise them.
 *   - The first call on a device sets up the array's device address on that
 *     device (so make it before any stream capture); the ticket that must
 *     start at zero is cleared on `stream` before every launch.
 *   - Launch shape is fixed (512 threads, up to 2 blocks per SM, 2 x 32-byte
 *     vectors per thread), so float SUM/PROD bits may differ from pr_reduce's
 *     tuned launch within the same error bounds. */
pr_status pr_reduce_noalloc(const void* x, int64_t n, pr_dtype dtype, pr_op op, void* out,
                            pr_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Failure handling: host-side fault injection (test hook)                   */
/* ---------------------------------------------------------------------- */

/* The paper has no counterpart: this is a hook for testing how failures
 * propagate.  pr_debug_inject_fault arms a one-shot fault at `site`:
 *   PR_FAULT_ALLOC   the library's next device allocation (per-stream
 *                    workspace, axis partials, scan state, line-search state,
 *                    host-pipeline buffers) fails: the entry point returns
 *                    PR_ERR_NOMEM and keeps no partly made state, so a later
 *                    call allocates afresh;
 *   PR_FAULT_LAUNCH  the library's next kernel launch fails: the entry point
 *                    returns PR_ERR_CUDA; launches it made before stay
 *                    enqueued, nothing after is, and no completion ticket is
 *                    left armed (kernels that never start touch none);
 *   PR_FAULT_NONE    disarms.
 * `after` (>= 0) allocations / launches of that site pass first.  The fault
 * is taken on the host before the CUDA call, so no GPU is faulted; argument
 * checks run first, so an invalid call neither fires nor consumes it.
 * *pending (may be NULL) receives 1 if a fault was armed and had not fired.
 * Process-wide; not meant to be armed while other threads use the library. */
typedef enum { PR_FAULT_NONE = 0, PR_FAULT_ALLOC = 1, PR_FAULT_LAUNCH = 2 } pr_fault_site;
pr_status pr_debug_inject_fault(int32_t site, int32_t after, int32_t* pending);

/* The launch that pr_reduce_ex (arg = 0; its configuration for n) or
 * pr_reduce_arg (arg = 1) would make for these arguments on `stream`, without
 * making it: *grid blocks of *block threads (either pointer may be NULL), and
 * *tail_vectors, the vectors of the configuration's width past the
 * grid-stride part that blocks claim in tiles (0: none; may be NULL).  Like
 * the first reduction on a stream, it creates the stream's workspace.  A hook
 * for tests and tuning, with no counterpart in the paper. */
pr_status pr_debug_reduce_plan(const void* x, int64_t n, pr_dtype dtype, pr_op op, pr_precision precision,
                               int32_t arg, pr_stream_t stream, int32_t* grid, int32_t* block,
                               int64_t* tail_vectors);

/* ---------------------------------------------------------------------- */
/* Set-up, status and tuning                                                */
/* ---------------------------------------------------------------------- */

/* Create the workspace for (current device, stream) now, so that later calls
 * on that stream allocate nothing (e.g. before CUDA-graph capture). */
pr_status pr_prepare(pr_stream_t stream);

/* Synchronise `stream`, read and clear its device error word.  *code receives
 * the status recorded by a kernel (PR_OK if none). */
pr_status pr_last_device_error(pr_stream_t stream, int32_t* code);

pr_dtype pr_out_dtype(pr_dtype dtype, pr_op op);
const char* pr_status_string(pr_status status);
/* Detail of the last non-OK status returned on the calling host thread. */
const char* pr_last_error_message(void);
const char* pr_version(void);

/* Configuration used for (kind, dtype, op, precision, n): the tuned entry for
 * n's power-of-two bucket if one exists, else the built-in default. */
pr_status pr_get_config(pr_kind kind, pr_dtype dtype, pr_op op, pr_precision precision,
                        int64_t n, pr_config* cfg);
/* Override the configuration for n's bucket (validated; see pr_config). */
pr_status pr_set_config(pr_kind kind, pr_dtype dtype, pr_op op, pr_precision precision,
                        int64_t n, const pr_config* cfg);
/* Time every candidate configuration on the caller's data (x, n; offsets and
 * nseg for PR_KIND_SEGMENTED; nseg = rows and n = rows*cols, offsets NULL,
 * for PR_KIND_ROWS, which is timed with the outputs the differentiation
 * forward uses; else NULL/0) with CUDA events on `stream`, keep
 * the fastest for n's bucket and return it in *best (may be NULL).  Blocks the
 * host; must not be called during graph capture.  Writes into the library's
 * workspace only. */
pr_status pr_autotune(pr_kind kind, const void* x, int64_t n, const int64_t* offsets,
                      int64_t nseg, pr_dtype dtype, pr_op op, pr_precision precision,
                      pr_stream_t stream, pr_config* best);

/* pr_autotune for PR_KIND_AXIS: x of shape [outer, n, inner] (inner > 1),
 * timed with the outputs the differentiation forward uses (argidx for
 * MAX/MIN, aux for PROD on F32/F64); keeps the winner for outer*n*inner's
 * bucket.  Same blocking and capture rules as pr_autotune. */
pr_status pr_autotune_axis(const void* x, int64_t outer, int64_t n, int64_t inner, pr_dtype dtype,
                           pr_op op, pr_precision precision, pr_stream_t stream, pr_config* best);
/* Persist / restore the tuned table (a small JSON file, keyed by GPU name). */
pr_status pr_tune_save(const char* path);
pr_status pr_tune_load(const char* path);

#ifdef __cplusplus
}
#endif

#endif /* PR_H */
