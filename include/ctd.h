/*
 * ctd.h -- C ABI of the GB300 CTD library (libctd.so).
 *
 * CTD (Lee, Choi, Sael) decomposes a sparse tensor X into C x_alpha (R U):
 *   R  holds actual, linearly independent mode-alpha fibers of X,
 *   U  = (R^T R)^{-1}  (the small pseudoinverse, Lemma 3.2),
 *   C  = X x_alpha R^T, i.e. C_(alpha) = R^T X_(alpha)  (Algorithm 1, Eq. 3).
 * CTD-S (Algorithm 1) does this for a static tensor; CTD-D (Algorithm 2)
 * updates the factors when a new time slice arrives.
 *
 * Conventions for every entry point:
 *  - Tensors are 3-way, in COO form (Section 2.1 "sparse-unordered"):
 *    int32 index vectors i, j, k (0-based) and int32 values.  Coordinates
 *    must be distinct; values may be zero or negative.  (ctd_static_nway
 *    takes tensors of order 1 to 8 with int32 or FP32 values; see there.)
 *  - Mode alpha is 1, 2 or 3 (the paper's 1-based notation).  Column f of
 *    X_(alpha) is the little-endian index over the other two modes
 *    (alpha=1: f = j + J*k; alpha=2: f = i + I*k; alpha=3: f = i + I*j).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    queued on it; entry points that must know a data-dependent size wait
 *    for the stream before they return.  Inputs must stay valid until the
 *    call returns.
 *  - Outputs (ctd_factors) are owned by the library and live in device
 *    memory until ctd_free.  Getters copy into caller-provided HOST buffers
 *    and synchronize.
 *  - No call throws.  Every call returns a ctd_status; on failure
 *    ctd_last_error() gives a message (per thread).  Outputs are left
 *    untouched on failure (for the in-place ctd_dynamic_step, see there).
 *  - Integer work (norms, CDF, draws, dedup, R, C) is exact.  U and the
 *    relative error are computed in FP64; with CTD_FP32_BULK the stored C
 *    values are float (each is an exactly rounded integer).
 *  - Limits: N_alpha < 2^31, I_alpha < 2^31, nnz < 2^31, 1 <= s <= 8192,
 *    1 <= d <= 8192, number of kept fibers <= 24576.  Larger inputs return
 *    CTD_EINVAL.
 */
#ifndef CTD_H
#define CTD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define CTD_API __attribute__((visibility("default")))
#else
#define CTD_API
#endif

typedef enum {
  CTD_OK = 0,
  CTD_EINVAL = 1,     /* bad argument, index out of range, size over a limit */
  CTD_ENOMEM = 2,     /* device allocation failed (host allocation, in a getter) */
  CTD_EOVERFLOW = 3,  /* ||X||_F^2 or an exact product does not fit 64 bits */
  CTD_ECUDA = 4,      /* a CUDA runtime call failed */
  CTD_ETIMEOUT = 5,   /* a bounded device wait gave up */
  CTD_ENOTSUP = 6     /* valid request this build does not handle */
} ctd_status;

typedef enum {
  CTD_FP64 = 0,       /* C stored as double */
  CTD_FP32_BULK = 1   /* C stored as float; U, Gram and filter stay FP64 */
} ctd_precision;

typedef enum {
  CTD_MEM_DEVICE = 0, /* i, j, k, val are device pointers */
  CTD_MEM_HOST = 1    /* host pointers: the library copies them in */
} ctd_memory;

/* Flags for ctd_static. */
#define CTD_SKIP_C 1u      /* do not materialize C (R, U and the error only) */
#define CTD_SKIP_ERROR 2u  /* do not compute the relative error */
/* Also for ctd_dynamic_create: after the matricization (Algorithm 1)
 * sort each column's entries of X_(alpha) by (row, value).  The scatter
 * that builds the columns leaves their entries in the order its atomics
 * were taken, which changes from run to run; integer results (C, R, the
 * Gram matrix, the kept set) are exact in any order, but floating-point
 * sums over a column's entries (the error through Q, W = Q^T X_c of CTD-D)
 * round differently in the last bits.  With this flag every result is
 * bit-identical from run to run, at the cost of the sort: about 0.4 ms per
 * 10^7 nonzeros on GB300, about 10% of a CTD-S call on a 10^7-nonzero
 * traffic tensor. */
#define CTD_DETERMINISTIC 8u
/* For ctd_static: keep the column distribution of the draws (the squared
 * column norms and their prefix sums, Eq. 1) in the factors, where
 * ctd_get_column_dist reads it.  Costs 16 bytes of device memory per
 * column of X_(alpha) for the life of the factors. */
#define CTD_KEEP_DIST 16u

typedef struct {
  int64_t dims[3];     /* I, J, K */
  int64_t nnz;
  const int32_t* i;
  const int32_t* j;
  const int32_t* k;
  const int32_t* val;
  int32_t memory;      /* ctd_memory */
} ctd_coo3;

typedef struct ctd_factors ctd_factors;   /* opaque */

typedef struct {
  int64_t n_rows;      /* I_alpha */
  int64_t n_cols;      /* N_alpha (CTD-D: columns of one slice) */
  int64_t s_draws;     /* s (or d of the last step) */
  int64_t s_unique;    /* s' (or d' of the last step) */
  int64_t s_kept;      /* s~ (CTD-D: d~_t, all steps) */
  int64_t nnz_R;
  int64_t nnz_C;       /* CTD-S: nonzeros of C_(alpha); CTD-D: of all new-column blocks */
  int64_t t_steps;     /* CTD-D: steps taken; CTD-S: 0 */
  int64_t nnz_X;       /* nonzeros of X (CTD-D: all slices so far) */
  double  sqnorm_X;    /* ||X||_F^2 (exact integer, as double) */
} ctd_sizes;

/*
 * ctd_static -- CTD-S, Algorithm 1 (REQUIRE: tensor X, mode alpha, sample
 * size s, tolerance eps; ENSURE: C, U, R).
 *  X        tensor (device or host memory, see ctd_coo3.memory)
 *  alpha    1..3
 *  s        number of draws with replacement, 1..8192
 *  eps      tolerance of the independence test, 0 <= eps < 1;
 *           a fiber x is kept iff ||res|| > eps ||x||
 *  seed     Philox4x64-10 key; draw k uses counter (k, 0, 0, 0)
 *  precision ctd_precision
 *  flags    CTD_SKIP_C | CTD_SKIP_ERROR | CTD_DETERMINISTIC | CTD_KEEP_DIST
 *  out      receives a new ctd_factors (free with ctd_free)
 * Errors: CTD_EINVAL (arguments, index out of range), CTD_EOVERFLOW,
 * CTD_ENOMEM, CTD_ECUDA.  An all-zero tensor gives empty factors and
 * error 0 (no draws).
 */
CTD_API ctd_status ctd_static(const ctd_coo3* X, int alpha, int64_t s, double eps,
                      uint64_t seed, int precision, unsigned flags,
                      void* stream, ctd_factors** out);

/*
 * ctd_static_nway -- CTD-S (Algorithm 1) on an N-way tensor (Section 2.1:
 * Algorithm 1 takes an N-way tensor and a mode alpha; its matricization
 * X_(alpha) has the mode-alpha index as row and the other modes, in
 * little-endian order, as column: f = sum over n != alpha of
 * i_n * prod over m < n, m != alpha of I_m).  Same result as ctd_static on
 * the 3-way tensor I_alpha x N_alpha x 1 with alpha = 1, which is what it
 * runs after mapping every nonzero on the device; the factors' column ids
 * (ctd_get_fibers, the columns of C) are the N-way f above.
 *  X        order N in 1 .. CTD_MAX_ORDER, dims[0 .. N), idx[0 .. N) the index
 *           arrays (int32, 0-based), val the values: int32 counts
 *           (val_type CTD_VAL_INT32) or real values as FP32 (CTD_VAL_FP32);
 *           device or host memory.  Real values take the draws on a
 *           fixed-point grid of the squares (each square rounded down to a
 *           multiple of 2^-32 of the smallest power of two above the
 *           largest square; exact and device-independent; the paper gives
 *           the draws of real values no precision) and FP64 arithmetic after the
 *           draws: R, U and C hold the same values as with integers up to
 *           rounding, the error is FP64, and the dense R/C copies this path
 *           makes need I_alpha * s' < 2^31 (else CTD_ENOTSUP).  CTD-D and
 *           the detector take integer counts only.
 *  alpha    1 .. N
 *  others   as ctd_static
 * Errors as ctd_static; CTD_EINVAL also when N_alpha >= 2^31, an index is
 * outside its mode, or a real value is not finite.
 */
#define CTD_MAX_ORDER 8
#define CTD_VAL_INT32 0
#define CTD_VAL_FP32 1
typedef struct {
  int32_t order;                       /* N */
  int64_t dims[CTD_MAX_ORDER];         /* I_1 .. I_N */
  int64_t nnz;
  const int32_t* idx[CTD_MAX_ORDER];   /* idx[n][e]: mode-(n+1) index of nonzero e */
  const void* val;                     /* int32 counts or FP32 values (val_type) */
  int32_t memory;                      /* ctd_memory */
  int32_t val_type;                    /* CTD_VAL_INT32 or CTD_VAL_FP32 */
} ctd_coon;
CTD_API ctd_status ctd_static_nway(const ctd_coon* X, int alpha, int64_t s, double eps,
                                   uint64_t seed, int precision, unsigned flags, void* stream,
                                   ctd_factors** out);

/*
 * ctd_static_batched -- CTD-S (Algorithm 1) on n independent tensors, each
 * exactly as ctd_static(&X[t], alpha, s[t], eps, seeds[t], precision, flags)
 * would decompose it.  The per-tensor pipelines run concurrently on
 * `workers` library-owned streams (0: 8), largest tensors first, so the
 * host read-backs of one tensor's data-dependent sizes overlap the kernels
 * of the others.  The work is ordered after `stream` and `stream` after
 * the work, as for one launch; the call returns when every tensor is done.
 * out[t] receives tensor t's factors.  On any failure every out[t] is
 * freed and NULL, and the first failing tensor's status is returned.
 */
CTD_API ctd_status ctd_static_batched(int n, const ctd_coo3* X, int alpha, const int64_t* s,
                                      const uint64_t* seeds, double eps, int precision,
                                      unsigned flags, int workers, void* stream,
                                      ctd_factors** out);

/*
 * ctd_dynamic_create -- empty CTD-D state for slices of size
 * dims2[0] x dims2[1] x 1 (Algorithm 2 with alpha in {1, 2}; the time mode
 * is the third).  `stream_id` selects an independent Philox counter space
 * (draw k of step t uses counter (k, t, stream_id, 0)).  flags: 0 keeps the
 * new-column block of every step; CTD_KEEP_LAST_C keeps only the newest
 * step's block (older columns can then no longer be read); CTD_DETERMINISTIC
 * sorts every slice's columns as for ctd_static.
 * Starting empty, the first kept fiber x gives U = 1/(x^T x) as in
 * Algorithm 1, so a first step equals ctd_static on that slice.
 */
#define CTD_KEEP_LAST_C 4u
CTD_API ctd_status ctd_dynamic_create(const int64_t dims2[2], int alpha, int precision,
                                      uint64_t seed, uint64_t stream_id, unsigned flags,
                                      ctd_factors** state);

/*
 * ctd_dynamic_step -- one step of CTD-D, Algorithm 2, in place:
 * (C^(t), U^(t), R^(t)) -> (C^(t+1), U^(t+1), R^(t+1)).
 *  dX   the new slice, dims = {dims2[0], dims2[1], 1}
 *  d    draws for this step, 1..8192
 *  eps  tolerance of the independence test
 * The new columns' block R^(t+1)^T dX is stored exactly; the lower-left
 * block of Eq. (C_t+1_final) is kept as M_{t+1} = ((dR)^T R^(t)) U^(t)
 * (the paper's left-to-right order) and applied to old columns on request.
 * On failure: a step that failed before it changed the state (invalid
 * arguments, an error while reading dX or drawing its columns) leaves the
 * state as it was, and the step may be retried.  A step that failed later
 * (e.g. CTD_ENOMEM while growing R) leaves the state incomplete: every
 * later step and getter on it returns CTD_EINVAL; only ctd_free applies.
 */
CTD_API ctd_status ctd_dynamic_step(ctd_factors* state, const ctd_coo3* dX, int64_t d,
                            double eps, void* stream);

/*
 * Serving loop for CTD-D with continuous batching (no counterpart in the
 * paper beyond Algorithm 2 itself).  A server holds one CTD-D state per
 * stream (stream k uses Philox counter space k), resident on the device.
 * ctd_server_submit queues one slice for one stream; slices of a stream are
 * applied in submission order, slices of different streams run
 * concurrently on `workers` internal CUDA streams (0: 8), each admitted as
 * soon as a worker is free, its stream idle, and the device's free memory
 * (times mem_fraction, less the estimates of running steps) covers its
 * estimate.  dX must stay valid until the request has completed
 * (ctd_server_wait).  ctd_server_result gives {queued, running, total} ms
 * per request.  ctd_server_state lends a stream's state to the getters
 * (do not free it; call after ctd_server_wait).
 */
typedef struct ctd_server ctd_server;
CTD_API ctd_status ctd_server_create(int n_streams, const int64_t dims2[2], int alpha,
                                     int precision, uint64_t seed, int64_t d, double eps,
                                     int workers, double mem_fraction, ctd_server** out);
CTD_API ctd_status ctd_server_submit(ctd_server* S, int stream_id, const ctd_coo3* dX,
                                     int64_t* ticket);
/* Wait for one request (ticket >= 0) or for all submitted so far (ticket < 0). */
CTD_API ctd_status ctd_server_wait(ctd_server* S, int64_t ticket);
CTD_API ctd_status ctd_server_result(ctd_server* S, int64_t ticket, int* status, double ms[3]);
CTD_API ctd_status ctd_server_state(ctd_server* S, int stream_id, ctd_factors** state);
CTD_API void ctd_server_free(ctd_server* S);

/* ctd_error -- relative error of Eq. (error), ||X~ - X||_F^2 / ||X||_F^2
 * (the squared ratio), for the tensor the factors were computed from
 * (CTD-D: all slices so far).  Waits for the work that produced it. */
CTD_API ctd_status ctd_error(const ctd_factors* F, double* rel_err);

/* Sizes; waits for outstanding work on the factors' stream. */
CTD_API ctd_status ctd_get_sizes(const ctd_factors* F, ctd_sizes* out);

/* The s draws I and the s' unique ones I' ascending. */
CTD_API ctd_status ctd_get_samples(const ctd_factors* F, int64_t* I, int64_t* I_unique);

/* Column ids of R's fibers in column order (CTD-D: the slice-local fiber id
 * of each fiber, and in `step` the time step it came from; step may be NULL). */
CTD_API ctd_status ctd_get_fibers(const ctd_factors* F, int64_t* fiber, int64_t* step);

/* R as CSC, I_alpha x s~: colptr[s~+1], row[nnz_R] (ascending within a
 * column), val[nnz_R]. */
CTD_API ctd_status ctd_get_R(const ctd_factors* F, int64_t* colptr, int32_t* row, int32_t* val);

/* U, s~ x s~, row-major (symmetric). */
CTD_API ctd_status ctd_get_U(const ctd_factors* F, double* U);
/* R as ctd_get_R with its values as double: integer counts, or the FP32
 * values of a real-valued tensor (ctd_get_R then returns their bits). */
CTD_API ctd_status ctd_get_R_f64(const ctd_factors* F, int64_t* colptr, int32_t* row,
                                 double* val);

/* Dense columns of C_(alpha): out is s~ x ncols, column-major.
 * CTD-S: cols are column ids of X_(alpha).  CTD-D: column c of step t is
 * t * N_slice + f; rows below the step's own block follow Eq. (C_t+1_final). */
CTD_API ctd_status ctd_get_C_columns(const ctd_factors* F, int64_t ncols, const int64_t* cols,
                             double* out);

/* CTD-S only: C_(alpha) as CSC with rows ascending: colptr[N_alpha+1],
 * row[nnz_C], val[nnz_C]. */
CTD_API ctd_status ctd_get_C(const ctd_factors* F, int64_t* colptr, int32_t* row, double* val);

/*
 * ctd_dynamic_from_static -- a CTD-D state that starts from CTD-S factors of
 * the historical part of a tensor, as in the paper's CTD-D experiments
 * (Sec. 4, "Performance of CTD-D": the first 80% of the time mode is the
 * history, decomposed by CTD-S; later slices arrive one by one).  The
 * tensor of S must have time as mode 3 and S alpha 1 or 2; the state's
 * slices are dims[0] x dims[1].  A fiber f = w + W k of S (W the slice's
 * column count, A1) becomes slice fiber w of time step k.  R is copied;
 * L (Cholesky factor of R^T R) and the orthonormal basis Q come from R's
 * exact Gram matrix and the same orthonormalization as a step's new
 * columns; C of the history is record 0 (ctd_get_step(0) describes the
 * history: d' = s', Delta d~ = s~), so the state's columns are the
 * history's N_alpha columns followed by W per later step.  The next step's
 * draws use counter step = dims[2] (the time index of the slice).
 *  S          CTD-S factors computed with C and the error (no skip flags);
 *             not modified
 *  stream_id, flags   as for ctd_dynamic_create
 *  stream     CUDA stream of the state
 * CTD_EINVAL: NULL arguments, S not CTD-S, alpha 3, or C or the error
 * skipped; CTD_ENOTSUP: R's columns numerically dependent.
 */
CTD_API ctd_status ctd_dynamic_from_static(const ctd_factors* S, uint64_t stream_id,
                                           unsigned flags, void* stream, ctd_factors** state);

/* CTD-D: per-step record.  info = {d', Delta d~, d~_t before the step,
 * nnz of the slice}, sq = {||dX||^2, ||dX - P dX||^2}. */
CTD_API ctd_status ctd_get_step(const ctd_factors* F, int64_t t, int64_t info[4], double sq[2]);

/* CTD-D: M_{t+1} = ((dR)^T R^(t)) U^(t) of step t, row-major
 * (Delta d~ x d~_t). */
CTD_API ctd_status ctd_get_M(const ctd_factors* F, int64_t t, double* M);

CTD_API void ctd_free(ctd_factors* F);

/*
 * ctd_get_column_dist -- the distribution Algorithm 1 draws fibers from
 * (Eq. 1): norm2[f] = ||X_(alpha)(:, f)||^2, the exact integer sum of the
 * squares of column f's values, and cdf[f] = norm2[0] + ... + norm2[f], for
 * the N_alpha columns in the order of A1 (f = j + J k for alpha = 1).  Draw
 * k takes the smallest f with cdf[f] > floor(u_k cdf[N_alpha - 1] / 2^64).
 *  norm2, cdf  host uint64[N_alpha] (either may be NULL)
 * Needs factors from ctd_static called with CTD_KEEP_DIST.  Waits for the
 * factors' stream.  CTD_EINVAL: NULL F, CTD-D factors, or factors made
 * without CTD_KEEP_DIST.
 */
CTD_API ctd_status ctd_get_column_dist(const ctd_factors* F, uint64_t* norm2, uint64_t* cdf);

/*
 * ctd_ddos_candidates -- the online DDoS detector of Section 5 ("CTD at
 * work") on the factor R.  With alpha = 1 (the source mode) each fiber of R
 * is the traffic of one destination: for CTD-D the fiber's slice-local id
 * is the destination index; for CTD-S factors the destination of fiber
 * f = j + J*k is j.  R's fibers are grouped by destination, the first fiber
 * of a destination in R's column order represents it, and a destination is
 * a candidate iff its representative's 2-norm (square root, rounded once, of
 * the column's exact integer sum of squares) exceeds the average norm over
 * all representatives.  The average is the exact sum of the norms rounded
 * once, divided by their count: the result does not depend on any
 * summation order.
 *  cap        entries of dst
 *  dst        host int64[cap] (NULL if cap = 0), receives the first cap
 *             candidates in ascending destination order
 *  n_found    host, receives the number of candidates (may exceed cap)
 *  mean_norm  host or NULL, receives the average
 * Runs on the factors' stream and waits for it.  CTD_EINVAL: NULL F or
 * n_found, cap < 0, dst NULL with cap > 0, or alpha != 1.
 */
CTD_API ctd_status ctd_ddos_candidates(const ctd_factors* F, int64_t cap, int64_t* dst,
                                       int64_t* n_found, double* mean_norm);

/*
 * ctd_sample_noalloc -- the draws I and their unique set I' of ctd_static
 * (same values as ctd_get_samples on ctd_static(X, alpha, s, eps, seed, ...)),
 * without allocating any device memory.  The paper has no counterpart: this
 * is for callers that cannot call cudaMalloc (code running inside another
 * allocator's arena or under a hard memory cap, or latency-critical paths
 * that must not enter the CUDA runtime's allocator).
 *  X         tensor in DEVICE memory (CTD_MEM_HOST is rejected: copying it
 *            in would need a buffer)
 *  draws     device int64[s], receives I;  unique: device int64[s],
 *            receives I' ascending in its first *n_unique entries
 *  n_unique  host int, receives s'
 * When ||X||_F = 0 there is nothing to draw from: every draws[k] is -1 and
 * *n_unique = 0 (ctd_static then reports s_draws = 0 and no samples).
 * Scratch lives in file-scope device arrays of the library, sized for
 * N_alpha <= CTD_NOALLOC_MAX_COLS columns (8 MiB); every GPU that loads the
 * library holds them until the process exits.  Larger N_alpha returns
 * CTD_EINVAL.  The first call on a device looks up the arrays' device
 * addresses for that device (once, with it current).  Every call reads its
 * status back and waits for its stream, so it cannot be called while that
 * stream is being captured into a CUDA graph.  Every call on a device
 * shares the same arrays: calls that overlap on the GPU (other streams,
 * other threads) race, so serialize them.  Errors as ctd_static, including
 * CTD_EOVERFLOW when a column's squared norm or ||X||_F^2 reaches 2^63.
 */
#define CTD_NOALLOC_MAX_COLS (1 << 20)
CTD_API ctd_status ctd_sample_noalloc(const ctd_coo3* X, int alpha, int64_t s, uint64_t seed,
                                      int64_t* draws, int64_t* unique, int* n_unique,
                                      void* stream);

/*
 * ctd_set_allocator -- where the library's device memory comes from (the
 * boundary's memory convention: the factors of Algorithms 1 and 2 and
 * every scratch array of a call).  The paper runs on a CPU and says
 * nothing of it.  With a hook set, every device allocation of the library
 * is alloc(bytes, stream) and is returned with release(ptr, stream); with
 * none (the default, or both NULL) the library uses the device's
 * stream-ordered pool (cudaMallocAsync / cudaFreeAsync).
 *  alloc    returns device memory usable by work enqueued on `stream` from
 *           now on, at least 256-byte aligned, or NULL (the call then
 *           returns CTD_ENOMEM and releases what it held)
 *  release  takes back a block alloc made, in stream order: work already
 *           enqueued on `stream` may still use it, work enqueued later on
 *           that stream may reuse it (the contract of a stream-ordered or
 *           stream-aware caching allocator, e.g. PyTorch's)
 * Both functions may be called from any thread that calls the library and
 * from the library's worker threads (batched and serving forms), with the
 * block's device current.  A block goes back to the functions that made
 * it, even if the hook changed in between.  Process-wide; set it while no
 * call of the library is running.  CTD_EINVAL: exactly one of the two NULL.
 */
typedef void* (*ctd_alloc_fn)(size_t bytes, void* stream);
typedef void (*ctd_release_fn)(void* ptr, void* stream);
CTD_API ctd_status ctd_set_allocator(ctd_alloc_fn alloc, ctd_release_fn release);

/* Device bytes the library holds right now (factors and scratch, from the
 * hook or the pool), as it requested them. */
CTD_API ctd_status ctd_allocated_bytes(size_t* bytes);

/* Launch-shape knobs of the hot kernels (no counterpart in the paper:
 * they change how the work is laid out on the GPU, never the arithmetic or
 * the results), for an autotuner to set per workload.  Keys:
 *   "qform_hot_kb"        shared memory (KB) for the rows of Q staged by the
 *                         error's Q-form (0 to 200; default 200; at most 100
 *                         for kept widths above 512)
 *   "cfill_dense_kb"      shared memory (KB) per block of the C fill's
 *                         multi-nonzero kernel: dense rows of R plus the
 *                         warps' accumulators (64 to 220; default 220)
 *   "copy_blocks_per_sm"  blocks per SM of the C fill's one-nonzero copy
 *                         (1 to 32; default 8)
 * ctd_set_tuning(key, -1) restores the default.  Process-wide; takes effect
 * at the next call.  CTD_EINVAL: unknown key, value out of range, NULL. */
CTD_API ctd_status ctd_set_tuning(const char* key, int64_t value);
CTD_API ctd_status ctd_get_tuning(const char* key, int64_t* value);

/* Diagnostics (no counterpart in the paper).  ctd_profile(1) clears and
 * starts per-phase device timing: each phase of a call is bracketed by a
 * CUDA event pair on the call's stream.  ctd_profile_report waits for the
 * recorded events and writes a JSON object
 *   {"launches": L, "phases": {"name": {"ms": total, "calls": n}, ...}}
 * into buf (NUL-terminated, truncated to len).  L counts every kernel the
 * library launched since the last ctd_profile call. */
CTD_API ctd_status ctd_profile(int enable);
CTD_API ctd_status ctd_profile_report(char* buf, size_t len);

/* Failure-path hooks for tests (no counterpart in the paper).
 * ctd_fault_inject_alloc(n): after n more successful device allocations
 *   every allocation of the library fails with CTD_ENOMEM (-1 disables);
 *   process-wide.  Calls then return CTD_ENOMEM and release what they held.
 * ctd_selftest_bounded_wait(limit, stream): one thread waits, with the wait
 *   of the skip-Cholesky's grid barrier, on a word nothing changes, for at
 *   most `limit` (1 .. 2^24) naps of ~32 ns; it gives up, records the
 *   timeout in the status word and returns CTD_ETIMEOUT, leaving the
 *   context usable.  Waits for the stream. */
CTD_API ctd_status ctd_fault_inject_alloc(int64_t fail_after);
CTD_API ctd_status ctd_selftest_bounded_wait(int64_t spin_limit, void* stream);

/* Self-test of the skip-Cholesky's FP64 inverse square root (no
 * counterpart in the paper): for the n host values d[i] > 0, out[i] = the
 * library's 1/sqrt(d[i]) and ref[i] = CUDA's 1.0 / sqrt(d[i]), both
 * computed on the device.  n in [0, 2^24]; CTD_EINVAL otherwise or on
 * NULL arrays. */
CTD_API ctd_status ctd_selftest_rsqrt(const double* d, int64_t n, double* out, double* ref);

/* Message of the last failing call on this thread ("" if none). */
CTD_API const char* ctd_last_error(void);

/* Library version string. */
CTD_API const char* ctd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CTD_H */
