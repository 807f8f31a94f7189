/*
 * fdsketch.h -- C ABI of the GB300 buffered Frequent Directions library.
 *
 * Method: Desai, Ghashami, Phillips, "Improved Practical Matrix Sketching with
 * Guarantees". A stream of rows a_i in R^d (Sec. 1.1, notation) is summarised
 * by an ell x d sketch B whose covariance B^T B approximates A^T A; the error
 * is cov-err = ||A^T A - B^T B||_2 / ||A||_F^2 (Sec. 1.1, "Error measures").
 * The update is Algorithm 1 (Sec. 2.3) with one of the ReduceRank rules:
 * FD (Sec. 2.3), parameterised FD (Algorithm 2, Sec. 3.1), SpaceSaving
 * Directions (Algorithm 3, Sec. 3.1), iterative SVD (Sec. 2.3) and Fast
 * alpha-FD (Sec. 3.1).
 *
 * Buffered form. The device keeps a working buffer of 2*ell rows (ell for
 * Fast alpha-FD, or the size chosen with fd_create_buffered). When it is
 * full, one reduction runs entirely on the GPU: Gram G = B B^T, symmetric
 * eigensolve G = U diag(sigma^2) U^T, the variant's sigma' (FP64), and the
 * rotate B' = diag(sigma'/sigma) U^T B, which leaves ell-1 rows (t-1 for Fast
 * alpha-FD). The index rules use ell itself (delta = sigma_ell^2 of the
 * buffer: Fast FD, Sec. 2.3). A reduction therefore fires when the buffer is
 * full and then every (buffer rows - rows left) rows, independent of the data.
 *
 * Conventions for every call:
 *  - Return 0 on success or a negative FD_E* code; fd_strerror() names it.
 *    No C++ exception crosses this boundary.
 *  - Row data is row-major; `ld` is the distance in elements between rows
 *    (ld >= d). `dtype` is FD_F32, FD_BF16 (raw bfloat16 bits) or FD_F64.
 *  - `on_device` != 0: the pointer is CUDA device memory. The call is ordered
 *    on the handle's stream; the caller keeps the memory valid until that
 *    stream has passed the call (as with cudaMemcpyAsync).
 *    `on_device` == 0: host memory; the call copies it through pinned staging
 *    before it returns, so the caller may reuse it at once.
 *  - The library owns all device state of a handle; the caller owns every
 *    pointer it passes in.
 *  - Calls on one handle must not overlap from several host threads.
 */
#ifndef FDSKETCH_H_
#define FDSKETCH_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ReduceRank variants. FD: sigma'_j = sqrt(max(sigma_j^2 - delta, 0)),
 * delta = sigma_ell^2 (Sec. 2.3). PFD: the first floor((1-alpha)*ell) values
 * are kept, the rest up to ell shrink by delta = sigma_ell^2, values past ell
 * are zeroed (Algorithm 2). SS: the second-smallest direction's squared value
 * is added to the smallest and the second-smallest is freed, repeated until
 * ell-1 directions remain (Algorithm 3); directions whose mass is below the
 * eigensolve's resolution are freed first and their total mass is added to
 * the smallest retained direction, so the sketch keeps ||A||_F^2.
 * ISVD: sigma'_j = sigma_j for j < ell, else 0 (Sec. 2.3).
 * FAST_PFD (Fast alpha-FD, Sec. 3.1 "Fast Parameterized FD"): the sketch is
 * its own ell-row buffer; delta = sigma_t^2 with t = ell - ell*alpha/2
 * (ell*alpha/2 rounded down, at least 1); the first floor((1-alpha)*ell)
 * values (at most t-1) are kept and the others become
 * sqrt(max(sigma_j^2 - delta, 0)), so a reduction leaves t-1 rows and the next
 * one comes ell-t+1 rows later. Single-sketch handles only (not batched). */
enum { FD_VAR_FD = 0, FD_VAR_PFD = 1, FD_VAR_SS = 2, FD_VAR_ISVD = 3, FD_VAR_FAST_PFD = 4 };

/* Arithmetic of the reduction.
 * FD_PREC_FP32:   FP32 buffer, FP32 CUDA-core Gram and rotate, FP32
 *                 eigensolve (tridiagonal: Householder reduction, bisection
 *                 to relative accuracy, twisted-factorisation vectors,
 *                 Cholesky-QR, then a Rayleigh-Ritz step with the original
 *                 Gram for FD, PFD and iSVD); a flush of a partial buffer is
 *                 solved at the full buffer size with the missing rows zero;
 *                 shrink and bookkeeping in FP64.
 * FD_PREC_BF16X3: buffer held as bfloat16 hi/lo pairs; Gram and rotate on the
 *                 tcgen05 tensor cores as split products hi*hi + hi*lo + lo*hi
 *                 (each K step in a fresh TMEM accumulator, the steps added in
 *                 FP32 registers, the mean shortfall of the MMA's rounding
 *                 toward zero added back); the Gram's diagonal from the FP64
 *                 squared norms of the stored rows; the same FP32 eigensolve;
 *                 FP64 shrink. Its values carry about 2^-16 of rounding per
 *                 reduction. On a stream of 200,000 x 2,000 rows at ell = 100
 *                 (1,979 reductions) its cov-err ends within 1e-6 of the FP64
 *                 run's and its singular values within 1e-4 of them.
 * FD_PREC_FP64:   FP64 buffer, FP64 Gram, rotate and Jacobi (slow; for
 *                 checking against FP64 references). */
enum { FD_PREC_FP32 = 0, FD_PREC_BF16X3 = 1, FD_PREC_FP64 = 2 };

enum { FD_F32 = 0, FD_BF16 = 1, FD_F64 = 2 };

enum {
  FD_OK = 0,
  FD_EINVAL = -1,  /* bad argument: null pointer, d < 1, ell < 2,
                      2*ell > FD_MAX_BUFFER_ROWS, alpha outside (0,1] for PFD,
                      ld < d, unknown enum, precision not built */
  FD_ENOMEM = -2,  /* a device or pinned host allocation failed */
  FD_ECUDA = -3,   /* a CUDA call failed; fd_strerror(FD_ECUDA) gives the text
                      of the last one */
  FD_ENOCONV = -4, /* an eigensolve reached its sweep cap; the result is still
                      written and the count is in fd_stats_t.noconv */
  FD_EBUSY = -5,   /* serving: no room to admit the request now */
  FD_ETOOBIG = -6  /* a size exceeds the fixed workspace of fd_cov_err_noalloc */
};

#define FD_MAX_BUFFER_ROWS 512 /* buffer rows of one sketch (2*ell by default) */

typedef struct fd_state* fd_handle;

typedef struct {
  int64_t d;
  int32_t ell;
  int32_t variant;
  double alpha;
  int32_t prec;
  int32_t pending;        /* rows held in the buffer (ell-1 .. 2*ell-1) */
  int64_t n_seen;         /* rows appended so far */
  int64_t reductions;     /* reductions run by fd_append */
  int64_t noconv;         /* eigensolves that hit the sweep cap */
  double norm_a2;         /* ||A||_F^2 of the rows seen, FP64 */
  double sum_delta;       /* Delta = sum of every delta subtracted (Sec. 3.1) */
  double last_delta;      /* delta of the latest reduction */
  double removed;         /* sum over reductions of sum_j (sigma_j^2 - sigma'_j^2) */
  double max_sweeps;      /* largest Jacobi sweep count seen */
  /* Totals including the final flush reduction of the latest fd_sketch call
   * (equal to the fields above when it had nothing to flush): */
  double sketch_sum_delta;
  double sketch_removed;
  double sketch_norm_b2;  /* ||B||_F^2 of the sketch fd_sketch returned */
  int64_t eig_fallbacks;  /* reductions whose eigenvectors needed the fallback of the
                             tridiagonal solve (nearly dependent vectors of close
                             eigenvalues recomputed by inverse iteration) */
} fd_stats_t;

/* Create a sketch of width d with ell output rows (fd_sketch returns ell x d;
 * the last row is always zero, as in Algorithm 1 a reduced sketch uses at most
 * ell-1 rows). alpha is used by FD_VAR_PFD and FD_VAR_FAST_PFD only. cuda_stream is a
 * cudaStream_t (NULL = the legacy default stream). Allocates all device state. */
int fd_create(int64_t d, int32_t ell, int32_t variant, double alpha, int32_t prec,
              void* cuda_stream, fd_handle* out);

/* fd_create with the buffer size chosen: buffer_rows rows are held before a
 * reduction (fd_create uses 2*ell, and ell for FD_VAR_FAST_PFD). For the
 * other variants 2*ell <= buffer_rows <= FD_MAX_BUFFER_ROWS: delta stays the
 * ell-th squared singular value of the buffer and a reduction leaves ell-1
 * rows, so one reduction handles buffer_rows - ell + 1 new rows (the buffer
 * of Fast FD, Sec. 2.3, taken larger to spread the eigensolve over more rows).
 * FD_VAR_FAST_PFD requires buffer_rows == ell. For the other rules,
 * buffer_rows == ell gives the literal, unbuffered Algorithms 1-3 (Sec. 2.3,
 * Algorithm 2, Algorithm 3): the sketch itself is the ell-row buffer, and a
 * reduction runs whenever an inserted row fills its last zero row, leaving
 * ell-1 rows (one reduction per row once the sketch is full). Any other
 * buffer_rows below 2*ell is FD_EINVAL. */
int fd_create_buffered(int64_t d, int32_t ell, int32_t variant, double alpha, int32_t prec,
                       int32_t buffer_rows, void* cuda_stream, fd_handle* out);

/* Append n rows (Algorithm 1's loop body, "insert a_i", reducing whenever the
 * 2*ell buffer is full). n = 0 is a no-op. Asynchronous for device rows. */
int fd_append(fd_handle h, const void* rows, int64_t n, int64_t ld, int32_t dtype,
              int32_t on_device);

/* Write the sketch B (ell x d, row-major, leading dimension d) to out in
 * `dtype` (FD_F32 or FD_F64). Non-destructive: if more than ell-1 rows are
 * pending, one more reduction with the same index rules runs on a copy (the
 * returned B then includes it; the handle's state is unchanged). For host
 * output the call synchronises the stream. */
int fd_sketch(fd_handle h, void* out, int32_t dtype, int32_t out_on_device);

/* Compensative FD (Sec. 3.1, "Compensative Frequent Directions"): the sketch
 * of fd_sketch, B = S' V^T, with every nonzero singular value replaced by
 * sigma-hat_j = sqrt(sigma'_j^2 + Delta), Delta = sketch_sum_delta (every delta
 * subtracted, the final flush included); V is unchanged and zero rows stay
 * zero. The rows of a reduced sketch are orthogonal with norms sigma'_j, so
 * each nonzero row is scaled by sqrt(1 + Delta / ||b_j||^2) (row norms in
 * FP64); a sketch that never reduced has Delta = 0 and is returned as is.
 * Same output contract as fd_sketch (ell x d, leading dimension d, FD_F32 or
 * FD_F64, non-destructive; host output synchronises the stream).
 * FD_EINVAL for variants other than FD_VAR_FD and FD_VAR_PFD, the ones whose
 * sketch keeps 0 <= x^T (A^T A - B^T B) x <= Delta, which the compensated
 * sketch turns into |x^T (A^T A - B-hat^T B-hat) x| <= Delta. */
int fd_sketch_compensated(fd_handle h, void* out, int32_t dtype, int32_t out_on_device);

/* Merge two sketches of the same width d. The paper states the problem for
 * streams that may be distributed (Sec. 1). src's current sketch (as
 * fd_sketch returns it, taken on a copy: src is unchanged) is appended to dst
 * as ordinary stream rows, up to its last nonzero row, so dst becomes a sketch
 * of the union of both streams. Every later reduction of dst is an ordinary
 * one, so Lemma 1 (Sec. 3.1), applied to both streams, gives
 * 0 <= x^T (A^T A - B^T B) x <= (sum of all deltas) for the union.
 * dst's counters take src's: ||A||_F^2 counts src's rows instead of the
 * appended sketch rows; src's deltas, removed mass, reductions and row count
 * are added. ell, variant and precision may differ (dst's apply).
 * Synchronises both handles' streams. Errors: FD_EINVAL (null, dst == src,
 * different d), FD_ECUDA. */
int fd_merge(fd_handle dst, fd_handle src);

/* fd_merge for a source sketch that lives elsewhere (another process or GPU,
 * a file): the same result as fd_merge(dst, src) when B holds the rows of
 * src's sketch (as fd_sketch returns them, up to its last nonzero row) and
 * *src the counters fd_stats gave for src after that fd_sketch call. This is
 * the exchange step of a stream split across GPUs (Sec. 1, distributed
 * streams): each GPU sketches its part, the rows and counters are gathered,
 * and one GPU folds them in with this call (Lemma 1, Sec. 3.1, then bounds
 * the union by the sum of all deltas).
 * B: rows x d values of `dtype`, row stride ld, device (on_device != 0) or
 * host memory; 0 <= rows <= dst's ell. From *src: d (must equal dst's),
 * n_seen (>= rows), norm_a2 (||A||_F^2 of the source stream, which replaces
 * the squared norms of the appended rows in dst's ||A||_F^2),
 * sketch_sum_delta and sketch_removed (added to dst's Delta and removed
 * mass) and reductions (added). Synchronises dst's stream.
 * Errors: FD_EINVAL (null, size or width mismatch), FD_ECUDA. */
int fd_merge_sketch(fd_handle dst, const void* B, int64_t rows, int64_t ld, int32_t dtype,
                    int32_t on_device, const fd_stats_t* src);

/* cov-err(A, B) = ||A^T A - B^T B||_2 / ||A||_F^2 (Sec. 1.1) for the handle's
 * current sketch B (as fd_sketch returns it) and the n x d matrix A, with
 * ||.||_2 = max |eigenvalue| (Sec. 1.1, the maximum of |(||Ax||^2 - ||Bx||^2)|
 * over unit x). Lanczos with full reorthogonalisation on the GPU; every
 * matrix-vector product streams A once and never forms the d x d matrix.
 * Synchronises the stream; *cov_err receives the value. */
int fd_cov_err(fd_handle h, const void* A, int64_t n, int64_t ld, int32_t dtype,
               int32_t on_device, double* cov_err);

/* proj-err (Sec. 1.1) of the current sketch B (as fd_sketch returns it) for
 * the stream rows A (n x d, leading dimension ld, FD_F32 or FD_F64, on the
 * device or on the host): ||A - pi_{B_k}(A)||_F^2 / ||A - A_k||_F^2, B_k the
 * span of the top k right singular vectors of B (fewer if B has lower rank),
 * A_k the best rank-k approximation of A. Numerator: ||A||_F^2 minus
 * sum_j ||A v_j||^2, the v_j from an FP64 eigensolve of B B^T and one pass over
 * A. Denominator: ||A||_F^2 minus the k largest eigenvalues of A^T A, found by
 * Lanczos with full reorthogonalisation that streams A (never forms d x d) and
 * stops when each carries a residual bound below 1e-10 ||A||_F^2. Returns 1.0
 * when both are zero. 1 <= k < ell, else FD_EINVAL. Allocates its workspace
 * and synchronises the handle's stream. */
int fd_proj_err(fd_handle h, const void* A, int64_t n, int64_t ld, int32_t dtype,
                int32_t on_device, int32_t k, double* proj_err);

/* Same evaluator for a caller-given sketch B (rows x d, row-major FP32/FP64
 * per dtype, leading dimension d), without a handle. stream may be NULL. */
int fd_cov_err_pair(const void* A, int64_t n, int64_t d, int64_t lda, int32_t a_dtype,
                    const void* B, int64_t rows, int32_t b_dtype, int32_t on_device,
                    void* cuda_stream, double* cov_err, double* lambda_min,
                    double* lambda_max);

/* The covariance-error evaluator of fd_cov_err_pair for callers that cannot
 * allocate device memory: code that runs inside a custom device allocator or
 * a memory-pool callback (a nested cudaMalloc would re-enter it), runtimes
 * that account for every byte of device memory themselves, and servers that
 * forbid allocation once they are up. The paper has no counterpart; this is
 * a deployment variant of the evaluator.
 *
 * A (n x d, row stride lda) and B (rows x d, contiguous) are device pointers
 * (FP32 or FP64 per dtype); *cov_err (host) receives the value. No device or
 * pinned memory is allocated: every intermediate vector lives in one
 * file-scope device array of about 4.6 MB, which each GPU that loads the
 * library keeps until the process exits. Limits: d <= FD_NOALLOC_MAX_D,
 * rows <= FD_NOALLOC_MAX_B_ROWS, at most FD_NOALLOC_MAX_STEPS Lanczos steps
 * (the value is then the estimate after that many steps); larger sizes return
 * FD_ETOOBIG. The first call on a device looks up the array's device address
 * (make it before any stream capture). Every call shares the array and clears
 * it first, so calls that overlap on the GPU (several streams or threads at
 * once) race: serialise them. Synchronises `cuda_stream`. */
#define FD_NOALLOC_MAX_D 1024
#define FD_NOALLOC_MAX_B_ROWS 512
#define FD_NOALLOC_MAX_STEPS 256
int fd_cov_err_noalloc(const void* A, int64_t n, int64_t d, int64_t lda, int32_t a_dtype,
                       const void* B, int64_t rows, int32_t b_dtype, void* cuda_stream,
                       double* cov_err);

/* Counters of the handle (synchronises the stream). */
int fd_stats(fd_handle h, fd_stats_t* s);

/* Record the spectrum of every reduction fd_append runs from now on (on != 0)
 * or stop (on = 0; the default). While recording, the eigensolve computes
 * every eigenvalue; otherwise the variants other than SS compute only the
 * ell+1 largest, the only ones their ReduceRank rule keeps. */
int fd_record_spectrum(fd_handle h, int32_t on);

/* Spectrum of the latest reduction run by fd_append while recording:
 * sigma^2 (descending, one value per buffer row: 2*ell, or the buffer_rows
 * of fd_create_buffered) and sigma'^2 aligned with it, FP64, host arrays of
 * that length. FD_EINVAL when not recording. */
int fd_last_spectrum(fd_handle h, double* sigma2, double* sigma_prime2);

/* Return the handle to its just-created state (empty buffer, zero counters)
 * while keeping its allocations; ordered on the handle's stream. */
int fd_reset(fd_handle h);

/* Device-time accounting per kernel class. fd_profile(h, 1) starts bracketing
 * every launch of the handle with CUDA events on its stream (and clears the
 * totals); fd_profile(h, 0) stops. fd_kernel_times synchronises the stream and
 * fills counts[c] (launches) and ms[c] (summed device milliseconds) for the
 * classes c < FD_KCLASSES: ingest, Gram, eigensolve + shrink, rotate. */
#define FD_KCLASSES 4
enum { FD_K_INGEST = 0, FD_K_GRAM = 1, FD_K_EIG = 2, FD_K_ROTATE = 3 };
int fd_profile(fd_handle h, int32_t enable);
int fd_kernel_times(fd_handle h, int64_t* counts, double* ms);

/* Release every resource of the handle (synchronises its stream). */
int fd_destroy(fd_handle h);

/* ---- Batched sketches --------------------------------------------------
 * Many independent sketches (each with its own d and ell, 2*ell <= 128) that
 * share one variant and are updated together: one fd_batch_append call runs a
 * single persistent launch in which every CTA takes work items (a sketch and a
 * block of its rows) from a device queue ordered longest-first and runs the
 * whole block through the buffered update of that sketch (ingest, Gram,
 * eigensolve, ReduceRank, rotate) without leaving the CTA. Per sketch the
 * arithmetic is that of a single handle with FD_PREC_FP32 (FP32 Gram,
 * tridiagonal eigensolve of a full buffer and rotate, FP64 ReduceRank), and
 * its results agree with one within rounding; the batched rotate also scales
 * each new row to its FP64 norm sigma'_j. */
typedef struct fd_batch_state* fd_batch;
typedef struct {
  int32_t id;        /* sketch index, 0 <= id < count; at most once per call */
  int32_t dtype;     /* FD_F32, FD_BF16 or FD_F64 */
  const void* rows;  /* device pointer, n rows of d_id values, row stride ld */
  int64_t n;
  int64_t ld;
} fd_work_t;

int fd_batch_create(int32_t count, const int64_t* d, const int32_t* ell, int32_t variant,
                    double alpha, int32_t prec, void* cuda_stream, fd_batch* out);
/* Append row blocks to sketches; asynchronous on the batch's stream. The
 * append is a CUDA graph (the queue reset and the persistent launch, captured
 * on the first call and relaunched for every call); only the item table and
 * its length are copied in before each launch, from pinned host memory. The
 * call waits for the previous call's item copy (not its kernel) before it
 * refills that memory. If the graph cannot be built, appends launch directly. */
int fd_batch_append(fd_batch b, const fd_work_t* items, int32_t n_items);
/* 1 if appends run as the CUDA graph, 0 if they launch directly (FD_EINVAL for
 * a null batch); *launches (optional) receives the graph launches so far. */
int fd_batch_uses_graph(fd_batch b, int64_t* launches);
/* Sketch `id` as ell_id x d_id rows (same flush rule as fd_sketch). */
int fd_batch_sketch(fd_batch b, int32_t id, void* out, int32_t dtype, int32_t out_on_device);
/* Every sketch at once, into one device buffer of FP32: sketch id is written
 * as ell_id x d_id rows (leading dimension d_id) at out + offsets[id]
 * (offsets: host array of count element offsets). Same flush rule as
 * fd_sketch; one launch, asynchronous on the batch's stream. */
int fd_batch_sketch_all(fd_batch b, float* out, const int64_t* offsets);
int fd_batch_stats(fd_batch b, int32_t id, fd_stats_t* s);
int fd_batch_reset(fd_batch b);
int fd_batch_destroy(fd_batch b);

/* ---- Serving: continuous batching of append requests --------------------
 * A request loop over `count` live sketches of one shape (d, ell). A request
 * (sketch id, n host rows of d FP32 values) is admitted when it fits the
 * device-memory budget (budget_bytes of pinned host plus device staging);
 * otherwise fd_serve_submit returns FD_EBUSY and the caller retries. A native
 * engine thread launches one batched update (the fd_batch kernel) over every
 * admitted request whose sketch is not already on the GPU, on the next of
 * `streams` streams, so launches overlap on the device while each sketch is
 * in at most one launch; requests of one sketch are applied in submit order.
 * Per sketch the result is that of fd_append of the same rows in that order.
 * The paper has no serving layer; the arithmetic is Algorithm 1's. */
typedef struct fd_server_state* fd_server;
int fd_serve_create(int32_t count, int64_t d, int32_t ell, int32_t variant, double alpha,
                    int64_t budget_bytes, int32_t streams, fd_server* out);
/* Copies the rows (row stride d) into staging before returning. */
int fd_serve_submit(fd_server s, int32_t id, const float* rows, int64_t n, int64_t* ticket);
/* Up to `max` completed requests since the last poll: tickets and their
 * latency in seconds (submit to completion seen by the engine). */
int fd_serve_poll(fd_server s, int64_t* tickets, double* latency_s, int32_t max, int32_t* count);
int fd_serve_drain(fd_server s);
/* Sketch `id` (ell x d, host out) after every submitted request is done. */
int fd_serve_sketch(fd_server s, int32_t id, void* out, int32_t dtype);
int fd_serve_counters(fd_server s, int64_t* admitted, int64_t* busy, int64_t* launches,
                      int64_t* rows_done);
int fd_serve_destroy(fd_server s);

/* Text for an FD_E* code (static storage). */
const char* fd_strerror(int32_t code);

/* Library version and the sm architecture it was built for. */
const char* fd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FDSKETCH_H_ */
