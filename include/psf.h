/*
 * psf.h -- C ABI of the GB300 (sm_103a) evaluator for near-sparse matrix
 * power series f(Z) = sum_i a_i Z^i by the Paterson-Stockmeyer scheme
 * combined with filtering (PSSCF), after Wu, Zhu, Zhao and Zhang, "A filtering
 * technique for the matrix power series being near-sparse".
 *
 * Conventions for every entry point:
 *  - Return value: PSF_OK (0) or one of the PSF_E* codes below; the message
 *    of the last failure on the calling thread is psf_last_error().  No C++
 *    exception or abort crosses this boundary.
 *  - Matrices are square CSR (psf_csr_t) in DEVICE memory: 0-based int32
 *    row pointers (n + 1) and column indices, FP64 values, columns strictly
 *    increasing within a row, finite values.  The library never writes to an
 *    input matrix.  An input must stay valid until the work enqueued on the
 *    stream has finished.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it; an entry point returns after the
 *    host-side decisions it needs (it may synchronize the stream, as stated
 *    per entry point).
 *  - Results (psf_result_t) own library-allocated device memory, released by
 *    psf_result_destroy() on the stream they were produced on, which must
 *    still exist at that point.
 *  - All arithmetic is IEEE FP64.  Products fold terms in a fixed order (see
 *    psf_product_filter) and matrix 1-norms use exactly rounded column sums,
 *    so results do not depend on thread scheduling.
 */
#ifndef PSF_H
#define PSF_H

#include <stdint.h>

#if defined(__GNUC__)
#define PSF_API __attribute__((visibility("default")))
#else
#define PSF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define PSF_OK 0
#define PSF_EINVAL 1    /* bad argument or malformed CSR input */
#define PSF_ENOMEM 2    /* device or host allocation failed */
#define PSF_ECUDA 3     /* a CUDA runtime call failed */
#define PSF_ENOTCONV 4  /* Theta found no truncation length within the coefficients
                           (Eq. 34), or Algorithm 1 reached its pass cap */
#define PSF_ETIMEOUT 5  /* a bounded device-side wait expired */
#define PSF_ETOOBIG 6   /* a size exceeds a documented limit (e.g. nnz >= 2^31) */
#define PSF_ECANCELED 7 /* a server request was cancelled before it was admitted */

/* ---- series flags (psf_series_create) ---- */
#define PSF_SERIES 0u        /* power series: N from Eq. (34), thresholds Eq. (36) */
#define PSF_POLY 1u          /* polynomial of the m given coefficients, thresholds Eq. (28) */
#define PSF_NOFILTER 2u      /* unfiltered PS scheme (every threshold 0) */
#define PSF_Z_SUBMULT 4u     /* z_i = ||Z||^i (Sec. 2.2) instead of exact ||Z^i||, i <= 10 */
/* PSF_Z_ESTIMATE: z_1 = ||Z||_1 exact and z_i, i = 2..10, from a deterministic
 * estimator instead of the exact norms of the powers (Sec. 3.2.2, Eq. 37:
 * the paper's normest1, here its single-vector core -- Hager's power
 * iteration with Higham's stopping rules and alternating test vector, at
 * most five products with Z^i; every product a fixed fma order, every sum
 * exact).  Cheaper than the powers Z^2..Z^10; the estimates are lower
 * bounds.  A column of Z with more than 4096 entries falls back to the exact
 * norms.  Not with PSF_Z_SUBMULT; psf_eval only (psf_eval_batch rejects it). */
#define PSF_Z_ESTIMATE 8u
/* PSF_Z_SQUARE: for a series with only even powers (cos, cosh) or only odd
 * powers (sin, sinh), run Algorithm 2 on W = Z^2 (an adjacent variant; the
 * paper evaluates cos with its zero odd coefficients in place, Eq. 40).
 * Even: f(Z) = g(W), g's coefficients c_k = a_{2k}.  Odd: f(Z) = Z g(W),
 * c_k = a_{2k+1}, g evaluated to tol / ||Z||_1 and the last product Z G
 * unfiltered (||Z (g(W) - G)||_1 <= ||Z||_1 ||g(W) - G||_1).  W = Z Z is
 * unfiltered; the norms of W's powers are z_{2i} of Z (Eq. 37 and Lemma 1 for
 * Z, or the PSF_Z_SUBMULT / PSF_Z_ESTIMATE variants).  The plan fields N, q,
 * b, g, trunc, budget and the thresholds are those of g in W; z[] and
 * alpha10 stay those of Z.  psf_series_create fails with PSF_EINVAL when
 * both parities have nonzero coefficients.  psf_eval, psf_eval_batch and
 * the server accept it; their results are bitwise the same. */
#define PSF_Z_SQUARE 16u

/* ---- tunable parameters (psf_series_set_param) ---- */
#define PSF_PARAM_ER 1            /* e_r of Algorithm 1 (default 0.1) */
#define PSF_PARAM_ALG1_MAXIT 2    /* cap on Algorithm 1 passes (default 1000) */
#define PSF_PARAM_POOL_ENTRIES 3  /* initial entry capacity of an evaluation's pool (0 = auto) */
#define PSF_PARAM_KERNEL 4        /* product slot map: 0 auto, 1 column table, 2 bitmap,
                                     3 bitmap with the wide column window for every product
                                     (auto picks it for a step whose rows spanned more than
                                     4608 columns in the series' previous evaluation),
                                     4 one row per block of four warps (shared bitmap map,
                                     2560 accumulator slots) for every product */
#define PSF_PARAM_CHUNK_COLS 5    /* > 0: fewer columns per row chunk (tests of row chunking) */
#define PSF_PARAM_CHUNK_SLOTS 6   /* > 0: fewer accumulator slots per row chunk (same) */
#define PSF_PARAM_DENSE_XOVER 7   /* dense-tile crossover of this series (see PSF_TUNE_DENSE_XOVER):
                                     a giant step with at least this many algorithmic
                                     multiply-adds per n^3 in the previous evaluation, n >= 512,
                                     runs as FP64 dense tiles (0: every product step, any n;
                                     1e300: none; -1, the default: the process-wide value) */

#define PSF_MAX_Q 23 /* largest supported PS block size q */

typedef struct psf_series_s* psf_series_t;
typedef struct psf_result_s* psf_result_t;

typedef struct {
    int32_t n;             /* rows = columns */
    int32_t nnz;           /* stored entries = rowptr[n] */
    const int32_t* rowptr; /* device, n + 1 */
    const int32_t* col;    /* device, nnz */
    const double* val;     /* device, nnz */
} psf_csr_t;

/* Plan of one evaluation (Alg. 2 steps 1-3 and the thresholds). */
typedef struct {
    int32_t N;          /* truncation length (Eq. 34) or m (polynomial) */
    int32_t q, b, g;    /* PS split (Eq. 6) */
    int32_t products;   /* matrix products in the PS phase (Eq. 5); with PSF_Z_SQUARE
                           also W = Z Z and, for an odd series, Z G */
    int32_t nsteps;     /* entries available through psf_result_step */
    double z[11];       /* ||Z^i||_1 (or ||Z||^i), i = 0..10 (Eq. 37) */
    double alpha10;     /* Lemma 1 growth factor */
    double trunc;       /* truncation bound sum_{i>=N} |a_i| z_i (0 for polynomials) */
    double budget;      /* filtering budget: tol - trunc (Eq. 35) or tol (Eq. 27) */
    int64_t nnz;        /* entries of the result */
    int64_t fma;        /* multiply-adds the product kernel executed in the evaluation
                           (norm powers included): sum over output rows r of
                           sum_{k in A_r} nnz(B_k) plus the addend entries; a baby
                           step equal to a power already computed (nothing dropped
                           before it) is not executed again and not counted here,
                           its step record still lists its product's count */
} psf_info_t;

/* Statistics of one filtered product of Algorithm 2 (a baby step, Eq. 11, or a giant step, Eq. 14). */
typedef struct {
    int32_t kind;       /* 0 baby step (Eq. 11), 1 giant step (Eq. 14), 2 plain add,
                           3 the unfiltered F = Z G of an odd series (PSF_Z_SQUARE) */
    int32_t index;      /* k of Z-hat_(k), or i of S-hat_i */
    double threshold;   /* bound on the dropped 1-norm (zeta_k or sigma_i; 0 = none) */
    int64_t nnz_pre;    /* nonzero entries before the filter */
    int64_t nnz_post;   /* entries kept */
    double eps_f;       /* final entry threshold of Algorithm 1 */
    int32_t iters;      /* Algorithm 1 passes */
    double dropped;     /* exact 1-norm of the dropped entries */
    int64_t fma;        /* algorithmic multiply-adds of this step */
} psf_step_info_t;

/* Library version, (major << 16) | minor. */
PSF_API int psf_version(void);

/* Thread-local message of the last failure on this thread ("" if none). */
PSF_API const char* psf_last_error(void);

/*
 * Create a series object from coefficients a_0..a_{m-1} (host memory, copied).
 *   s     > 0 overrides the PS block size q (Eq. 6 uses q = floor(sqrt(N-1))),
 *         clamped to N-1; must be <= PSF_MAX_Q.
 *   tol   eps_tol > 0: the target bound on ||f(Z) - result||_1 (Alg. 2), or the
 *         filtering budget eps of Eq. (27) for PSF_POLY.
 *   flags PSF_SERIES or PSF_POLY, optionally | PSF_NOFILTER | PSF_Z_SUBMULT
 *         (or PSF_Z_ESTIMATE) | PSF_Z_SQUARE.
 * In series mode the coefficients past a_{m-1} are taken as 0; supply enough
 * terms for the tail sum of Eq. (34) to fall below tol/2 before the last one.
 * Errors: PSF_EINVAL (m < 1, tol not finite and > 0, non-finite a_i, unknown
 * flags, PSF_Z_SUBMULT with PSF_Z_ESTIMATE, PSF_Z_SQUARE with coefficients of
 * both parities), PSF_ENOMEM.
 */
PSF_API int psf_series_create(const double* coeffs, int64_t m, int32_t s, double tol, uint32_t flags,
                      psf_series_t* out);

/* Set a PSF_PARAM_* value.  Not safe concurrently with psf_eval on the same
 * series.  Errors: PSF_EINVAL (unknown key, out-of-range value). */
PSF_API int psf_series_set_param(psf_series_t series, int32_t key, double value);

PSF_API int psf_series_destroy(psf_series_t series);

/*
 * Evaluate the series at Z (Algorithm 2): exact ||Z^i||_1 for i <= 10, the
 * plan (Eqs. 6, 24-26, 34-37), baby steps Z-hat_(k+1) = filter(Z Z-hat_(k))
 * and giant steps S-hat_i = filter(B-hat_{b-1-i} + Z-hat_(q) S-hat_{i-1}) with
 * Algorithm 1 after every product.  Synchronizes `stream` three times (input
 * validation; after the norms, to plan; at the end, to size the result).
 * What the host reads at those points is written by a kernel into pinned,
 * device-mapped host memory (kept by the library, a few 64 KB buffers for
 * the life of the process), not copied by a copy engine: a large
 * device-to-host copy on another stream, such as the previous result's
 * psf_result_copy, does not delay the evaluation.
 * The result CSR is canonical (sorted columns, no stored zeros).
 * The series records sizes seen by the evaluation (pool entries, row
 * lengths) and sizes the next evaluation's workspace from them; from its
 * second evaluation on, one pool holds both phases and baby steps reuse the
 * powers of the norm phase while no entry has been dropped.  Results do not
 * depend on these records.  Evaluations of one series must not run
 * concurrently (they update the records); distinct series may.
 * Errors: PSF_EINVAL (malformed Z), PSF_ENOTCONV, PSF_ENOMEM, PSF_ECUDA,
 * PSF_ETIMEOUT, PSF_ETOOBIG.
 */
PSF_API int psf_eval(psf_series_t series, const psf_csr_t* Z, void* stream, psf_result_t* out);

/*
 * psf_eval on a matrix given in HOST memory (Z's arrays on the host; pinned
 * memory makes the copies asynchronous): Z is copied into device memory on
 * `stream`, evaluated, and its copy released after the evaluation's work.
 * With psf_result_copy into host arrays this is the whole host-to-host
 * path.  Same errors as psf_eval.
 */
PSF_API int psf_eval_from_host(psf_series_t series, const psf_csr_t* Z, void* stream, psf_result_t* out);

/*
 * Evaluate `count` independent instances Zs[i] (each square, any size n_i)
 * with series[i] (Algorithm 2 each).  The instances are laid out as one
 * block-diagonal matrix, so every stage (each of Z^2..Z^10, each baby step,
 * S_0, each giant step) of all instances runs as one launch of the product
 * kernel and, where filtered, one launch of the Algorithm 1 kernel; the
 * number of launches depends on the largest q_i and b_i, not on `count`.
 * Instances differ per stage only in small device tables (what the stage
 * does to the instance, its coefficients and Algorithm 1 threshold).
 * Results are bitwise identical to psf_eval on each instance, whatever else
 * is in the batch; outs[i] receives instance i's result (all results of a
 * batch share one device allocation, released with the last of them).
 * Slot-map and chunking parameters are taken from series[0].
 * Synchronizes `stream` three times (validation, norms, result sizes).
 * Instances are processed in groups of at most 1024 instances and 2^24 rows.
 * Errors: any instance's error fails the whole call (outs[i] all NULL);
 * the message names the instance where it is known.
 */
PSF_API int psf_eval_batch(const psf_series_t* series, const psf_csr_t* Zs, int32_t count, void* stream,
                   psf_result_t* outs);

/*
 * Serving loop with continuous batching (no counterpart in the paper, which
 * evaluates one matrix at a time).
 *
 * `workers` host threads each own a CUDA stream.  A worker that is free
 * admits the oldest waiting requests, as many as fit both `max_batch` and
 * the device-memory budget (each request's footprint is predicted from its
 * n and nnz), and evaluates them together as one psf_eval_batch on its
 * stream.  Requests that arrive while other batches are running are admitted
 * by the next free worker as soon as memory allows, so their work overlaps
 * on the device with the batches in flight.  A request that would not fit
 * the budget even alone is admitted when nothing else is in flight.  If a
 * batch fails, its requests are evaluated again one by one, so a bad request
 * fails alone.  Results are bitwise identical to psf_eval.
 *
 * psf_server_submit: Z (device CSR) must stay valid, and neither the series
 *   nor Z may be changed or destroyed, until the request's completion has been
 *   polled.  `tag` is returned with the completion.  Thread-safe.
 * psf_server_poll: up to `max` completions, waiting up to `wait_ms` (-1:
 *   until at least one is available or nothing is pending) for the first;
 *   *got receives the number returned.  Each completion owns its result
 *   (destroy it with psf_result_destroy before psf_server_destroy).
 * psf_server_destroy: waits for the requests in flight and drops the
 *   completions not polled (their results are destroyed).
 * Errors: PSF_EINVAL (null arguments, more than 64 workers, max_batch above
 * 1024, a PSF_Z_ESTIMATE series or a malformed Z size on submit), PSF_ENOMEM,
 * PSF_ECUDA.  A request's own failure is its completion's status.
 */
typedef struct psf_server_s* psf_server_t;

typedef struct {
    int32_t workers;      /* host threads = concurrent batches (default 4) */
    int32_t max_batch;    /* requests per batch (default 64, <= 1024) */
    int64_t hbm_budget;   /* bytes of device memory for requests in flight (0: half the free memory) */
} psf_server_config_t;

typedef struct {
    uint64_t tag;         /* as submitted */
    int32_t status;       /* PSF_OK or the request's error code */
    int32_t batch_size;   /* requests evaluated together with this one (itself included) */
    psf_result_t result;  /* NULL unless status == PSF_OK */
    double queue_ms;      /* submit -> admission */
    double latency_ms;    /* submit -> result available */
} psf_completion_t;

typedef struct {
    int64_t submitted, completed, failed, batches;
    int32_t max_concurrent;  /* most batches in flight at once */
    int32_t pending;         /* waiting for admission */
    int64_t budget_peak;     /* most predicted bytes in flight at once */
    int64_t cancelled;       /* withdrawn by psf_server_cancel (counted in completed) */
} psf_server_stats_t;

PSF_API int psf_server_create(const psf_server_config_t* config, psf_server_t* out);
PSF_API int psf_server_submit(psf_server_t server, psf_series_t series, const psf_csr_t* Z, uint64_t tag);
PSF_API int psf_server_poll(psf_server_t server, psf_completion_t* out, int32_t max, int32_t wait_ms,
                            int32_t* got);
PSF_API int psf_server_stats(psf_server_t server, psf_server_stats_t* stats);
/* psf_server_cancel: withdraw the oldest request with this tag that is still
 * waiting for admission.  *cancelled receives 1 if one was withdrawn (it
 * then completes at once with status PSF_ECANCELED and no result, so every
 * submit still gives one completion, and its memory no longer counts
 * against the budget) and 0 if no waiting request has the tag (unknown, or
 * already admitted: an admitted request runs to completion).  Thread-safe.
 * Errors: PSF_EINVAL (null arguments). */
PSF_API int psf_server_cancel(psf_server_t server, uint64_t tag, int32_t* cancelled);
PSF_API int psf_server_destroy(psf_server_t server);

/*
 * One filtered product, the building block of every PS step:
 *   C = sum_{t < nadd} alphas[t] * M_t  +  A * B,   then Algorithm 1.
 * addends[t] == NULL means M_t = I.  A and B may both be NULL (a pure
 * weighted sum).  Rounding order of each output entry c_rj: start from 0,
 * fold the addends in order t = 0, 1, ... as c = fma(alpha_t, m_rj, c), then
 * for each k of A's row r in ascending column order c = fma(a_rk, b_kj, c).
 * Entries that are exactly 0 are not stored.  threshold > 0 runs Algorithm 1
 * with eps_g = threshold / (1 + e_r), so the dropped 1-norm is <= threshold;
 * threshold == 0 keeps every nonzero entry.  Synchronizes `stream` once.
 * Limits: nadd <= PSF_MAX_Q + 1.
 * Errors: PSF_EINVAL (malformed or mismatched matrices, nadd out of range,
 * a threshold that is negative or not finite),
 * PSF_ENOTCONV (Algorithm 1 reached maxit passes), PSF_ETOOBIG (the product
 * needs more than 2^31 - 2^20 pool entries), PSF_ENOMEM, PSF_ECUDA.
 */
PSF_API int psf_product_filter(const psf_csr_t* A, const psf_csr_t* B, int32_t nadd, const double* alphas,
                       const psf_csr_t* const* addends, double threshold, double e_r,
                       int32_t maxit, void* stream, psf_result_t* out);

/* ||M||_1 with exactly rounded column sums; synchronizes `stream`. */
PSF_API int psf_norm1(const psf_csr_t* M, void* stream, double* out);

/*
 * psf_norm1_noalloc: the same exact ||M||_1 as psf_norm1 (bit for bit),
 * computed without allocating any memory.  The paper has no counterpart: it
 * is an operational variant for callers that must not allocate, e.g. a
 * serving loop whose device memory is already committed to admitted
 * requests (an allocation could fail or evict them), or code that overlaps
 * work on other streams and cannot afford the device-wide synchronisation
 * that freeing device memory implies.
 *
 * Instead of a workspace per call, it uses one scratch region compiled into
 * the library: a static device array of 4,456,960 bytes (4.25 MiB) holding
 * the fixed-point column sums of PSF_NORM1_NOALLOC_MAX_N columns and a
 * control block, which every device that loads the library keeps until the
 * process exits.  It reads M's entries in place.
 *  - M: device CSR, n <= PSF_NORM1_NOALLOC_MAX_N (else PSF_ETOOBIG, nothing
 *    is launched); malformed input gives PSF_EINVAL as for psf_norm1.
 *  - out: host pointer, receives the norm.  Every call copies the result to
 *    host memory and synchronizes `stream`, so it can never be called on a
 *    stream that is being captured into a CUDA graph.
 *  - The first call on a device (with that device current) looks up the
 *    scratch region's address and configures the kernels, which may load the
 *    library's device code; while another stream captures in global mode
 *    that would invalidate the capture, so make the first call before any
 *    capture starts.  The address is kept for the life of the process: do
 *    not call it again after cudaDeviceReset() on that device.
 *  - The scratch region is shared: calls that overlap in time on one device
 *    (several threads, or several streams without ordering between them)
 *    race on it and give wrong results.  Serialize them.  Each call clears
 *    the parts that must start at zero, so what a previous call left there
 *    does not matter.
 */
#define PSF_NORM1_NOALLOC_MAX_N 65536
PSF_API int psf_norm1_noalloc(const psf_csr_t* M, void* stream, double* out);

/*
 * Host-only planner: from coefficients, tol, flags, the block-size override
 * s and the norms z_0..z_10 (||Z^i||_1, or only z_0 = 1, z_1 = ||Z||_1 with
 * PSF_Z_SUBMULT), fill N, q, b, g, products, z, alpha10, trunc, budget, and
 * the thresholds zeta[k] (k = 2..q, index k) and sigma[j] (j = 1+g..b-1,
 * index j), each array of length PSF_MAX_Q + 2 (host), entries not defined
 * set to 0.  zeta/sigma may be NULL (a plan with q > PSF_MAX_Q + 1 or
 * b > PSF_MAX_Q + 2, possible with a small s or a very long series, has
 * thresholds past those arrays: PSF_ETOOBIG unless they are NULL).  With
 * PSF_Z_SQUARE the plan is that of
 * g in W = Z^2 (see the flag; tol / z_1 for an odd series, infinite when
 * z_1 = 0); info->z still lists the z_i of Z.
 * Errors: PSF_EINVAL (null arguments, m < 1, tol, s, a non-finite
 * coefficient, a norm that is negative or not finite, mixed parities with
 * PSF_Z_SQUARE), PSF_ETOOBIG (m > 100000; thresholds past the arrays, see
 * above), PSF_ENOTCONV (Eq. 34 finds no truncation length within the m
 * coefficients).
 */
PSF_API int psf_plan(const double* coeffs, int64_t m, int32_t s, double tol, uint32_t flags,
             const double* norms, psf_info_t* info, double* zeta, double* sigma);

/*
 * Tuning, process-wide (no counterpart in the paper).
 * PSF_TUNE_TABLE_CROSSOVER: products per output row (mean over a step's
 *   rows, from the previous evaluation's or the norm phase's statistics)
 *   from which the product kernel uses its column-table slot map instead of
 *   the bitmap map (default: never, the bitmap map measured faster on the
 *   2D Laplacian and banded workloads).  Both maps give bitwise identical
 *   results; the choice only changes speed.
 * psf_autotune: evaluate `series` at Z once with each slot map (after one
 *   warm-up evaluation), time every product launch, and set the crossover
 *   that minimises the summed product time; returns it, and the time it
 *   saves against the previous setting (ms per evaluation) if `saved_ms` is
 *   not NULL.  Synchronizes `stream`.  Not thread-safe with evaluations that
 *   run concurrently on other threads (they may see either setting).
 */
#define PSF_TUNE_TABLE_CROSSOVER 1
/* PSF_TUNE_BATCH_GRAPH: 1 (default) runs the PS phase of psf_eval_batch as
 * one captured CUDA graph, 0 launches its kernels directly (same results). */
#define PSF_TUNE_BATCH_GRAPH 2
/* PSF_TUNE_BATCH_REUSE: 1 (default) lets psf_eval_batch take baby step k of
 * an instance that has dropped no entry yet from the power Z^k its norm
 * phase computed (k <= 10: the same entries as the product), 0 always runs
 * the product (same results). */
#define PSF_TUNE_BATCH_REUSE 3
/* PSF_TUNE_ALG1_FAR_SHIFT: Algorithm 1's first rescan sets the candidates at
 * or below eps_g / 2^shift apart; later passes read them again only once
 * eps_f falls below that bound (default 6; 0 sets every candidate apart,
 * 2047 none).  An integer in [0, 2047]; results are the same for all. */
#define PSF_TUNE_ALG1_FAR_SHIFT 4
/* PSF_TUNE_BARRIER_BUDGET_NS: how long a block of a cooperative kernel
 * (Algorithm 1's passes, the exact norms) waits at a grid-wide barrier
 * before it gives up, in nanoseconds (default 2e9).  A wait that runs out
 * records a device status and the call returns PSF_ETIMEOUT; the kernel's
 * blocks all return (each wait is bounded), the GPU context stays usable and
 * later calls are unaffected (every evaluation has its own control block).
 * 0 gives up at once at any barrier not yet complete: a test of that path.
 * An integer in [0, 6e10]. */
#define PSF_TUNE_BARRIER_BUDGET_NS 5
/* PSF_TUNE_FAIL_ADMISSION: fault injection for the serving loop.  k > 0
 * makes the k-th request admitted from now on (by any worker of any server)
 * fail as if its device memory could not be allocated: it completes with
 * PSF_ENOMEM without running, and the other requests of its batch run as
 * usual.  The count then returns to 0 (off).  An integer >= 0. */
#define PSF_TUNE_FAIL_ADMISSION 6
/* PSF_TUNE_DENSE_XOVER: process-wide dense-tile crossover.  A product step of
 * psf_eval (unless the series sets PSF_PARAM_DENSE_XOVER) or
 * psf_product_filter runs as an FP64 dense tile product when its algorithmic
 * multiply-adds (sum over output rows of sum_{k in A_r} nnz(B_k)) reach this
 * value times n^3 and n >= 512.  The count is, for psf_eval, that of the same
 * giant step in the series' previous evaluation (a first evaluation runs
 * sparse), and for psf_product_filter n times the product of the operands'
 * mean row lengths.  A crossover of 0 makes every product step dense, at any
 * n.  Dense tiles: both operands expanded to dense n x n arrays, every output
 * entry folded over k = 0..n-1 in order (the sparse order with zero terms,
 * which leave it unchanged), then the nonzero entries written back with
 * Algorithm 1's first pass.  Results are bitwise those of the sparse kernel.
 * Needs 3 n^2 doubles of device memory; steps with n > 16384 always run
 * sparse, and psf_eval_batch always runs sparse.  Default 0.15: one product
 * of random matrices (n = 1000..4000, GB300) ran faster as dense tiles from
 * 0.14-0.19 multiply-adds per n^3 on (the tiles run at 0.97-1.19 TFLOP/s,
 * the sparse kernel at 0.1-0.5); a value >= 0. */
#define PSF_TUNE_DENSE_XOVER 7
/* PSF_TUNE_ROW_BITMAPS: the sparse product kernel of psf_eval and
 * psf_product_filter can mark a row's output pattern from column bitmaps of
 * B's rows (built by one launch before the product, a 32-bit word per entry
 * of the entry pool) a word at a time instead of a column at a time; B rows
 * with more bitmap words than entries are marked by column.  0: never.
 * 1 (default): for products whose A rows average at least 12 entries and
 * whose B rows average at least 32 (each B row is marked many times and has
 * words to share; the giant steps of near-sparse series).  2: for every
 * product.  Results are the same either way; with 0 a call allocates no
 * bitmap words. */
#define PSF_TUNE_ROW_BITMAPS 8
PSF_API int psf_tune_set(int32_t key, double value);
PSF_API int psf_tune_get(int32_t key, double* value);
PSF_API int psf_autotune(psf_series_t series, const psf_csr_t* Z, void* stream, double* crossover,
                         double* saved_ms);

/*
 * psf_autotune_batch: tune the process-wide settings for one batch of
 * instances (series[i], Z[i]), i < count, on that batch itself:
 *  1. one warm-up psf_eval_batch (sizes are learnt), then the batch's time
 *     with the settings on entry (median of 3 event-timed calls);
 *  2. the slot map per stage: the batch evaluated once with the column-table
 *     map and once with the bitmap map (graph capture off for these two),
 *     every product launch event-timed with its work per row, and the
 *     PSF_TUNE_TABLE_CROSSOVER that minimises the summed product time (as
 *     psf_autotune, over the batch's size classes of work per row);
 *  3. with that crossover, PSF_TUNE_ROW_BITMAPS in {0, 1} and
 *     PSF_TUNE_BATCH_REUSE in {0, 1}, each timed as whole batches (median
 *     of 3); the fastest is kept.
 * The chosen settings are set process-wide and returned in *out with the
 * batch's time before and after.  Every setting gives bitwise the same
 * results; only speed changes.  Synchronizes `stream`; not thread-safe with
 * evaluations running concurrently on other threads.
 */
typedef struct {
    double table_crossover;   /* chosen PSF_TUNE_TABLE_CROSSOVER (1e300: never) */
    int32_t row_bitmaps;      /* chosen PSF_TUNE_ROW_BITMAPS */
    int32_t batch_reuse;      /* chosen PSF_TUNE_BATCH_REUSE */
    int32_t configs;          /* whole-batch configurations timed */
    int32_t launches;         /* product launches timed per slot map */
    double ms_before;         /* median ms of one psf_eval_batch with the settings on entry */
    double ms_after;          /* the same with the chosen settings */
} psf_batch_tune_t;
PSF_API int psf_autotune_batch(const psf_series_t* series, const psf_csr_t* Z, int32_t count, void* stream,
                               psf_batch_tune_t* out);

/*
 * Instrumentation (no counterpart in the paper).  psf_launch_count: kernels
 * this library has launched in this process.  psf_profile(1) makes every later product-kernel launch
 * record a CUDA event pair on its stream; psf_profile_read waits for the
 * recorded events and returns the number of timed launches, their summed
 * duration in milliseconds and their algorithmic multiply-adds, then clears
 * the record if `reset`.  Not thread-safe with concurrent evaluations.
 */
PSF_API int psf_launch_count(int64_t* count);
/* psf_fp64_peak: this GPU's FP64 fused multiply-add rate, measured: every
 * thread of 4 blocks x 256 threads per SM runs eight independent fma chains
 * of 8192 steps; the best of five event-timed launches (after three warm-up
 * launches, about 50 ms, while the clocks rise) on `stream`, in TFLOP/s
 * (2 flop per fma).  The denominator of the product
 * kernel's roofline, whose work is FP64 multiply-adds.  Synchronizes
 * `stream`.  Errors: PSF_EINVAL (null tflops), PSF_ECUDA. */
PSF_API int psf_fp64_peak(void* stream, double* tflops);
PSF_API int psf_profile(int32_t enable);
PSF_API int psf_profile_read(int64_t* launches, double* ms, double* fma, int32_t reset);

/* Read access to a result. */
PSF_API int psf_result_csr(psf_result_t r, psf_csr_t* view);          /* library-owned device arrays */
/* psf_result_copy: into caller arrays, device or host (pinned: asynchronous
 * on `stream`; a null array is skipped).  On a stream other than the next
 * evaluation's (ordered after this result's evaluation by an event), the
 * copy of one result runs while the next evaluation computes. */
PSF_API int psf_result_copy(psf_result_t r, int32_t* rowptr, int32_t* col, double* val,
                    void* stream);
PSF_API int psf_result_info(psf_result_t r, psf_info_t* info);
PSF_API int psf_result_step(psf_result_t r, int32_t i, psf_step_info_t* step);
PSF_API int psf_result_destroy(psf_result_t r);

#ifdef __cplusplus
}
#endif

#endif /* PSF_H */
