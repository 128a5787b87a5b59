/*
 * tsnnls.h -- C ABI of a GB300 (sm_103a) block principal pivoting solver for
 *
 *     min_x 1/2 ||A x - b||_2^2   subject to   x >= 0              (Eq. 1)
 *
 * where A is an m x n sparse matrix with m > n and full column rank, given in
 * CSR form.  The method is the block principal pivoting algorithm of Section 2
 * (algorithm box): it moves through complementary basic solutions
 *     x_F = argmin ||A_F x_F - b||                                  (Eq. 4)
 *     y_G = A_G^T (A_F x_F - b)                                      (Eq. 5)
 * exchanging the infeasible variables (negative entries of x_F and y_G)
 * between the index sets F and G, with a backup counter p = 3 and a
 * single-variable fallback, and zeroing entries within 1e-12 of zero.  As in
 * Section 3, A^T A and A^T b are formed once and every pivot factors the
 * F x F block of A^T A.
 *
 * All computation runs on the GPU in this library's own kernels.  There is no
 * CPU fallback: without a usable CUDA device every call returns
 * TSNNLS_ENODEV or TSNNLS_ECUDA.
 *
 * Conventions for every function below
 *   - Return value: a TSNNLS_* status code; no function throws or aborts.
 *   - Pointers marked "device" must be device memory of the context's GPU;
 *     "host" pointers are ordinary (pageable or pinned) host memory.
 *   - Input arrays are read-only and remain owned by the caller.  The library
 *     copies what it needs, except where a call says the caller's buffers must
 *     stay alive until the call (or its ticket) completes.
 *   - Indices are 0-based.  CSR column indices must be strictly ascending
 *     within a row (sorted, no duplicates); violations give TSNNLS_EINVAL.
 *   - Calls on one context are serialised by the context (thread-safe), but
 *     run in the order they are made.
 */
#ifndef TSNNLS_H
#define TSNNLS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define TSNNLS_OK 0
#define TSNNLS_EINVAL 1    /* bad argument: m <= n, n == 0, malformed CSR, NULL pointer */
#define TSNNLS_ENOMEM 2    /* device allocation failed */
#define TSNNLS_EADMIT 3    /* the problem's device footprint exceeds the context's HBM budget */
#define TSNNLS_ENOTPD 4    /* Cholesky breakdown of (A^T A)_FF: A_F is (numerically) rank deficient */
#define TSNNLS_EMAXITER 5  /* the pivot loop hit opts.max_iter without a feasible split */
#define TSNNLS_ENOCONV 6   /* iterative refinement stagnated above opts.rel_tol */
#define TSNNLS_ETIMEOUT 7  /* a bounded device-side wait gave up (no kernel hangs) */
#define TSNNLS_PENDING 8   /* tsnnls_poll: the ticket has not finished yet */
#define TSNNLS_ECUDA 9     /* a CUDA runtime call failed */
#define TSNNLS_ENODEV 10   /* no usable CUDA device / the requested device does not exist */
#define TSNNLS_ENOTFOUND 11 /* tsnnls_tune_cache_get: the cache holds no entry for the key */
#define TSNNLS_EBOUNDS 12  /* bounds-checked build only: a kernel met an index outside its buffer
                              (the access was skipped; tsnnls_check_report says where) */

/* ---- precision / path selectors ---------------------------------------- */
/* MIXED: Gram block gathered and factored in FP32 (tensor-core trailing
 *   updates), FP32 triangular solves, and FP64 iterative refinement of x_F
 *   with FP64 residuals b - A_F x_F, FP64 A^T r and FP64 sign tests.
 * FP64: every step in FP64, one normal-equations solve per pivot and no
 *   refinement (the plain baseline path). */
#define TSNNLS_MIXED 0
#define TSNNLS_FP64 1

#define TSNNLS_PATH_AUTO 0    /* factor when A^T A fits the budget, LSQR otherwise */
#define TSNNLS_PATH_FACTOR 1  /* normal equations on the cached A^T A (Sections 2-3) */
#define TSNNLS_PATH_LSQR 2    /* LSQR on A_F for each pivot (Section 3's LSQR, no A^T A) */
#define TSNNLS_PATH_SPARSE 3  /* normal equations with A^T A kept sparse and a supernodal sparse Cholesky
                                 of its F x F block per pivot (Section 3: the paper's TAUCS factor);
                                 for Grams with a small-separator pattern.  AUTO never picks it */

/* A sparse matrix in CSR form.  row_ptr has m+1 entries, row_ptr[0] == 0 and
 * row_ptr[m] == nnz; col_idx and val have nnz entries.  on_device selects
 * where row_ptr/col_idx/val AND the b / x_out arguments of the call live:
 * 0 = host memory, 1 = device memory of the context's GPU. */
typedef struct {
    int64_t m, n, nnz;
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const double *val;
    int32_t on_device;
} tsnnls_csr;

typedef struct {
    double rel_tol;      /* refinement stops when ||dx_F||_inf <= rel_tol ||x_F||_inf (default 1e-14) */
    double zero_tol;     /* |x_i|, |y_i| below this are set to 0 after each update (default 1e-12, Section 2) */
    int32_t p_max;       /* backup full exchanges before the single-variable rule (default 3) */
    int32_t max_iter;    /* pivot limit; 0 means 10 n + 100 */
    int32_t precision;   /* TSNNLS_MIXED (default) or TSNNLS_FP64 */
    int32_t path;        /* TSNNLS_PATH_* (default AUTO) */
    int32_t max_refine;  /* refinement steps per pivot before TSNNLS_ENOCONV (default 30) */
    int32_t full_refine; /* 0 (default): a pivot's refinement may stop before rel_tol once no
                            sign or zeroing decision of the next exchange can change (only signs
                            matter before the last pivot, Section 3; the last pivot is always
                            refined to rel_tol); 1: refine every pivot to rel_tol */
    int32_t no_fallback; /* MIXED: 0 (default): if the refinement on the FP32 factor stagnates
                            (the factor is too inaccurate for this conditioning), the solve is
                            redone with an FP64 factor and FP64 refinement (info.fallback_used);
                            1: return TSNNLS_ENOCONV instead */
    int32_t cond_est;    /* 1: estimate kappa_1((A^T A)_FF) at the last pivot into info.cond_est
                            (a dpocon-style 1-norm estimate, Section 3; a few extra solves);
                            0 (default): skip */
    int32_t no_reuse;    /* MIXED: 0 (default): a pivot that adds and removes only a few variables
                            since the last factorisation is solved on that factor, bordered
                            (info.factor_reuses); 1: refactor at every pivot, as the paper does */
    int32_t reserved;
} tsnnls_opts;

typedef struct {
    int32_t status;          /* same as the return value of the call */
    int32_t iters;           /* pivots performed (exchange + solve) */
    int32_t refine_steps;    /* total refinement steps over all pivots */
    int32_t nF;              /* |F| at the solution */
    int32_t path_used;       /* TSNNLS_PATH_FACTOR, TSNNLS_PATH_LSQR or TSNNLS_PATH_SPARSE */
    int32_t precision_used;  /* TSNNLS_MIXED or TSNNLS_FP64 */
    double last_rel_step;    /* ||dx_F||_inf / ||x_F||_inf of the last refinement step */
    double time_ms;          /* device time of the solve, CUDA events */
    int64_t kernel_launches; /* kernels this call launched */
    double cond_est;         /* opts.cond_est: estimated kappa_1((A^T A)_FF) at the last pivot, else 0 */
    int32_t fallback_used;   /* 1 if a MIXED solve was redone in FP64 (opts.no_fallback) */
    int32_t factor_reuses;   /* pivots solved on an earlier pivot's factor, bordered (MIXED) */
    double kkt_viol;         /* largest violation of Eq. 3 at the returned x, computed on the
                                device in FP64 with y = A^T (A x - b):
                                max(-min x, -min y, max_i |x_i y_i| / max(1, |x_i|)) / ||A^T b||_2
                                (the solve's target is <= 1e-10); 0 unless status is OK */
    double rel_resid_change; /* ||A dx||_2 / ||b - A x||_2 for the last refinement correction dx
                                (the FP64 refinement that stands in for Section 3's final
                                recompute): how much the last step still changed the residual;
                                0 when the last pivot took no refinement step (the plain FP64
                                path) or status is not OK */
} tsnnls_info;

typedef struct tsnnls_ctx tsnnls_ctx;
typedef int64_t tsnnls_ticket;

/* Fill *opts with the defaults listed above. */
void tsnnls_opts_default(tsnnls_opts *opts);

/* Human-readable name of a status code (static string, never NULL). */
const char *tsnnls_strerror(int status);

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the
 * device memory the context may hold for problem state at once (0 = 90 % of
 * the free memory at creation).  All work runs on the context's own
 * non-blocking streams.  *ctx is set only on TSNNLS_OK. */
int tsnnls_ctx_create(tsnnls_ctx **ctx, int device, size_t hbm_budget_bytes);

/* Wait for all outstanding tickets, free every device buffer, destroy ctx. */
void tsnnls_ctx_destroy(tsnnls_ctx *ctx);

/* Blocking solve of Eq. 1 (Section 2 algorithm box; Section 3 caching of
 * A^T A).  b has m entries, x_out n entries, both in host or device memory
 * as A->on_device says.  x_out is written only on TSNNLS_OK.  opts may be
 * NULL (defaults); info may be NULL, and is filled on every return.
 * Thread-safe on one context. */
int tsnnls_solve(tsnnls_ctx *ctx, const tsnnls_csr *A, const double *b, double *x_out,
                 const tsnnls_opts *opts, tsnnls_info *info);

/* tsnnls_solve with extra outputs, for inspection and tests.  y_out (n
 * doubles) receives y = A^T (A x - b) on G and 0 on F (Eq. 3, Eq. 5);
 * inF_out (n bytes) the final F as 0/1 -- both in the same memory space as
 * x_out and written only on TSNNLS_OK.  trace (host, 6 * trace_cap int64)
 * receives one row per pivot: {infeasible count, N before the branch
 * (INT64_MAX = infinity), p after the branch, branch (0 = count dropped and
 * full exchange, 1 = backup full exchange, 2 = single exchange of the
 * largest infeasible index), |F| after the exchange, the index that a single
 * exchange moved (-1 after a full exchange)}.  Any of the three may be
 * NULL. */
int tsnnls_solve_ex(tsnnls_ctx *ctx, const tsnnls_csr *A, const double *b, double *x_out,
                    double *y_out, uint8_t *inF_out, int64_t *trace, int64_t trace_cap,
                    const tsnnls_opts *opts, tsnnls_info *info);

/* Asynchronous solve: returns at once with *ticket.  A's arrays, b and x_out
 * must stay valid and unmodified until tsnnls_poll/tsnnls_wait reports
 * completion of the ticket.  The request is admitted by device footprint:
 * it waits in the context's queue until its state fits the HBM budget and a
 * slot is free, then runs concurrently with the other admitted requests
 * (continuous batching across the context's streams). */
int tsnnls_submit(tsnnls_ctx *ctx, const tsnnls_csr *A, const double *b, double *x_out,
                  const tsnnls_opts *opts, tsnnls_ticket *ticket);

/* TSNNLS_PENDING while the ticket runs; otherwise its final status (and the
 * ticket is released; polling it again gives TSNNLS_EINVAL).  Also takes the
 * tickets of tsnnls_submit_batch (below). */
int tsnnls_poll(tsnnls_ctx *ctx, tsnnls_ticket ticket, tsnnls_info *info);

/* Wait up to timeout_us microseconds (< 0: no limit).  Returns
 * TSNNLS_PENDING if the time ran out, else as tsnnls_poll. */
int tsnnls_wait(tsnnls_ctx *ctx, tsnnls_ticket ticket, int64_t timeout_us, tsnnls_info *info);

/* Asynchronous batch of independent solves under one ticket (Section 1 sets
 * the method inside a larger application that has many such problems).
 * Problem i is A[i] (an array of `count` CSR descriptors, each with its own
 * on_device), right-hand side b[i] and output x_out[i] (host arrays of
 * `count` pointers, each in the memory space its A[i].on_device names).
 * Every member is checked first (as for tsnnls_submit); if any is invalid
 * (TSNNLS_EINVAL) or can never fit the context's budget (TSNNLS_EADMIT),
 * nothing is queued.  Otherwise the call returns at once with *ticket; each
 * member is then admitted by its own device footprint and runs beside the
 * other members and the context's other requests (continuous batching).
 * The arrays of descriptors and pointers are copied; the matrices, b[i] and
 * x_out[i] must stay valid and unmodified until the ticket completes.
 * tsnnls_poll / tsnnls_wait on the ticket return TSNNLS_PENDING until every
 * member has finished, then the first failing member's status (in
 * submission order) or TSNNLS_OK, and release the ticket; their info sums
 * the members' pivots, refinement steps, |F|, device times, launches,
 * fallbacks and reuses, and takes the largest last_rel_step, cond_est,
 * kkt_viol and rel_resid_change.  x_out[i] is written only if member i
 * succeeded. */
int tsnnls_submit_batch(tsnnls_ctx *ctx, int32_t count, const tsnnls_csr *A, const double *const *b,
                        double *const *x_out, const tsnnls_opts *opts, tsnnls_ticket *ticket);

/* Status and info of member i (0-based, submission order) of a batch ticket
 * that has not been released yet: TSNNLS_PENDING while the member runs,
 * else its own final status (info filled).  Does not release anything, so
 * members' results can be collected as they finish, before tsnnls_poll /
 * tsnnls_wait releases the ticket.  TSNNLS_EINVAL for an unknown ticket or i
 * out of range. */
int tsnnls_batch_member_info(tsnnls_ctx *ctx, tsnnls_ticket ticket, int32_t i, tsnnls_info *info);

/* Counters of the asynchronous queue since the context was created. */
typedef struct {
    int64_t submitted;         /* tickets accepted by tsnnls_submit */
    int64_t completed;         /* tickets whose solve has finished */
    int64_t max_in_use_bytes;  /* largest sum of admitted footprints seen */
    int64_t budget_bytes;      /* the context's HBM budget */
    int32_t lanes;             /* streams that run admitted requests */
    int32_t max_active;        /* largest number of requests running at once */
} tsnnls_queue_stats;

int tsnnls_queue_stats_read(tsnnls_ctx *ctx, tsnnls_queue_stats *out);

/* Batched dense solves (many small or uneven problems).  Problem i has
 * A_i = a[i] (m[i] x n[i], row-major FP32, device memory), b_i = b[i]
 * (m[i] doubles, device) and x_i = x_out[i] (n[i] doubles, device).  The
 * pointer arrays a, b, x_out, m and n are host arrays of `count` entries.
 * All pivot iterations of all problems run in one persistent kernel launched
 * from a captured CUDA graph; A^T A is formed by one batched GEMM.  MIXED
 * refines each intermediate pivot only until its sign decisions are settled
 * (opts.full_refine = 1: every pivot to rel_tol), as tsnnls_solve does.  status_out
 * (host, count entries, may be NULL) receives each problem's status.
 * Returns TSNNLS_OK if every problem succeeded, else the first failure. */
int tsnnls_solve_batch_dense(tsnnls_ctx *ctx, int32_t count, const int32_t *m, const int32_t *n,
                             const float *const *a, const double *const *b,
                             double *const *x_out, const tsnnls_opts *opts,
                             int32_t *status_out, tsnnls_info *info);

/* tsnnls_solve_batch_dense with each problem's pivot trace: trace (host
 * array of count host pointers, may be NULL; an entry may be NULL) receives
 * for problem i up to trace_cap (1 .. 2^20) rows of six int64 in the layout
 * of tsnnls_solve_ex (infeasible count, N before the branch, p after it,
 * branch, |F| after the exchange, the index a single exchange moved). */
int tsnnls_solve_batch_dense_ex(tsnnls_ctx *ctx, int32_t count, const int32_t *m, const int32_t *n,
                                const float *const *a, const double *const *b, double *const *x_out,
                                const tsnnls_opts *opts, int32_t *status_out, tsnnls_info *info,
                                int64_t *const *trace, int64_t trace_cap);

/* Autotuner of the batched path's Cholesky panel width.  For each problem
 * size bucket (n <= 64, 128, 256, 512, 1024) it times the batched solve of a
 * synthetic batch with every candidate width and keeps the fastest in the
 * process-wide table that tsnnls_solve_batch_dense reads.  per_bucket caps
 * the number of problems per timing batch (<= 0: 64).  nb_out (host, 5
 * entries, may be NULL) receives the chosen widths. */
int tsnnls_batch_autotune(tsnnls_ctx *ctx, int32_t precision, int32_t per_bucket, int32_t *nb_out);

/* Set the table directly (e.g. from a cached autotune result); 5 widths in
 * [4, 64], clamped to what the kernel's shared memory allows. */
int tsnnls_batch_set_panel(int32_t precision, const int32_t *nb);

/* The autotuner with a JSON cache on disk.  The cache key names the device
 * (its name, compute capability and SM count), the precision, per_bucket and
 * the build of this library; on a hit the cached widths are installed
 * without timing anything (*hit_out = 1), on a miss the autotuner runs and
 * its result is added to the file (*hit_out = 0), which is created if
 * absent.  cache_path: a file path (host string).  nb_out (5 entries) and
 * hit_out may be NULL.  TSNNLS_EINVAL if the file exists but is not a cache
 * of this format (it is then left untouched) or cannot be written. */
int tsnnls_batch_autotune_cached(tsnnls_ctx *ctx, int32_t precision, int32_t per_bucket,
                                 const char *cache_path, int32_t *nb_out, int32_t *hit_out);

/* The cache key tsnnls_batch_autotune_cached uses on this context, as a
 * NUL-terminated string in buf (len bytes); TSNNLS_EINVAL if it does not fit. */
int tsnnls_batch_tune_key(tsnnls_ctx *ctx, int32_t precision, int32_t per_bucket, char *buf, size_t len);

/* Direct access to the cache file (host only, no device needed).  The file
 * is one JSON object {"format": "tsnnls-batch-panel-widths/1", "entries":
 * {key: [5 widths], ...}}.  get: TSNNLS_OK and the 5 widths in nb_out,
 * TSNNLS_ENOTFOUND if the file or the key is absent, TSNNLS_EINVAL if the
 * file does not parse.  put: adds or replaces the key's entry, keeping the
 * others, and replaces the file through a rename (a concurrent reader sees
 * the old or the new file, never a mix); TSNNLS_EINVAL if the existing file
 * does not parse (it is left untouched) or cannot be written.  Keys are
 * non-empty strings without control characters. */
int tsnnls_tune_cache_get(const char *path, const char *key, int32_t *nb_out);
int tsnnls_tune_cache_put(const char *path, const char *key, const int32_t *nb);

/* ---- bounds-checked build ------------------------------------------------
 * Built with -DTSNNLS_CHECK (libtsnnls_check.so), the kernels test every
 * data-dependent index (the F lists, CSR column and row indices, the sparse
 * factor's assembly maps, the exchange's moved index) against the buffer it
 * addresses.  A failing access is skipped, never trapped; the call that ran
 * the kernel returns TSNNLS_EBOUNDS once its stream is idle.  It stands in
 * for a memory checker in tests.  tsnnls_check_build: 1 in that build, else
 * 0.  tsnnls_check_report: the failing accesses since the previous call (0
 * if none, always 0 in the normal build), and in buf (len bytes, may be
 * NULL) "file:line: index i outside [0, bound)" for the first of them;
 * clears the record.  Process-wide: with several contexts or lanes at once
 * a report names the site, not the request. */
int tsnnls_check_build(void);
int tsnnls_check_report(char *buf, size_t len);

/* ---- per-phase device-time accounting ----------------------------------
 * When enabled, blocking solves on the context bracket every phase of the
 * pivot loop with CUDA events on the stream the kernels run on, and add up
 * the elapsed device time, the launches, and the phase's algorithmic work
 * (bytes for bandwidth-bound phases, flops for the factorisation) as the
 * per-unit figures of the method give them.  Off by default. */
#define TSNNLS_PHASE_SETUP 0     /* validation and CSR -> CSC transpose */
#define TSNNLS_PHASE_GRAM 1      /* A^T A and A^T b (Section 3) */
#define TSNNLS_PHASE_EXCHANGE 2  /* zeroing, infeasible count, exchange (Section 2) */
#define TSNNLS_PHASE_GATHER 3    /* (A^T A)_FF */
#define TSNNLS_PHASE_FACTOR 4    /* Cholesky */
#define TSNNLS_PHASE_TRSV 5      /* the two triangular solves */
#define TSNNLS_PHASE_SPMV 6      /* FP64 A x and A^T r (Eq. 5, refinement) */
#define TSNNLS_PHASE_VECTOR 7    /* small vector kernels (gathers, updates) */
#define TSNNLS_PHASE_LSQR 8      /* LSQR iterations on A_F */
#define TSNNLS_PHASE_FACTOR_DIAG 9     /* per kernel inside FACTOR: diagonal block factor + inverse */
#define TSNNLS_PHASE_FACTOR_PANEL 10   /*   block column below it (X = B W^T) */
#define TSNNLS_PHASE_FACTOR_UPDATE 11  /*   trailing update (tensor cores in MIXED) */
#define TSNNLS_PHASE_REUSE 12          /* setup of a bordered solve on an earlier factor (opts.no_reuse) */
#define TSNNLS_NUM_PHASES 13

typedef struct {
    double ms;          /* summed device time */
    int64_t launches;   /* kernel launches */
    double bytes;       /* algorithmic DRAM bytes (bandwidth-bound phases) */
    double flops;       /* algorithmic flops */
} tsnnls_phase_stat;

/* enable != 0 turns accounting on and zeroes the counters; 0 turns it off.
 * enable == 2 also times each kernel of the factorisation separately
 * (TSNNLS_PHASE_FACTOR_DIAG/_PANEL/_UPDATE instead of TSNNLS_PHASE_FACTOR),
 * at the cost of two events per kernel launch. */
int tsnnls_profile_enable(tsnnls_ctx *ctx, int32_t enable);

/* Copy min(count, TSNNLS_NUM_PHASES) phase records (host array). */
int tsnnls_profile_read(tsnnls_ctx *ctx, tsnnls_phase_stat *out, int32_t count);

/* ---- step-level entry points --------------------------------------------
 * Each runs one step of the pivot loop on caller-owned DEVICE buffers, on
 * the context's stream, and returns after the step completes.  They exist so
 * that every step can be checked on its own against an independent
 * implementation. */

/* Section 3: G = A^T A by column dot products (lower triangle written,
 * column-major, leading dimension ldg >= n; the strict upper triangle is not
 * touched) and c = A^T b.  precision TSNNLS_MIXED writes G as float,
 * TSNNLS_FP64 as double; c is always double.  A must be on the device. */
int tsnnls_gram(tsnnls_ctx *ctx, const tsnnls_csr *A, const double *b, int32_t precision,
                void *G, int64_t ldg, double *c);

/* Section 3: S = G_FF (lower triangle, column-major, leading dimension lds)
 * for the index list F (k ascending int32 indices < n) from a G laid out as
 * tsnnls_gram writes it.  Element type by precision as above. */
int tsnnls_gather(tsnnls_ctx *ctx, int32_t precision, const void *G, int64_t ldg,
                  const int32_t *F, int64_t k, void *S, int64_t lds);

/* Section 2 (normal equations solver): in-place lower Cholesky S = L L^T of a
 * k x k column-major symmetric positive definite matrix.  Blocked,
 * right-looking with panel width NB (128 for MIXED, which runs in FP32; 64
 * for FP64).  The lower triangle is read and overwritten with L.  The strict
 * upper triangle of each NB x NB diagonal block receives the transpose of
 * that block's inverse (L_KK^-1), which the solves use; the rest of the
 * upper triangle is untouched.  *info_out (host, may be NULL) = 0, or 1 +
 * the column of the first non-positive pivot (then the call returns
 * TSNNLS_ENOTPD).  Any lds >= k is accepted; the kernels work in place when
 * S is 16-byte aligned and lds is a multiple of 32, otherwise on a temporary
 * aligned copy (k x round_up(k, 32) elements) that is copied back. */
int tsnnls_cholesky(tsnnls_ctx *ctx, int32_t precision, void *S, int64_t k, int64_t lds,
                    int32_t *info_out);

/* Eq. 4 through the factor: overwrite rhs (k entries, float for MIXED,
 * double for FP64) with (L L^T)^{-1} rhs, using S as written by
 * tsnnls_cholesky with the same precision (L and the diagonal-block
 * inverses).  Two blocked triangular solves, one CTA per NB-row block. */
int tsnnls_chol_solve(tsnnls_ctx *ctx, int32_t precision, const void *L, int64_t k, int64_t lds,
                      void *rhs);

/* Allocation-free variant of tsnnls_chol_solve.  The paper has no
 * counterpart: this is a library-integration convenience.
 *
 * Some callers may not allocate device memory at all: applications whose
 * own pool already reserves the device memory they are allowed to use, and
 * latency-critical host threads that cannot afford cudaMalloc/cudaFree,
 * which may synchronise the whole device and can fail at run time.  This
 * call needs no context and allocates nothing: the caller passes the factor
 * L and the right-hand side (device memory, as for tsnnls_chol_solve), and
 * the solve's scratch (block flags, a ticket counter, the published solution
 * words, one partial vector per helper CTA and a status word) lives in one
 * fixed array in the library's static device memory: about 5.3 MB (sized
 * for k = TSNNLS_NOALLOC_MAX_K) that every GPU which loads the library keeps
 * until the process exits.
 *
 *   precision  TSNNLS_MIXED (float L, rhs) or TSNNLS_FP64 (double)
 *   k, lds     order of L and its leading dimension; k may be at most
 *              TSNNLS_NOALLOC_MAX_K, larger k returns TSNNLS_EINVAL
 *   stream     the cudaStream_t to run on (NULL: the default stream); the
 *              call returns after the work on it has finished
 *
 * Runs on the current CUDA device.  The first call on each device looks up
 * the device address of the static array (cudaGetSymbolAddress); make that
 * first call before any stream capture.  The address is kept until the
 * process exits, so do not call this after a cudaDeviceReset.  All calls share the array: calls
 * that overlap on the GPU (other host threads, other streams) race on it and
 * must be serialised by the caller.  Returns TSNNLS_ETIMEOUT if a bounded
 * wait inside the solve gave up. */
#define TSNNLS_NOALLOC_MAX_K 65536
int tsnnls_chol_solve_noalloc(int32_t precision, const void *L, int64_t k, int64_t lds,
                              void *rhs, void *stream);

/* Self-test of the failure path of the device-side waits (every wait in the
 * library is bounded and ends in TSNNLS_ETIMEOUT instead of hanging): one
 * kernel polls, at most `polls` times, a device flag that nothing sets.
 * polls may be at most TSNNLS_WAIT_PROBE_MAX_POLLS, the bound of every wait
 * inside the solver (seconds of polling at most).  Returns TSNNLS_ETIMEOUT (the
 * expected outcome; the device stays usable), TSNNLS_EINVAL for polls < 0 or
 * above the maximum, or a CUDA error status.  Current device, no context;
 * runs on a private non-blocking stream, but allocates and frees two small
 * device buffers (cudaMalloc / cudaFree may synchronise the device). */
#define TSNNLS_WAIT_PROBE_MAX_POLLS 4194304
int tsnnls_wait_probe(int64_t polls);

/* Symbolic analysis of the sparse normal-equations factor of
 * TSNNLS_PATH_SPARSE, on the host only (no GPU, no context): the pattern of
 * A^T A from the pattern of A (host CSR: row_ptr m + 1 entries, col_idx
 * row_ptr[m] entries), a nested-dissection order, the elimination tree of
 * the reordered matrix in postorder, the row structure of L and its
 * supernodes of at most max_width columns, small ones merged with their
 * parents (Section 3: the structure TAUCS computes before its numeric
 * factorisation).  perm_out (n entries, may be
 * NULL) receives the order (position -> original column); parent_out (n, may
 * be NULL) the elimination tree in positions (-1 at a root); stats (may be
 * NULL) the sizes below.  TSNNLS_EINVAL for a malformed pattern. */
typedef struct {
    int64_t n;             /* columns */
    int64_t nnz_gram;      /* entries of the lower triangle of A^T A's pattern, diagonal included */
    int64_t nnz_l;         /* entries of L's structure (lower triangle, diagonal included) */
    int64_t supernodes;
    int64_t max_height;    /* rows of the tallest supernode */
    double factor_flops;   /* sum over the stored columns of L of (entries in the column)^2 */
    double analysis_ms;    /* host wall time */
    int64_t nnz_l_stored;  /* entries the supernodal panels store: nnz_l plus the explicit zeros
                              that relaxed amalgamation of small supernodes adds */
    int64_t update_entries;  /* entries of the multifrontal update matrices (device memory) */
} tsnnls_sparse_stats;
int tsnnls_sparse_analyze(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col_idx, int32_t max_width,
                          int32_t *perm_out, int32_t *parent_out, tsnnls_sparse_stats *stats);

/* The supernodal tree of the same analysis (host only, no GPU, no context;
 * the arguments before ns_out as for tsnnls_sparse_analyze).  *ns_out
 * receives the number of supernodes ns; each array (caller-owned, may be
 * NULL, so a first call with NULL arrays learns ns) receives:
 *   sn_first (ns + 1): supernode s holds positions sn_first[s] ..
 *     sn_first[s + 1] - 1 of the order, supernodes in postorder;
 *   sparent (ns): the parent supernode, -1 at a root;
 *   order_up (ns): the order in which the persistent factor and forward-solve
 *     kernels take supernodes by ticket (by height: every child before its
 *     parent, which their waits rely on);
 *   order_down (ns): the same for the backward solve (by depth: every parent
 *     before its children).
 * TSNNLS_EINVAL for a malformed pattern or a NULL ns_out. */
int tsnnls_sparse_supernodes(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                             int32_t max_width, int64_t *ns_out, int32_t *sn_first, int32_t *sparent,
                             int32_t *order_up, int32_t *order_down);

/* Sparse products in FP64 on a device CSR matrix:
 *   trans == 0:  out = alpha * A x + beta * z   (x: n entries, out, z: m)
 *   trans == 1:  out = alpha * A^T x + beta * z (x: m entries, out, z: n)
 * z may be NULL when beta == 0.  All vectors are device doubles.  Each output
 * entry is summed in a fixed order, so results are reproducible. */
int tsnnls_spmv(tsnnls_ctx *ctx, const tsnnls_csr *A, int32_t trans, double alpha,
                const double *x, double beta, const double *z, double *out);

#ifdef __cplusplus
}
#endif

#endif /* TSNNLS_H */
