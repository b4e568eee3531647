/*
 * sccs.h -- C ABI of the GB300 (sm_103a) library for the Bayesian self-controlled case
 * series (BSCCS) MAP fit by cyclic coordinate descent, after Suchard, Simpson, Zorych,
 * Ryan and Madigan, "Massive parallelization of serial inference algorithms for a complex
 * generalized linear model" (arXiv 1208.0945).
 *
 * Conventions for every entry point:
 *   - Return value: int status.  0 = SCCS_OK; positive = a non-error status; negative = an
 *     error.  On an error nothing the call was to produce is written, and
 *     sccs_last_error() describes the cause.
 *   - Array arguments are HOST pointers unless a comment says otherwise.  The caller keeps
 *     ownership of every array it passes; the library copies what it needs before returning.
 *   - A handle owns its device memory and CUDA stream work.  Calls on one handle must not
 *     overlap (the library does not lock); distinct handles are independent.
 *   - Indices are zero-based.  Row k is an era; subject i a patient; column j a drug.
 *
 * Paper notation (Section 2.1 and 2.3): y_k events, l_k era length (offset), x_kj in {0,1},
 * n_i = sum of y over subject i's eras, X the K x J design (compressed column storage),
 * M the N x K subject loading matrix (each subject's eras contiguous, Eq. 5).
 */
#ifndef SCCS_H
#define SCCS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SCCS_ABI_VERSION 1

/* ---- status codes ---------------------------------------------------------------- */
#define SCCS_OK 0
#define SCCS_NOT_CONVERGED 1     /* sccs_fit stopped at max_cycles */
#define SCCS_PENDING 2           /* serving: request not finished yet */
#define SCCS_E_INVAL (-1)        /* bad argument: null pointer, size, range, non-positive offset */
#define SCCS_E_UNSORTED (-2)     /* patient ids decrease somewhere */
#define SCCS_E_NONBINARY (-3)    /* an explicit X value is not exactly 1 */
#define SCCS_E_NOMEM (-4)        /* host or device allocation failed */
#define SCCS_E_CUDA (-5)         /* a CUDA runtime call failed */
#define SCCS_E_TIMEOUT (-6)      /* a device-side wait exceeded its bound; the handle is reset */
#define SCCS_E_NUMERIC (-7)      /* non-finite gradient, Hessian, step or log-posterior */
#define SCCS_E_BUSY (-8)         /* serving: queue full */
#define SCCS_E_DUPLICATE (-9)    /* a row appears twice in one column */
#define SCCS_E_UNSUPPORTED (-10) /* option not supported by this library or device */

/* ---- priors (Eq. 3: Normal(0, s2) or Laplace(0, s2), s2 the variance) ----------------- */
#define SCCS_PRIOR_NONE 0
#define SCCS_PRIOR_NORMAL 1
#define SCCS_PRIOR_LAPLACE 2     /* lambda = sqrt(2 / s2) */

/* ---- convergence tests, evaluated once per full cycle (Section 2.2) ------------------- */
#define SCCS_TOL_ABS_LOGPOST 0   /* |P_t - P_{t-1}| < tol */
#define SCCS_TOL_REL_LOGPOST 1   /* |P_t - P_{t-1}| / max(1, |P_t|) < tol */
#define SCCS_TOL_GENKIN_XBETA 2  /* sum|Xb_t - Xb_{t-1}| / (1 + sum|Xb_t|) < tol (Xb_k = log(E_k/l_k); FP64
                                     state: SCCS_PREC_FP64, or the polish of SCCS_PREC_FP32_POLISH) */

/* ---- arithmetic ----------------------------------------------------------------------- */
#define SCCS_PREC_FP64 0         /* every step in FP64 */
#define SCCS_PREC_FP32_POLISH 1  /* FP32 phase (FP32 E, compensated per-subject sums, each
                                    thread's terms summed exactly, FP64 cross-thread and
                                    cross-CTA sums in a fixed order, FP64 step) to a relative change of
                                    1e-6, then FP64 cycles from that point to the requested tol
                                    (tol < 0: exactly max_cycles FP64 cycles) */
#define SCCS_PREC_FP32 2         /* the FP32 phase alone, to the requested tol (no polish) */

typedef struct sccs_handle sccs_handle;

/* Optional device allocator (for example a framework's caching allocator).  alloc returns a
 * device pointer aligned to at least 256 bytes or NULL; free receives the same size. */
typedef void *(*sccs_alloc_fn)(size_t bytes, void *ctx);
typedef void (*sccs_free_fn)(void *ptr, size_t bytes, void *ctx);

typedef struct sccs_create_opts {
    int32_t struct_size;       /* sizeof(sccs_create_opts) */
    int32_t device;            /* CUDA device ordinal */
    void *stream;              /* cudaStream_t for all work; NULL = a stream the handle owns */
    int32_t num_shards;        /* subject shards = resident CTAs of the fit kernel; 0 = one per SM */
    int32_t threads_per_block; /* 0 = 512; must be a multiple of 32 in [64, 512] */
    sccs_alloc_fn alloc;       /* NULL = cudaMalloc */
    sccs_free_fn free;
    void *alloc_ctx;
    int32_t narrow_max_nnz;    /* columns with at most this many nonzeros (and at most 2048
                                  subjects) run whole on one CTA of the team with block-level sums
                                  instead of a grid-wide reduction per coordinate (FP64 fits,
                                  4 or more shards): 0 = the default 1024; < 0 = never */
    int32_t narrow_group_max;  /* consecutive narrow columns whose subjects are pairwise disjoint
                                  have their steps taken side by side, up to this many at a time
                                  (the result is the sequential one): 0 = the default 8; 1 = one
                                  at a time */
    int32_t cluster_ctas;      /* FP64 fits (sccs_fit, served fits): columns with at most
                                  cluster_max_nnz nonzeros run on one thread-block cluster of this
                                  many CTAs, whose partial sums meet in distributed shared memory
                                  instead of a grid-wide reduction per coordinate; the other columns
                                  run on the whole team.  The team is then the CTAs the device holds
                                  in whole clusters.  0 = the default (16 when num_shards is 0, else
                                  off); 2, 4, 8 or 16; < 0 = off.  The result is the same as without
                                  clusters up to rounding (the sums are split differently). */
    int32_t cluster_max_nnz;   /* 0 = the default 8192 */
} sccs_create_opts;

typedef struct sccs_data_info {
    int64_t rows_in, rows_kept;         /* K before / after removing subjects with n_i = 0 */
    int64_t subjects_in, subjects_kept; /* N before / after */
    int64_t nnz_kept;                   /* nonzeros of X on kept rows */
    int64_t segments;                   /* (subject, column) pairs with at least one nonzero */
    int64_t max_column_nnz;
    int64_t device_bytes;               /* device memory held by the handle */
    int64_t upload_bytes;               /* bytes copied host -> device by sccs_create */
    int32_t columns;                    /* J */
    int32_t num_shards;
    int32_t threads_per_block;
    int32_t narrow_columns;             /* columns run whole on one CTA (see narrow_max_nnz) */
    int32_t cluster_ctas;               /* cluster size of the cluster columns (0: none) */
    int32_t cluster_columns;            /* columns run on one cluster (see cluster_ctas) */
} sccs_data_info;

typedef struct sccs_fit_opts {
    int32_t struct_size;       /* sizeof(sccs_fit_opts) */
    int32_t warm_start;        /* 1: start from the handle's current beta (the previous fit) */
    const double *beta0;       /* host, J values; overrides warm_start; NULL and warm_start = 0
                                  start from beta = 0 as Algorithm 1 does */
    int32_t tol_mode;          /* SCCS_TOL_* */
    int32_t max_cycles;        /* >= 0; 0 only evaluates P at the start point */
    double tol;                /* < 0 runs exactly max_cycles cycles */
    int32_t precision;         /* SCCS_PREC_FP64, SCCS_PREC_FP32_POLISH or SCCS_PREC_FP32 */
    int32_t reserved;
    double *logpost_history;   /* optional host buffer of max_cycles + 1 values: P_0 .. P_c of the
                                  last phase run (the FP64 polish in SCCS_PREC_FP32_POLISH) */
    const int32_t *subject_weights;  /* host, one weight w_i >= 0 per INPUT subject (a run of
                                  equal patient_id, dropped subjects included, in input order), or
                                  NULL for all 1.  Subject i counts w_i times in Eq. 2 and Eqs. 7-9
                                  (n_i -> w_i n_i, Y'X_j -> sum over X_j of w_i y): Section 2.5's
                                  bootstrap multiplicities, or a cross-validation fold's 0/1 mask
                                  for the fit on the other folds.  Integer arithmetic, so all-ones
                                  weights give exactly the unweighted fit.  SCCS_E_INVAL if a
                                  weight is negative or w_i n_i exceeds 2^31 - 1. */
} sccs_fit_opts;

typedef struct sccs_fit_info {
    int32_t status;            /* SCCS_OK or SCCS_NOT_CONVERGED */
    int32_t cycles;            /* full cycles run */
    int64_t steps;             /* coordinate steps = cycles * J */
    int64_t nonzero_steps;     /* steps with db_j != 0 (Algorithm 1's test) */
    double logpost;            /* P(beta) at the end, constants dropped */
    double conv_value;         /* last convergence statistic */
    double kernel_ms;          /* device time of the fit kernel (CUDA events) */
    double total_ms;           /* host wall time of the call */
    int32_t warnings;          /* bit 0: an unbounded coordinate took the trust-region bound */
    int32_t fp32_cycles;       /* cycles of the FP32 phase (FP32 modes), included in `cycles` */
} sccs_fit_info;

/* Library identification: ABI version and "sm_103a" build string. */
int sccs_version(int32_t *abi_version, const char **build);

/* Thread-local description of the last error raised by a call on this thread ("" if none).
 * The handle argument may be NULL. */
const char *sccs_last_error(const sccs_handle *h);

/*
 * sccs_create -- validate, canonicalise and upload one SCCS dataset (Section 2.3,
 * "Representation in Memory": X in compressed column storage, ones implicit).
 *   K            rows (eras); >= 0
 *   patient_id   [K] non-decreasing subject ids; a subject's eras are contiguous (Eq. 5)
 *   y            [K] event counts >= 0
 *   offset_L     [K] era lengths l_k > 0, finite
 *   J            columns (drugs); >= 0
 *   col_ptr      [J+1] column starts into row_idx; col_ptr[0] = 0, non-decreasing
 *   row_idx      [col_ptr[J]] row of each nonzero, in [0, K); any order within a column
 *   x_values     NULL for an indicator matrix, else [col_ptr[J]] values that must all be 1
 *                (the Hessian form of Eq. 9 needs x_kj^2 = x_kj)
 *   opts         NULL for defaults
 * Subjects with n_i = 0 contribute nothing (Section 2.1) and are removed here; data with no
 * event at all (K = 0 included) is rejected with SCCS_E_INVAL.  Errors: SCCS_E_INVAL, SCCS_E_UNSORTED, SCCS_E_NONBINARY, SCCS_E_DUPLICATE, SCCS_E_NOMEM,
 * SCCS_E_CUDA.  On success *out owns device memory until sccs_destroy.  The prior starts as
 * SCCS_PRIOR_NONE and beta as 0.
 */
int sccs_create(sccs_handle **out, int64_t K, const int64_t *patient_id, const int32_t *y,
                const double *offset_L, int32_t J, const int64_t *col_ptr,
                const int32_t *row_idx, const double *x_values, const sccs_create_opts *opts);

/* Release the handle and its device memory.  NULL is accepted. */
int sccs_destroy(sccs_handle *h);

/* Dimensions and memory of a created handle. */
int sccs_get_info(const sccs_handle *h, sccs_data_info *info);

/*
 * sccs_set_prior -- choose the prior of Eq. 3 for later fits: SCCS_PRIOR_NONE, or
 * SCCS_PRIOR_NORMAL / SCCS_PRIOR_LAPLACE with variance s2 > 0 (Laplace scale sqrt(s2/2)).
 * Errors: SCCS_E_INVAL.
 */
int sccs_set_prior(sccs_handle *h, int32_t prior_type, double variance);

/*
 * sccs_fit -- MAP estimate by cyclic coordinate descent (Algorithm 1): for j = 1..J take
 * the prior-regularised Newton step of Eq. 4 under a Genkin trust region, built from the
 * gradient and Hessian of Eqs. 7-9, and update L x exp(Xb) and M[L x exp(Xb)] on the rows of
 * X_j (Section 2.3 steps 1-3); refresh M[L x exp(Xb)] and test convergence after each cycle.
 * The whole fit runs in one persistent kernel on the handle's stream; the call returns when
 * it is done.
 *   opts      NULL = beta0 0, SCCS_TOL_REL_LOGPOST, tol 1e-12, max_cycles 1000, FP64
 *   beta_out  host [J] or NULL: the final beta
 *   info      host or NULL
 * Returns SCCS_OK, SCCS_NOT_CONVERGED, or an error (SCCS_E_INVAL, SCCS_E_NUMERIC,
 * SCCS_E_TIMEOUT, SCCS_E_CUDA, SCCS_E_UNSUPPORTED).  After an error the handle's beta is 0.
 */
int sccs_fit(sccs_handle *h, const sccs_fit_opts *opts, double *beta_out, sccs_fit_info *info);

/*
 * sccs_fit_batch -- independent MAP fits (Algorithm 1 on each handle's dataset and prior) in
 * one persistent cooperative launch.  Handle k's num_shards CTAs form team k; a team exchanges
 * partial sums only with itself, so teams never wait on one another and each fit gives bit for
 * bit what sccs_fit gives on the same handle.  Teams that do not fit on the device together run
 * in successive launches.  Handles must share the device and threads_per_block; the work runs
 * on handles[0]'s stream.
 *   opts      shared by all fits (NULL = sccs_fit's defaults); beta0 must be NULL (warm_start
 *             applies to every handle)
 *   beta_out  NULL, or n host pointers (each NULL or [J_k])
 *   infos     NULL, or n entries; infos[k].kernel_ms is the time of the whole batch
 * Returns SCCS_OK, or the first failing fit's error (every infos[k].status is filled).
 */
int sccs_fit_batch(sccs_handle *const *handles, int32_t n, const sccs_fit_opts *opts, double *const *beta_out,
                   sccs_fit_info *infos);

/*
 * sccs_grad_hess -- the log-likelihood derivatives along coordinate j (Eqs. 7-9, no prior):
 *   g_j = Y'X_j - N'W,  h_j = -N'[W x (1 - W)],  W = M[L x exp(Xb) x X_j] / M[L x exp(Xb)].
 *   beta  host [J]: evaluate there (the handle's state is moved to beta); NULL: at the
 *         handle's current state.
 * Errors: SCCS_E_INVAL (j out of range), SCCS_E_TIMEOUT, SCCS_E_CUDA.
 */
int sccs_grad_hess(sccs_handle *h, int32_t j, const double *beta, double *g, double *hess);

/*
 * sccs_logpost -- P(b) = L(b) + log p(b) with constants dropped (Eq. 2 and Eq. 3) under the
 * handle's prior.  beta as for sccs_grad_hess.  loglik may be NULL; it receives L(b).
 */
int sccs_logpost(sccs_handle *h, const double *beta, double *logpost, double *loglik);

/* Copy the handle's current beta (host [J]). */
int sccs_get_beta(const sccs_handle *h, double *beta_out);

/*
 * sccs_heldout_loglik -- the predictive log-likelihood of Section 2.5's cross-validation: Eq. 2
 * with subject i counted weights[i] times (the held-out fold's 0/1 mask, one value per input
 * subject as in sccs_fit_opts.subject_weights; NULL = all subjects once).
 *   beta  host [J]: evaluate there (the state L x exp(Xb) is rebuilt from it in FP64, trust
 *         radii kept, so a warm-started fit afterwards continues as if nothing had happened);
 *         NULL: at the handle's current state (after a fit, its MAP; rebuilt in FP64 from the
 *         handle's beta first if the last fit ran in SCCS_PREC_FP32 alone).
 * Errors: SCCS_E_INVAL (bad weights, non-finite beta), SCCS_E_TIMEOUT, SCCS_E_CUDA.
 */
int sccs_heldout_loglik(sccs_handle *h, const double *beta, const int32_t *weights, double *loglik);

/* ---- serving: continuous batching of fit requests (cross-validation / prior grids) ---- */

typedef struct sccs_server sccs_server;

typedef struct sccs_server_opts {
    int32_t struct_size;       /* sizeof(sccs_server_opts) */
    int32_t device;            /* CUDA device ordinal (datasets must live there) */
    int32_t max_inflight;      /* fits on the device at once; 0 is invalid; default 64 */
    int32_t queue_capacity;    /* queued requests before sccs_submit returns SCCS_E_BUSY; default 4096 */
    int64_t hbm_budget_bytes;  /* device memory for per-fit state (datasets not counted); 0 = no limit */
} sccs_server_opts;

typedef struct sccs_request {
    int32_t struct_size;       /* sizeof(sccs_request) */
    int32_t prior_type;        /* SCCS_PRIOR_* */
    sccs_handle *dataset;      /* from sccs_create; must outlive the request */
    double variance;           /* prior variance (Eq. 3) */
    int32_t tol_mode;          /* SCCS_TOL_* */
    int32_t max_cycles;
    double tol;
    int32_t precision;         /* SCCS_PREC_* */
    int32_t reserved;
    const double *beta0;       /* host [J] start point (copied at submit) or NULL for 0 */
    const int32_t *subject_weights;  /* per input subject, as sccs_fit_opts.subject_weights
                                  (copied at submit): a bootstrap replicate's multiplicities, or a
                                  cross-validation fit's training mask; NULL = all 1 */
    const int32_t *heldout_weights;  /* per input subject (copied at submit): after the fit,
                                  res->heldout_loglik = sccs_heldout_loglik at the fitted beta with
                                  these weights (the held-out fold's mask); NULL = not evaluated */
    sccs_handle *dataset_alt;  /* NULL, or the same data created with another shard count: when the
                                  device is idle and no other request waits, the request runs on
                                  whichever of the two has the larger team (lower latency); otherwise
                                  on the smaller (more fits side by side).  res->team says which. */
} sccs_request;

typedef struct sccs_result {
    int32_t status;            /* SCCS_OK, SCCS_NOT_CONVERGED or the fit's error */
    int32_t cycles;
    int32_t fp32_cycles;
    int32_t team;              /* shards (CTAs) of the handle the fit ran on (dataset or dataset_alt) */
    double logpost;
    double queue_ms;           /* submit -> start on the device */
    double latency_ms;         /* submit -> result ready */
    double *beta;              /* caller's host buffer [J] to receive beta, or NULL */
    double heldout_loglik;     /* the request's held-out predictive log-likelihood, NaN if none */
} sccs_result;

typedef struct sccs_server_stats {
    int64_t pending, running, completed;
    int64_t slot_bytes;        /* device memory held for per-fit state */
    int32_t ctas_in_use, capacity_ctas;
} sccs_server_stats;

/*
 * sccs_server_create -- start a fit server on one device.  Section 2.5 turns one analysis into
 * many independent MAP fits of the same data: cross-validation fits every candidate prior
 * variance on each training portion (10 folds) and scores the held-out portion's predictive
 * log-likelihood, and the bootstrap refits resampled subjects (200 replicates); across outcomes
 * the same drugs are fitted again for every outcome of interest.  The server runs such fits as
 * they are requested: a scheduler thread admits queued requests in arrival order as soon as
 * their per-fit device state fits the HBM budget and their dataset's CTA team fits next to the
 * fits already running; each admitted fit runs (Algorithm 1, as sccs_fit) on a stream of its
 * own, so fits that arrive while others run overlap with them (continuous batching).  A fit
 * gives the same result alone or in the mix.  Errors: SCCS_E_INVAL, SCCS_E_CUDA.
 */
int sccs_server_create(sccs_server **out, const sccs_server_opts *opts);

/* Queue one fit of Section 2.5's workflows: a (prior, variance) point of the cross-validation
 * grid fitted on the training folds (subject_weights = the training mask) with the held-out fold's
 * predictive log-likelihood (heldout_weights = the fold's mask), or a bootstrap replicate
 * (subject_weights = the resampled multiplicities).  Never waits for the GPU.  SCCS_E_BUSY when
 * the queue is full; SCCS_E_INVAL on a bad request.  *ticket identifies the request for sccs_poll. */
int sccs_submit(sccs_server *srv, const sccs_request *req, uint64_t *ticket);

/* The result of one submitted fit: the MAP beta of Algorithm 1 (Section 2.2), P(beta), and for a
 * cross-validation request the held-out predictive log-likelihood of Section 2.5 (Eq. 2 over the
 * held-out subjects), with its queueing time and latency.  SCCS_PENDING until the fit is done;
 * then fills *res (and res->beta if given), retires the ticket and returns SCCS_OK.  The fit's
 * own outcome is res->status.  Unknown ticket: SCCS_E_INVAL. */
int sccs_poll(sccs_server *srv, uint64_t ticket, sccs_result *res);

/* Queue depth, fits running, fits completed, state memory, CTAs in use. */
int sccs_server_get_stats(sccs_server *srv, sccs_server_stats *stats);

/* Finish the running fits, cancel the queued ones, release the server's device memory. */
int sccs_server_destroy(sccs_server *srv);

/*
 * sccs_selftest_exp -- diagnostic for tests: the library's e^x, used for e^{Delta beta} in every
 * coordinate step (Section 2.3's update of L x exp(X beta)), and CUDA's exp on the same n host
 * values (x, ours, ref: host arrays of n doubles; the library copies them).  Errors:
 * SCCS_E_INVAL (n < 0 or null arrays with n > 0), SCCS_E_NOMEM, SCCS_E_CUDA.
 */
int sccs_selftest_exp(int32_t device, const double *x, int64_t n, double *ours, double *ref);

/*
 * sccs_selftest_div -- diagnostic for tests: the library's quotient a/b, used for W_i = num_i/D_i
 * (Eq. 8) and the Newton step (Eq. 4) in every coordinate step, and CUDA's IEEE division on the
 * same n pairs (a, b, ours, ref: host arrays of n doubles; the library copies them).  Errors:
 * SCCS_E_INVAL (n < 0 or null arrays with n > 0), SCCS_E_NOMEM, SCCS_E_CUDA.
 */
int sccs_selftest_div(int32_t device, const double *a, const double *b, int64_t n, double *ours, double *ref);

/*
 * sccs_debug_layout -- diagnostic for tests: a copy of one array of the handle's data layout
 * (the representation of M and X_j that Section 2.4 puts in device memory, in this library's
 * sharded jagged-diagonal form), so that a test can check it against its definition.
 * which: one of SCCS_DBG_*; dst: host buffer of capacity bytes, or NULL to ask only for the size;
 * *bytes (not NULL): the array's size in bytes.  Element types: int64 for the *_PTR, SLICE_*,
 * SHARD_*, GRP_BASE, KEPT_FROM and SCALARS arrays; int32 for NEV, ROWS, YSUB, YCNT, NEXT_*,
 * NAR_ROW, NAR_GROUP, CGROUP, CROWS, ROW_COL; {int32 subject, int32 length} pairs for SEGS and
 * CSEGS; {subject, rows, first row, mark} int32 quadruples for NAR_SEG; uint8 for NARROW and CCLS;
 * double for L and YTX.  SCALARS: {kept nonzeros, input subjects, narrow columns, cluster columns,
 * first grid column, stash stride, E-stash stride, first wide column}.  An array the layout does not
 * have (no narrow or cluster columns) has size 0.  Synchronous.  Errors: SCCS_E_INVAL (null
 * handle or bytes, unknown which, capacity too small), SCCS_E_CUDA.
 */
#define SCCS_DBG_PAT_PTR 1
#define SCCS_DBG_NEV 2
#define SCCS_DBG_L 3
#define SCCS_DBG_YTX 4
#define SCCS_DBG_ROWS 5
#define SCCS_DBG_SEGS 6
#define SCCS_DBG_GRP_BASE 7
#define SCCS_DBG_SLICE_ROW 8
#define SCCS_DBG_SLICE_SEG 9
#define SCCS_DBG_SLICE_GRP 10
#define SCCS_DBG_SHARD_ROW 11
#define SCCS_DBG_SHARD_PAT 12
#define SCCS_DBG_YCOL_PTR 13
#define SCCS_DBG_YSUB 14
#define SCCS_DBG_YCNT 15
#define SCCS_DBG_NARROW 16
#define SCCS_DBG_NEXT_WIDE 17
#define SCCS_DBG_NAR_PTR 18
#define SCCS_DBG_NAR_SEG 19
#define SCCS_DBG_NAR_ROW 20
#define SCCS_DBG_NAR_GROUP 21
#define SCCS_DBG_CCLS 22
#define SCCS_DBG_NEXT_GRID 23
#define SCCS_DBG_CGROUP 24
#define SCCS_DBG_CROWS 25
#define SCCS_DBG_CSEGS 26
#define SCCS_DBG_CGRP_BASE 27
#define SCCS_DBG_CSLICE_ROW 28
#define SCCS_DBG_CSLICE_SEG 29
#define SCCS_DBG_CSLICE_GRP 30
#define SCCS_DBG_CSHARD_ROW 31
#define SCCS_DBG_CSHARD_PAT 32
#define SCCS_DBG_KEPT_FROM 33
#define SCCS_DBG_ROW_PTR 34
#define SCCS_DBG_ROW_COL 35
#define SCCS_DBG_SCALARS 36
#define SCCS_DBG_COUNT 37
int sccs_debug_layout(const sccs_handle *h, int32_t which, void *dst, int64_t capacity, int64_t *bytes);

/*
 * sccs_check_wait_timeout -- self-test of the bounded device-side waits (failure detection).
 * Launches the gradient kernel on one CTA fewer than the all-reduce counts, so the last
 * partial is never written and every launched CTA's wait must run out after timeout_ms
 * (0 < timeout_ms <= 10000).  Nothing faults or hangs: the CTAs raise the abort flag and
 * return.  Returns SCCS_E_TIMEOUT when the waits ran out as designed (the expected result),
 * SCCS_E_INVAL otherwise.  The handle is reset to beta = 0 and stays usable.  Needs at least
 * two shards and one column.
 */
int sccs_check_wait_timeout(sccs_handle *h, double timeout_ms);

/*
 * sccs_grad_hess_noalloc -- g_j and h_j of one column (the same quantities as
 * sccs_grad_hess) from arrays the caller already holds on the device, without allocating
 * any device memory.  The paper has no counterpart: this entry point exists for callers that
 * cannot allocate at the point of the call -- for example a serving process whose framework
 * reserved all device memory for its own pool up front (there a cudaMalloc fails, or
 * synchronises the device and stalls other streams), or code running inside a callback of
 * another library that forbids allocation.
 *
 * The reduction across CTAs uses a scratch array compiled into the library (about 197 KB,
 * room for SCCS_NOALLOC_MAX_SEGMENTS segments); every device that loads the library holds it
 * until the process exits.  The first call on a device looks up that array's device address
 * (with the device current); make that first call before any stream capture.  The address is
 * looked up again when the device's context has changed since (after cudaDeviceReset, say), so
 * the first call after such a reset is a set-up call too.  The call runs
 * on the calling thread's current device and is asynchronous on `stream`.  All calls share
 * the one array, so calls that overlap on the GPU (on different streams, or from different
 * host threads) race and give wrong results: order them on one stream.
 *
 *   seg_ptr      device int64 [P+1]: segment s of the column covers rows[seg_ptr[s] .. seg_ptr[s+1])
 *   seg_subject  device int32 [P]: the subject of segment s (all its rows belong to it)
 *   rows         device int32 [seg_ptr[P]]: row (era) indices into E
 *   E            device double [K]: L x exp(Xb) per row
 *   D            device double [N]: M[L x exp(Xb)] per subject
 *   n            device int32 [N]: events per subject
 *   ytx          Y'X_j, the events on the column's rows
 *   P            segments, 0 <= P <= SCCS_NOALLOC_MAX_SEGMENTS
 *   gh_out       device double [2]: receives g_j, h_j (NaN if an input was not finite or D <= 0)
 *   stream       cudaStream_t (NULL = default stream)
 * Errors: SCCS_E_INVAL (P out of range, null pointer), SCCS_E_CUDA.  No handle is needed.
 */
#define SCCS_NOALLOC_MAX_SEGMENTS 1048576
int sccs_grad_hess_noalloc(const int64_t *seg_ptr, const int32_t *seg_subject, const int32_t *rows,
                           const double *E, const double *D, const int32_t *n, double ytx, int64_t P,
                           double *gh_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SCCS_H */
