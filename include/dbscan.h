/*
 * dbscan.h — C ABI of the GB300 (sm_103a) exact DBSCAN library, libdbscan_gb300.so.
 *
 * The method is the three data-parallel steps of Wang et al., "Design and
 * optimization of DBSCAN Algorithm based on CUDA" (Section I's step list,
 * Section IV):
 *   1. the eps-neighbourhood test of every candidate pair, with ||p-q||^2
 *      compared against eps^2 (Section IV-A) — never stored as a distance matrix;
 *   2. core points (at least MinPts neighbours, the point itself counted;
 *      Section II, definition 2) fused with the pair test (Section IV-B,
 *      "calculate distance and construct primitive clusters at the same time");
 *   3. merging of reachable core points into clusters (Section II, definition 3;
 *      Section IV-C), here by a lock-free union-find over core-core eps-edges,
 *      then border assignment and labelling.
 *
 * Exactness.  Coordinates must be multiples of 2^-10 in [0, 1).  With
 * u = 1024 x (integers 0..1023) and T = floor(eps^2 * 2^20) computed in double
 * from the float eps, q is a neighbour of p iff sum_k (u_pk - u_qk)^2 <= T.
 * Every kernel decides this predicate exactly, so the labels are a pure
 * function of the input:
 *   - a core point's label is the smallest core index of its cluster;
 *   - a border point (non-core with a core neighbour) takes the label of its
 *     smallest-index core neighbour;
 *   - noise is -1;
 *   - DBSCAN_LABEL_COMPACT renumbers cluster ids to 0..k-1 in increasing order
 *     of their smallest core index.
 *
 * Memory.  Unless a function says otherwise, `points` and `labels_out` are
 * DEVICE pointers owned by the caller; the library never frees them and keeps
 * no reference after the call (serve jobs hold theirs until they are done).
 * Points are row-major float32 n x d.  A plan owns all its workspace (device
 * memory allocated in dbscan_plan_create).
 *
 * Errors.  Every function returns an int status: 0 (DBSCAN_OK) or a
 * DBSCAN_ERR_* code; dbscan_strerror() names it.  Checks done on the device
 * (the 2^-10 grid test, bounded waits) are reported when the plan is
 * synchronous, or by dbscan_plan_sync() otherwise.
 *
 * Threads.  A plan is not thread-safe: one host thread at a time.  The serve
 * API's submit/poll/wait are thread-safe.
 */
#ifndef DBSCAN_GB300_H
#define DBSCAN_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DBSCAN_ABI_VERSION 2

/* Status codes. */
#define DBSCAN_OK 0
#define DBSCAN_ERR_ARG 1           /* null pointer, n < 0, d < 1, eps <= 0 or not finite, min_pts < 1, n > max_n, d > max_d */
#define DBSCAN_ERR_NOT_QUANTISED 2 /* a coordinate is not k * 2^-10 with 0 <= k <= 1023 (checked on the device) */
#define DBSCAN_ERR_OOM 3           /* device or host allocation failed */
#define DBSCAN_ERR_CUDA 4          /* a CUDA runtime call failed */
#define DBSCAN_ERR_TIMEOUT 5       /* a bounded device-side wait or a host wait expired */
#define DBSCAN_ERR_BUSY 6          /* serve admission is full (slots or HBM budget) */
#define DBSCAN_ERR_UNSUPPORTED 7   /* option or shape this build does not handle; also n above 2^29 on the
                                      grid paths or above 2^25 on the all-pairs paths (int32 index ranges) */
#define DBSCAN_ERR_NOT_FOUND 8     /* unknown serve job id */

/* Pair-test arithmetic. */
#define DBSCAN_PREC_AUTO 0       /* tensor-core FP16 Gram for d >= 16 all-pairs, SIMT otherwise */
#define DBSCAN_PREC_EXACT_SIMT 1 /* FP32/INT32 CUDA-core pair test, exact by construction */
#define DBSCAN_PREC_FP16_GRAM 2  /* tcgen05 FP16 Gram product, exact by proof (band 0) */
#define DBSCAN_PREC_BF16_GRAM 3  /* tcgen05 BF16 Gram product (two-term split) + exact recheck of the band */

/* Candidate generation. */
#define DBSCAN_GRID_AUTO 0 /* eps-grid for d <= 3, projected grid for 4 <= d <= 8 (when its cells, of side
                              floor(sqrt(T)) + 1 units, split each axis at least 4 ways), all pairs otherwise */
#define DBSCAN_GRID_ON 1   /* a grid path (d <= 8 and, for d >= 4, cells as above; else DBSCAN_ERR_UNSUPPORTED) */
#define DBSCAN_GRID_OFF 2  /* all pairs */

/* Label numbering. */
#define DBSCAN_LABEL_ROOT_INDEX 0 /* cluster id = smallest core index in the cluster */
#define DBSCAN_LABEL_COMPACT 1    /* cluster ids 0..k-1 in increasing order of that index */

/* Which path a run took (dbscan_stats.path). */
#define DBSCAN_PATH_NONE 0
#define DBSCAN_PATH_GRID 1
#define DBSCAN_PATH_ALLPAIRS_SIMT 2
#define DBSCAN_PATH_ALLPAIRS_TC 3
#define DBSCAN_PATH_GRID_PROJECTED 4 /* 4 <= d <= 8: cells of the first three coordinates, full-d test */
#define DBSCAN_PATH_PAPER 5          /* dbscan_run_paper: the paper's materialised matrices */

typedef struct dbscan_plan dbscan_plan;

typedef struct dbscan_opts {
    int32_t device;      /* CUDA device ordinal */
    int32_t synchronous; /* 1: dbscan_run waits for the device and reports its errors; 0: enqueue only */
    void *stream;        /* cudaStream_t to enqueue on; NULL = the legacy default stream.  The
                            eps-grid path forks independent kernels onto an internal stream of
                            the plan and joins them back by events before the run ends, so a
                            run stays ordered on this stream (and can be graph-captured). */
    int64_t max_n;       /* largest n this plan accepts (workspace is sized for it) */
    int32_t max_d;       /* largest d this plan accepts */
    int32_t precision;   /* DBSCAN_PREC_* */
    int32_t grid;        /* DBSCAN_GRID_* */
    int32_t label_mode;  /* DBSCAN_LABEL_* */
    int32_t profile;     /* 1: record a CUDA event after every kernel (see dbscan_plan_phase_times) */
    int32_t reserved[7]; /* zero */
} dbscan_opts;

typedef struct dbscan_stats {
    int64_t n_clusters;      /* clusters found */
    int64_t n_core;          /* core points */
    int64_t n_border;        /* border points */
    int64_t n_noise;         /* noise points */
    int64_t candidate_pairs; /* ordered pairs the method must decide: n^2 (all pairs) or the pairs
                                inside each cell's neighbourhood (grid paths) */
    int64_t band_pairs;      /* tensor-core path: pairs inside the rounding band, rechecked exactly */
    int32_t path;            /* DBSCAN_PATH_* */
    int32_t cells;           /* grid path: occupied cells */
    int64_t threshold;       /* T = floor(eps^2 * 2^20) */
    float ms_total;          /* device time of the run (CUDA events), when measured */
    int32_t kernels;         /* kernel launches the run enqueued */
    int64_t pair_tests;      /* pair predicates evaluated on the device, all passes (the count, merge
                                and border passes' counters; pairs decided without a test, such as
                                the pairs inside a clique cell or those skipped by an early exit,
                                are not counted) */
    float reserved_f[4];
} dbscan_stats;

/* Fills *opts with defaults: device 0, synchronous, default stream, max_n 1<<20,
 * max_d 64, PREC_AUTO, GRID_AUTO, LABEL_ROOT_INDEX. */
void dbscan_opts_default(dbscan_opts *opts);

/* Creates a plan and allocates its device workspace for (max_n, max_d): the
 * point rows of Section IV-A (packed, the paper's point[3][N] layout idea),
 * the neighbour counts and core flags of Section IV-B (its `valid` vector),
 * the union-find forest that replaces Section IV-C's cluster matrix, and the
 * candidate structures of the grid paths.
 * *out receives the plan; on error *out is NULL.  DBSCAN_ERR_OOM if the
 * workspace does not fit. */
int dbscan_plan_create(dbscan_plan **out, const dbscan_opts *opts);

/* Waits for the plan's stream, frees its workspace and the plan.  NULL is a no-op. */
int dbscan_plan_destroy(dbscan_plan *plan);

/* Clusters one point set (Section I's three steps; Section IV).
 *   points     device, row-major float32 [n][d], on the 2^-10 grid in [0,1)
 *   n, d       0 <= n <= max_n, 1 <= d <= max_d; n = 0 is a no-op
 *   eps        finite, > 0 (float32); min_pts >= 1
 *   labels_out device int32 [n]
 *   stats      host, nullable; when given, the call synchronises and fills it
 * Enqueued on the plan's stream.  Synchronous plans return device-side errors
 * (DBSCAN_ERR_NOT_QUANTISED); asynchronous plans report them from
 * dbscan_plan_sync().  On an error labels_out is unspecified. */
int dbscan_run(dbscan_plan *plan, const float *points, int64_t n, int32_t d, float eps, int32_t min_pts,
               int32_t *labels_out, dbscan_stats *stats);

/* dbscan_run plus per-point diagnostics, both device pointers and nullable:
 *   counts_out int32 [n]: |eps-neighbourhood| with the point itself (Section II,
 *              definition 1).  Asking for it turns off the early exit at min_pts.
 *   core_out   uint8 [n]: 1 for core points (count >= min_pts). */
int dbscan_run_detail(dbscan_plan *plan, const float *points, int64_t n, int32_t d, float eps,
                      int32_t min_pts, int32_t *labels_out, int32_t *counts_out, uint8_t *core_out,
                      dbscan_stats *stats);

/* dbscan_run with HOST buffers: copies points host->device into plan
 * workspace, clusters, copies labels device->host and waits.  Pinned host
 * memory gives the fastest copies; pageable memory works.  This is the
 * end-to-end call. */
int dbscan_run_host(dbscan_plan *plan, const float *host_points, int64_t n, int32_t d, float eps,
                    int32_t min_pts, int32_t *host_labels, dbscan_stats *stats);

/* The paper's own pipeline, as a comparison variant (Section IV): an N x N
 * matrix of squared distances (Section IV-A), the primitive-cluster matrix and
 * the `valid` vector of core points (Section IV-B), and one merge launch per
 * target cluster, ORing every mergeable cluster's row into the target's
 * (Section IV-C), swept over the targets until a sweep merges nothing.  Two
 * clusters merge iff a core point lies in both rows.  Labels are those of
 * dbscan_run (same canonical form and label mode).  Arguments as dbscan_run,
 * with d <= 16 and n <= DBSCAN_PAPER_MAX_N (the matrices take 5 n^2 bytes of
 * device memory, allocated by the plan on first use and kept until it is
 * destroyed).  Always synchronous (the merge sweeps are driven from the host);
 * stats->cells receives the number of sweeps.  DBSCAN_ERR_OOM if the matrices
 * do not fit. */
#define DBSCAN_PAPER_MAX_N 65536
int dbscan_run_paper(dbscan_plan *plan, const float *points, int64_t n, int32_t d, float eps, int32_t min_pts,
                     int32_t *labels_out, dbscan_stats *stats);

/* Waits for everything enqueued on the plan and returns the first device-side
 * error recorded since the last sync (then clears it). */
int dbscan_plan_sync(dbscan_plan *plan);

/* Per-kernel device times of the plan's last run, measured with CUDA events
 * on the plan's stream (opts.profile must be 1).  Waits for the run.  Writes
 * up to max_phases entries: ms[i] is the time of kernel i, names[i] a static
 * string naming it (nullable arrays); *count receives the number of kernels. */
int dbscan_plan_phase_times(dbscan_plan *plan, int32_t max_phases, float *ms, const char **names, int32_t *count);

/* Check of the tensor-core pair test's rounding band (Section IV-B's Gram
 * form on FP16/BF16 tensor cores): runs the count pass over all n^2 pairs of
 * `points` (device, row-major float32 [n][d], d <= 64) deciding every pair
 * both the fast way and exactly in int32, and reports what it saw.  For
 * diagnosis and tests (it is slow: an exact recheck per pair).  The plan needs
 * max_d >= 16.  bf16 = 0 checks FP16 operands, 1 BF16. */
typedef struct dbscan_tc_report {
    int64_t pairs;              /* ordered pairs examined (n^2) */
    int64_t band_pairs;         /* pairs inside the band, which the fast path rechecks */
    int64_t wrong_outside_band; /* pairs outside the band decided differently from exact: must be 0 */
    int64_t max_abs_error_2g;   /* largest |2G_tensor - 2G_exact| seen, in squared grid units */
    int64_t band_halfwidth_2g;  /* band half-width in the same units (FP16: 0, exact by proof; BF16: 16 K, K = d padded to 16) */
    int64_t threshold;          /* T */
} dbscan_tc_report;
int dbscan_tc_verify(dbscan_plan *plan, const float *points, int64_t n, int32_t d, float eps, int32_t bf16,
                     dbscan_tc_report *out);

/* Raw device counters of the plan's last run (diagnostics): copies up to n of
 * the plan's 32 64-bit counters to out (host).  Slot 6 counts band pairs
 * rechecked exactly; slot 15 is 1 when the FP16 tensor-core count pass ran
 * its folded form (the column norm subtracted inside the MMA, used when
 * 3 max|v|^2 + 1 <= 2^25 for the centred units v = u - 512, which keeps it
 * exact); slots 16..19 count the pair predicates evaluated by the
 * count, merge, border and (eps-grid path) outer-ring merge passes (their sum
 * is dbscan_stats.pair_tests);
 * builds made for pipeline diagnostics fill slots 9..13, 20..24 and 25..29
 * (tensor-core count, merge and border passes) with cycles spent
 * blocked per pipeline role.  Waits for the plan's stream. */
int dbscan_plan_counters(dbscan_plan *plan, uint64_t *out, int32_t n);

/* Device bytes the plan's workspace holds. */
int64_t dbscan_plan_workspace_bytes(const dbscan_plan *plan);

/* Failure-detection test hook (the paper has none).  DBSCAN_HOOK_TC_STALL
 * makes the plan's next run that takes the tensor-core path issue no MMA in
 * its counting pass: every bounded device-side wait of that pass then expires
 * (50 ms budget instead of about 2 s), the CTAs take their abort path (wait
 * for their own copies, free tensor memory, return), and the run returns
 * DBSCAN_ERR_TIMEOUT with unspecified labels.  The hook is consumed by that
 * run; the plan stays usable.  No GPU fault, trap or hang is involved.
 * Returns DBSCAN_ERR_ARG for a null plan or an unknown hook. */
#define DBSCAN_HOOK_NONE 0
#define DBSCAN_HOOK_TC_STALL 1
int dbscan_plan_test_hook(dbscan_plan *plan, int32_t hook);

/* ---- Batched form: many independent instances in one graph-captured launch sequence ---- */

typedef struct dbscan_instance {
    const float *points; /* device, row-major float32 [n][d] */
    int64_t n;
    int32_t d;
    float eps;
    int32_t min_pts;
    int32_t *labels_out; /* device int32 [n]; labels are local indices 0..n-1 of this instance */
} dbscan_instance;

/* Clusters `count` independent instances, each by Section I's three steps as
 * dbscan_run would (with the plan's label mode; the all-pairs CUDA-core tile
 * of Sections IV-A/IV-B, 1 <= d <= 16, larger d gives
 * DBSCAN_ERR_UNSUPPORTED).  Batching many instances into one launch sequence
 * is this library's addition: the paper clusters one point set.  All instances run in one graph-captured launch
 * sequence of persistent kernels that share a work queue of (instance, row
 * tile, column chunk) items.  The first call autotunes the chunk size and grid
 * on the given batch.  Uses its own device workspace, grown on demand and kept
 * by the plan.  Synchronous; per_inst (host, nullable, `count` entries)
 * receives per-instance counts.  DBSCAN_ERR_ARG above 2^30 points in all;
 * DBSCAN_ERR_UNSUPPORTED when the work items (32-point row tiles x column
 * chunks of four 64-point tiles, the finest shape the autotuner tries: about
 * n^2 / 8,192 per instance) exceed 2^31.  With per_inst given,
 * each entry's pair_tests counts the instance's evaluated pair predicates and
 * the plan's counters 16..18 (dbscan_plan_counters) hold the batch's totals
 * for the count, merge and border passes. */
int dbscan_batch(dbscan_plan *plan, const dbscan_instance *inst, int32_t count, dbscan_stats *per_inst);

/* The configuration dbscan_batch's autotuner picked for this plan on its first
 * call: column tiles (64 points each) per work item and resident blocks per SM.
 * DBSCAN_ERR_NOT_FOUND before the first batch. */
int dbscan_batch_config(dbscan_plan *plan, int32_t *chunk_tiles, int32_t *blocks_per_sm);

/* The tile shape dbscan_batch's autotuner picked with that configuration:
 * rows per row tile (32, 64 or 128) by 64 columns per column tile.
 * DBSCAN_ERR_NOT_FOUND before the first batch. */
int dbscan_batch_tile(dbscan_plan *plan, int32_t *tile_rows, int32_t *tile_cols);

/* ---- Served form: continuous batching of submitted jobs under an HBM budget ---- */

typedef struct dbscan_server dbscan_server;

typedef struct dbscan_serve_opts {
    int32_t device;
    int32_t slots;            /* jobs that may be on the device at once (each slot: one stream, one plan) */
    int64_t hbm_budget_bytes; /* admission cap on the summed device workspace of the jobs on the device */
    int32_t label_mode;       /* DBSCAN_LABEL_* */
    int32_t precision;        /* DBSCAN_PREC_* */
    int64_t max_n;            /* largest job accepted */
    int32_t max_d;            /* largest d accepted */
    int32_t max_queue;        /* jobs waiting for a slot before submit answers DBSCAN_ERR_BUSY */
    int32_t reserved[4];
} dbscan_serve_opts;

/* What a server has done and holds (dbscan_serve_info). */
typedef struct dbscan_serve_stats {
    int64_t jobs_done;                /* jobs completed since the server started */
    int64_t jobs_queued;              /* jobs waiting for admission now */
    int32_t jobs_running;             /* jobs on the device now */
    int32_t max_jobs_running;         /* most jobs that were on the device at once */
    int64_t hbm_budget_bytes;         /* the admission cap */
    int64_t bytes_in_flight;          /* summed workspace of the jobs on the device now */
    int64_t peak_bytes_in_flight;     /* largest such sum so far */
    int64_t pool_reserved_bytes;      /* device memory the server's pool holds now */
    int64_t pool_peak_reserved_bytes; /* largest it has held */
    int64_t reserved[4];
} dbscan_serve_stats;

/* Defaults: device 0, 8 slots, 120 GiB budget, root-index labels, PREC_AUTO,
 * max_n 500,000, max_d 64, max_queue 1,000,000. */
void dbscan_serve_opts_default(dbscan_serve_opts *opts);

/* Starts a server: creates every slot (stream, event, a plan without
 * workspace), a stream-ordered device memory pool and the worker thread that
 * admits queued jobs to free slots (continuous batching: a job is admitted as
 * soon as a slot and enough of the HBM budget are free, while other jobs still
 * run).  An admitted job's workspace, exactly what its (n, d) needs
 * (dbscan_serve_job_bytes), is taken from the pool on its slot's stream and
 * returned to it there behind the job's kernels, so the budget limits the
 * device memory the jobs on the device hold; a job larger than the whole
 * budget still runs, alone.  Freed blocks stay in the pool (up to the budget)
 * for later jobs.  The serving form of the paper's method has no counterpart
 * in the paper: it is the continuous-batching server this library adds. */
int dbscan_serve_create(dbscan_server **out, const dbscan_serve_opts *opts);
/* Queues a job (Section I's three steps on one instance, as dbscan_run; the
 * server around it has no counterpart in the paper).  The
 * instance's device buffers must stay valid until it is done.  *job_id
 * receives its id.  DBSCAN_ERR_ARG for a bad instance or n > max_n / d >
 * max_d; DBSCAN_ERR_BUSY when max_queue jobs already wait.  Thread-safe. */
int dbscan_serve_submit(dbscan_server *srv, const dbscan_instance *inst, uint64_t *job_id);
/* *done = 1 once the job's labels are written; the job's own status is
 * returned then (0 otherwise).  DBSCAN_ERR_NOT_FOUND for an unknown or
 * released id.  Thread-safe. */
int dbscan_serve_poll(dbscan_server *srv, uint64_t job_id, int32_t *done);
/* Waits up to timeout_us (< 0: forever) for the job and releases it.
 * DBSCAN_ERR_TIMEOUT if it is not done by then (the job stays).  latency_us
 * (nullable) receives its submit-to-done time in microseconds.  Returns the
 * job's status.  Thread-safe. */
int dbscan_serve_wait(dbscan_server *srv, uint64_t job_id, int64_t timeout_us, double *latency_us);
/* Statistics of the server (host, filled): jobs, concurrency, budget, the
 * workspace bytes of the jobs on the device and what the pool holds.
 * Thread-safe. */
int dbscan_serve_info(dbscan_server *srv, dbscan_serve_stats *out);
/* Device workspace bytes a job of n points in d dimensions holds while it
 * runs (what admission charges against the budget); -1 for n or d out of the
 * server's range. */
int64_t dbscan_serve_job_bytes(const dbscan_server *srv, int64_t n, int32_t d);
/* Waits for every admitted job, stops the worker and frees the slots.  Jobs
 * still queued are dropped (they complete with DBSCAN_ERR_BUSY).  Threads
 * blocked in dbscan_serve_wait at that moment return (with their job's status)
 * before anything is freed; no submit, poll or wait call may start after
 * destroy has returned, and none may start once it has begun except by a
 * thread that was already blocked in wait. */
int dbscan_serve_destroy(dbscan_server *srv);

/* ---- Entry point that allocates nothing (the paper has no counterpart) ----
 *
 * For callers that cannot call cudaMalloc: a process that reserved all device
 * memory for its own pool up front, code that may not take the allocator's
 * locks while other work runs, a fixed memory budget.  Clusters one instance
 * like dbscan_run with the all-pairs CUDA-core path, taking its scratch from a
 * fixed array in the library's device image (about 1.3 MiB, held on every GPU
 * that loads the library until exit) instead of a plan.
 *   points     device, row-major float32 [n][d], on the 2^-10 grid in [0,1)
 *   n, d       0 <= n <= DBSCAN_NOALLOC_MAX_N, 1 <= d <= DBSCAN_NOALLOC_MAX_D;
 *              larger sizes return DBSCAN_ERR_ARG
 *   label_mode DBSCAN_LABEL_ROOT_INDEX or DBSCAN_LABEL_COMPACT
 *   labels_out device int32 [n]
 *   stream     cudaStream_t (NULL = legacy default stream); the call waits for it
 * Runs on the calling thread's current device.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) and caches it
 * with the id of the current CUDA context; a call in a new context on that
 * device (after cudaDeviceReset, say) looks it up again.  Make the first call,
 * and the first after such a change, before any stream capture.  All calls
 * share the one array and it keeps the last call's contents (each call clears
 * what must start at zero): calls whose work overlaps on the GPU race and must
 * not be issued.
 * Returns DBSCAN_ERR_NOT_QUANTISED for off-grid input. */
#define DBSCAN_NOALLOC_MAX_N 16384
#define DBSCAN_NOALLOC_MAX_D 16
int dbscan_run_noalloc(const float *points, int64_t n, int32_t d, float eps, int32_t min_pts, int32_t label_mode,
                       int32_t *labels_out, void *stream);

/* Static description of a status code. */
const char *dbscan_strerror(int status);

/* DBSCAN_ABI_VERSION of the loaded library. */
int32_t dbscan_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DBSCAN_GB300_H */
