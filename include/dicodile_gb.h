/*
 * dicodile_gb.h -- C ABI of the GB300 (sm_103a) convolutional sparse coding
 * library: locally greedy coordinate descent (LGCD) with the soft-lock rule of
 * DiCoDiLe, and the dictionary-update statistics and step that follow it.
 *
 * Problem (Section 2, Eq. csc / Eq. cdl):
 *     min_Z  1/2 || X - Z * D ||_2^2 + lambda ||Z||_1,
 *     min_D  1/2 || X - Z * D ||_2^2   s.t. ||D_k||_2 <= 1.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Shapes: d convolutional dimensions (1 or 2), P channels, K atoms, signal
 *    size T, atom size L.  For d == 1 only T[0] and L[0] are used and T[1],
 *    L[1] must be 1.  For d == 2, index 0 is the row (slow) axis.
 *  - The activation domain is the "valid" one: Tz_i = T_i - L_i + 1, so that
 *    X = Z * D covers the signal exactly.
 *  - Layouts are dense, row-major, fp32 unless stated:
 *        X    [P][T0][T1]          D    [K][P][L0][L1]
 *        Z    [K][Tz0][Tz1]        beta [K][Tz0][Tz1]
 *        dtd  [K][K][2L0-1][2L1-1] phi  [K][K][2L0-1][2L1-1]
 *        psi  [K][P][L0][L1]
 *    (for d == 1 drop the size-1 axes: X [P][T], D [K][P][L], ...).
 *    dtd[k][k2][delta + L - 1] = sum_p sum_tau D_kp[tau] D_k2p[tau + delta].
 *  - All array pointers are DEVICE pointers owned by the caller; the library
 *    never allocates device memory.  Scratch space is a caller-owned device
 *    buffer of at least csc_workspace_size() bytes.  Host scalars read back
 *    from the device (and the queue's control records) pass through one 8 KB
 *    pinned host buffer per calling host thread, allocated on first use and
 *    kept until the process ends: copies through pageable memory cost
 *    hundreds of microseconds on the GB300 platform.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL is the legacy default
 *    stream).  Calls that return a host scalar or a stats struct synchronise
 *    that stream before returning; this is stated per call.
 *  - Every call returns a status code (CSC_OK == 0).  On CSC_ERR_INVALID
 *    nothing was enqueued.  On CSC_ERR_CUDA the CUDA error is also available
 *    from csc_last_cuda_error().
 */
#ifndef DICODILE_GB_H
#define DICODILE_GB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define CSC_API __attribute__((visibility("default")))
#else
#define CSC_API
#endif

typedef void *csc_stream_t; /* a cudaStream_t */

enum csc_status {
    CSC_OK = 0,
    CSC_ERR_INVALID = 1,       /* bad shape, null pointer, L > T, bad option   */
    CSC_ERR_CUDA = 2,          /* a CUDA runtime call failed                   */
    CSC_NOT_CONVERGED = 3,     /* max_updates reached before max|dZ| < tol     */
    CSC_ERR_TIMEOUT = 4,       /* a device-side wait hit its time limit        */
    CSC_ERR_DIVERGED = 5,      /* ||Z||_inf > min_k 50 / ||D_k||_inf (Sec. 5.1) */
    CSC_ERR_UNIMPLEMENTED = 6, /* shape/option combination not supported       */
    CSC_ERR_WORKSPACE = 7      /* workspace too small for this call            */
};

enum csc_mode {
    CSC_MODE_ASYNC = 0,   /* tiles update asynchronously; border updates pass the soft-lock test */
    CSC_MODE_PHASED = 1,  /* deterministic checkerboard phases (for testing)                     */
    CSC_MODE_NOLOCK = 2   /* asynchronous without the soft-lock (ablation only)                   */
};

typedef struct {
    int d;     /* 1 or 2                                  */
    int P;     /* channels                                */
    int K;     /* atoms                                   */
    int T[2];  /* signal size                             */
    int L[2];  /* atom size                               */
} csc_shape;

typedef struct {
    int tile[2];          /* worker tile per dimension (0 = planned automatically; at least
                             L_i, and at least 2 L_i - 1 for asynchronous tiles in global
                             memory, else CSC_ERR_INVALID)                              */
    int sub[2];           /* LGCD sub-domain per dimension (0 = 2 L_i, Section 3)          */
    int mode;             /* enum csc_mode                                                 */
    int max_workers;      /* upper bound on the number of tiles (0 = all co-resident)      */
    long long max_updates;/* stop with CSC_NOT_CONVERGED after this many (0 = no limit)    */
    double timeout_s;     /* device wall-clock limit of one solve launch (0 = 30 s)        */
    int beta_refresh;     /* re-solves allowed after recomputing beta from scratch (>= 0)  */
    int divergence_guard; /* 1 = stop with CSC_ERR_DIVERGED when the Section 5.1 bound hits */
    int warm_start;       /* 1 = Z and beta on entry are a consistent starting point        */
    int placement;        /* 0 = automatic, 1 = tiles in shared memory, 2 = tiles in global
                             memory (used when a tile's beta, Z and table do not fit)      */
    int beta_init;        /* cdl_fit: 0 = beta-init in FP32 (csc_init_beta), 1 = on the
                             tensor cores in split bf16 (csc_init_beta_bf16x3) after the
                             first iteration, whose exact beta also fixes lambda; cdl_step:
                             the same choice when lambda is given                       */
    double stop_margin;   /* workers stop when no |dZ| reaches stop_margin * tol, in (0, 1]
                             (0 = 0.99 in FP32, 1 in FP64); the check on a beta
                             recomputed from scratch always uses tol itself            */
} csc_solve_opts;

typedef struct {
    long long updates;           /* accepted coordinate updates                          */
    long long iterations;        /* sub-domain iterations over all workers               */
    long long rejected_softlock; /* border candidates rejected by the soft-lock test     */
    long long skipped_subtol;    /* iterations whose best |dZ| was below tol             */
    long long messages;          /* neighbour notifications (k0, s0, dZ) sent            */
    long long refresh_rounds;    /* beta recomputations from scratch                     */
    int workers;                 /* tiles (one CTA each)                                 */
    int placement;               /* 1 = shared-memory tiles, 2 = global-memory tiles     */
    int tiles[2];                /* tile grid                                            */
    int tile_size[2];            /* full tile size                                       */
    double max_dz_final;         /* max |dZ| on a freshly recomputed beta (final KKT)    */
    double objective;            /* 1/2||X - Z*D||^2 + lambda||Z||_1, FP64 accumulation   */
    long long nnz;               /* nonzeros of Z at the end                             */
    double kernel_ms;            /* device time of the LGCD launches (CUDA events)       */
    long long deferred;          /* accepted candidates postponed: a neighbour inbox was full */
    long long max_worker_iterations; /* iterations of the busiest worker (critical path)  */
    long long max_worker_updates;    /* updates of the busiest worker                      */
    long long last_active_wave;  /* latest wave (per worker) that found work             */
    double t_first_pause_us;     /* latest worker-local time of a first pause             */
    double t_exit_us;            /* latest worker-local exit time                         */
    long long wakeups;           /* pauses ended by an incoming message (all workers)     */
    long long phase_cycles[6];   /* SM cycles summed over workers: wave start, neighbour
                                    messages, scan + apply, soft-lock tests, end of wave,
                                    pauses                                                */
    long long candidates;        /* coordinates scanned: K x |C_m| summed over iterations */
    int status;                  /* the returned status                                  */
} csc_solve_stats;

/* Default options: automatic tiling, sub-domains of 2L, ASYNC mode, refresh 2. */
CSC_API void csc_default_opts(csc_solve_opts *opts);

/* Bytes of device workspace needed by csc_lgcd_solve, csc_objective and
 * cdl_dict_stats / cdl_dict_update for `shape` under `opts` (opts may be NULL
 * for the defaults).  Host-only; does not touch the GPU beyond querying the
 * device properties of the current device. */
CSC_API int csc_workspace_size(const csc_shape *shape, const csc_solve_opts *opts, size_t *bytes);

/* beta = D~ * X and the atom cross-correlation table (Alg. 1 initialisation,
 * Eq. beta_update table, Section 3; lambda_max of Section 2).
 *   X [P][T] in, D [K][P][L] in, beta [K][Tz] out, dtd [K][K][2L-1] out.
 *   beta_k[s] = sum_p sum_tau D_kp[tau] X_p[s + tau]  (cross-correlation).
 *   lambda_max_out: host pointer, may be NULL; when given, receives
 *   max |beta| and the call synchronises `stream`.
 *   workspace: device scratch of csc_workspace_size() bytes (holds the
 *   max |beta| reduction). */
CSC_API int csc_init_beta(const csc_shape *shape, const float *X, const float *D, float *beta,
                  float *dtd, double *lambda_max_out, void *workspace, size_t workspace_bytes,
                  csc_stream_t stream);

/* Convolutional sparse coding by LGCD (Alg. 1) over a grid of worker tiles
 * with the soft-lock rule (Alg. 3, Eq. soft_lock), one persistent CTA per tile.
 *   X, D     : the problem (needed to recompute beta from scratch at the end).
 *   dtd      : table from csc_init_beta.
 *   beta     : in: beta for the starting Z (from csc_init_beta when Z = 0);
 *              out: beta recomputed from scratch for the returned Z.
 *   Z        : out (zeroed by the call unless opts->warm_start).
 *   lambda   : absolute regularisation (not a fraction of lambda_max).
 *   tol      : eps of Alg. 1: the solve stops when no coordinate can change
 *              by tol or more; this is then re-checked on a fresh beta
 *              (stats->max_dz_final) and the solve resumes if it fails.
 *   stats    : host pointer, may be NULL.
 *   workspace: csc_workspace_size() bytes.  FP32 solves on tiles in global
 *              memory use its tail for the initial beta (the final beta is
 *              rebuilt from it and the nonzeros of Z), the table laid out for
 *              the staged window update and the bins of that rebuild; with
 *              less (but at least the required head) they recompute beta by
 *              correlation and read the table from L2 instead.  Such solves
 *              also need beta and Z on 16-byte boundaries (CSC_ERR_INVALID).
 * Synchronises `stream` before returning (the status comes from the device). */
CSC_API int csc_lgcd_solve(const csc_shape *shape, const float *X, const float *D, const float *dtd,
                   float *beta, float *Z, float lambda, float tol, const csc_solve_opts *opts,
                   void *workspace, size_t workspace_bytes, csc_solve_stats *stats,
                   csc_stream_t stream);

/* 1/2 ||X - Z*D||^2 + lambda ||Z||_1 accumulated in FP64 (Eq. csc).
 * objective_out is a host pointer; synchronises `stream`. */
CSC_API int csc_objective(const csc_shape *shape, const float *X, const float *D, const float *Z,
                  double lambda, double *objective_out, void *workspace,
                  size_t workspace_bytes, csc_stream_t stream);

/* Sufficient statistics of the dictionary update (Section 4.2, Eq. phi):
 *   phi_{k,k2}[delta] = sum_s Z_k[s] Z_k2[s + delta],  delta in prod ]-L_i, L_i[
 *   psi_kp[tau]       = sum_s Z_k[s] X_p[s + tau],     tau in Theta
 * computed from the nonzeros of Z.  phi [K][K][2L-1], psi [K][P][L] out.
 * Asynchronous. */
CSC_API int cdl_dict_stats(const csc_shape *shape, const float *Z, const float *X, float *phi,
                   float *psi, void *workspace, size_t workspace_bytes, csc_stream_t stream);

/* Dictionary step (Alg. 2): projected gradient descent on D with Armijo
 * backtracking, gradient phi * D - psi, projection D_k /= max(1, ||D_k||_2).
 * The first step is 1 / max_k sum_k2 sum_delta |phi_{k,k2}[delta]|, each later
 * iteration starts from twice the last accepted step; at most max_iter
 * iterations, stop when ||D+ - D|| < tol ||D||.  D is held in FP32, so a
 * relative change below 4 x 2^-24 cannot be resolved: a smaller tol acts as
 * 4 x 2^-24.  The step also stops when its FP32 estimate of ||D+ - D||^2
 * (from per-atom scalars) lies within its own rounding bound, where the
 * change can no longer be resolved.
 *   D: in/out.  x_sqnorm: ||X||_2^2.  objective_out: host pointer (may be
 *   NULL) receiving F(D) = 1/2||X - Z*D||^2 at the end (FP64);
 *   iterations_out: host pointer (may be NULL).
 * Synchronises `stream` when either output pointer is given. */
CSC_API int cdl_dict_update(const csc_shape *shape, const float *phi, const float *psi,
                    double x_sqnorm, float *D, int max_iter, double tol,
                    double *objective_out, int *iterations_out, void *workspace,
                    size_t workspace_bytes, csc_stream_t stream);

/* Convolutional dictionary learning, the outer loop of Alg. 2: repeat
 *   Z <- csc_lgcd_solve(X, D) from Z = 0, lambda = reg * lambda_max(X, D0)
 *        fixed at the first iteration;
 *   phi, psi <- cdl_dict_stats(Z, X);
 *   D <- cdl_dict_update(phi, psi) (pgd_max_iter, pgd_tol)
 * until the cost 1/2||X - Z*D||^2 + lambda ||Z||_1 after the dictionary step
 * changes by less than nu (relative) or max_outer iterations are done.
 *   D: in (D0) / out.  Z, beta, dtd, phi, psi: caller-owned buffers of the
 *   layouts above (outputs of the last iteration).
 *   trace: host array of 2 * max_outer doubles (may be NULL): the cost after
 *   the CSC step and after the dictionary step of every iteration, both from
 *   the residual with FP64 sums (as csc_objective).
 *   n_outer: host int (may be NULL): iterations made.
 * Synchronises `stream` several times per iteration.  Returns
 * CSC_NOT_CONVERGED if some CSC step did not reach tol. */
CSC_API int cdl_fit(const csc_shape *shape, const float *X, float *D, float *Z, float *beta, float *dtd,
                    float *phi, float *psi, double reg, double tol, int max_outer, double nu,
                    int pgd_max_iter, double pgd_tol, const csc_solve_opts *opts, void *workspace,
                    size_t workspace_bytes, double *trace, int *n_outer, csc_stream_t stream);

/* One pass of the loop body of Alg. 2 as a single call:
 *   beta, dtd <- csc_init_beta(X, D) (csc_init_beta_bf16x3 when lambda is
 *        given and opts->beta_init = 1);
 *   lambda: the given one when lambda > 0 (reg is then ignored), so that the
 *        calls of an outer loop solve one fixed problem; otherwise
 *        reg * lambda_max(X, D) from the FP32 beta-init (rounded to float as
 *        csc_lgcd_solve receives it);
 *   Z <- csc_lgcd_solve(X, D, lambda, tol, opts) (from Z = 0 unless
 *        opts->warm_start);
 *   phi, psi <- cdl_dict_stats(Z, X);
 *   D <- cdl_dict_update(phi, psi, x_sqnorm) (pgd_max_iter, pgd_tol).
 * Same buffers, layouts and results as those calls; between the statistics
 * and the dictionary step nothing waits for the device (the nonzero count is
 * read back once, with the dictionary step's results).
 *   D: in / out.  Z, beta, dtd, phi, psi: outputs.  x_sqnorm: ||X||_2^2, or a
 *   negative value to have it summed on the device (FP64).
 *   stats: the solve's statistics (may be NULL).  lambda_out (the lambda
 *   used), dict_cost_out (F(D) after the step, as cdl_dict_update's
 *   objective_out) and dict_iters_out: host pointers (may be NULL).
 * Synchronises `stream` two or three times (lambda_max when it is computed,
 * the end of the solve, the end of the step).  Returns the solve's status
 * (CSC_OK or CSC_NOT_CONVERGED; the dictionary step still ran),
 * CSC_ERR_INVALID for neither lambda > 0 nor reg > 0, CSC_ERR_WORKSPACE when
 * Z has more nonzeros than the workspace's list holds (phi and psi are then
 * not valid and D is left unchanged), or the first error of a stage. */
CSC_API int cdl_step(const csc_shape *shape, const float *X, float *D, float *Z, float *beta, float *dtd,
                     float *phi, float *psi, double reg, double lambda, double tol, double x_sqnorm,
                     int pgd_max_iter, double pgd_tol, const csc_solve_opts *opts, void *workspace,
                     size_t workspace_bytes, csc_solve_stats *stats, double *lambda_out,
                     double *dict_cost_out, int *dict_iters_out, csc_stream_t stream);

/* csc_init_beta with the correlation on the tensor cores (tcgen05) in
 * split-bf16 precision: each X and D value is split into bf16 hi + lo parts
 * and beta accumulates hi*hi + hi*lo + lo*hi in FP32 (the mixed-precision
 * beta-init of Alg. 1's initialisation).  Elementwise
 *   |beta - beta_exact| <= (2^-16 + 2 gamma_n) sum_p sum_tau |D_kp[tau]| |X_p[s+tau]|,
 * n = P L0 roundup(L1, 16).  dtd is computed in FP32 as in csc_init_beta.
 * lambda_max_out (may be NULL) receives max |beta| of this beta (same error
 * bound); the call then synchronises `stream`.  Returns CSC_ERR_UNIMPLEMENTED
 * when the split dictionary (4 x roundup(K, 16) x P L0 roundup(L1, 16) bytes)
 * and two operand chunks do not fit in one CTA's shared memory or K > 256,
 * CSC_ERR_TIMEOUT when a device wait gave up. */
CSC_API int csc_init_beta_bf16x3(const csc_shape *shape, const float *X, const float *D, float *beta,
                                 float *dtd, double *lambda_max_out, void *workspace,
                                 size_t workspace_bytes, csc_stream_t stream);

/* beta recomputed from scratch for a given Z (Eq. beta_update's invariant:
 * beta_k = D~_k * (X - Z*D) + ||D_k||^2 Z_k), with max |dZ| over every
 * coordinate (the KKT test of Alg. 1's stop) and the objective of Eq. csc,
 * both accumulated from FP64 sums.  beta: out.  max_dz_out, objective_out:
 * host pointers (may be NULL); the call synchronises `stream`. */
CSC_API int csc_refresh_beta(const csc_shape *shape, const float *X, const float *D, const float *Z,
                             float lambda, float *beta, double *max_dz_out, double *objective_out,
                             void *workspace, size_t workspace_bytes, csc_stream_t stream);

/* Coordinate descent in a given order on one worker: the randomized
 * baseline (RCD) of the coordinate-selection comparison (Section 5.1) when
 * the order is drawn at random.  For each flat index c = k |Omega| + s of
 * coords[0..n) (device, uint32) in turn, Z_k[s] <- ST(beta_k[s], lambda) /
 * ||D_k||^2 (Eq. pb_coord) with the beta update of Eq. beta_update when the
 * value changes -- the same result as one coordinate at a time.  beta, Z:
 * in/out, a consistent state (Z = 0 with beta from csc_init_beta for a cold
 * start); dtd from csc_init_beta.  updates_out (host, may be NULL): the
 * number of coordinates that changed.  Synchronises the stream.
 * CSC_ERR_INVALID for an index outside K x Omega (the walk stops there);
 * CSC_ERR_TIMEOUT after 60 s.  Greedy CD and cyclic CD need no separate
 * call: csc_lgcd_solve with one worker and one sub-domain covering the domain
 * (greedy) or sub-domains of one position (cyclic) (Section 3). */
CSC_API int csc_rcd_solve(const csc_shape *shape, const float *D, const float *dtd, float *beta, float *Z,
                          float lambda, const unsigned *coords, long long n, long long *updates_out,
                          void *workspace, size_t workspace_bytes, csc_stream_t stream);

/* Batched solves: many images of uneven size in one persistent launch.
 * A persistent grid (two or three CTAs of 256 threads per SM) takes the tiles of queued
 * images (jobs) in order and runs the global-memory LGCD worker (Alg. 3) on
 * each; an image starts when all of its tiles are held.  Images share the atom
 * shape, the resident dictionary D and its D^T D table.  Jobs are appended
 * while the kernel runs; completion is reported through pinned host memory.
 * Every device wait is bounded by run_seconds. */
typedef struct csc_queue csc_queue;

/* Device and pinned-host workspace for a queue (atoms: d = 2, P, K, L; T is
 * ignored) holding up to max_jobs jobs in total, ctl_slots of them at once,
 * with the given grid density (as for csc_queue_create). */
CSC_API int csc_queue_workspace_size(const csc_shape *atoms, int max_jobs, int ctl_slots, int ctas_per_sm,
                                     size_t *device_bytes, size_t *host_bytes);

/* Start the persistent kernel on kernel_stream.  D [K][P][L0][L1] and dtd
 * (from csc_init_beta) stay resident and must outlive the queue.
 * device_workspace: caller-owned device memory; host_workspace: caller-owned
 * pinned host memory the device can write (cudaHostAlloc / pinned tensors).
 * side_stream carries the control copies.  Both streams must be distinct and
 * created with cudaStreamNonBlocking (CSC_ERR_INVALID otherwise): the kernel
 * runs until csc_queue_close, and the legacy default stream waits for every
 * blocking stream.  The kernel takes the largest shared-memory carveout, and
 * the library's beta-init, refresh and objective kernels are loaded before it
 * starts, so that they run beside it on every SM.  Other kernels that first
 * load while the queue runs may wait for it to end (lazy module loading). 
 * opts: tile / sub-domain sizes, mode, timeout of each solve (may be NULL).
 * ctas_per_sm: 2 (0 = default) leaves each SM room for the tensor-core
 * beta-init (csc_init_beta_bf16x3) beside the queue; 3 runs more tiles at
 * once but leaves room only for the FP32 calls (csc_init_beta,
 * csc_refresh_beta, csc_objective) -- a bf16x3 beta-init launched beside it
 * would wait for the queue to end.  Other values: CSC_ERR_INVALID.
 * The library allocates only the host-side handle. */
CSC_API int csc_queue_create(const csc_shape *atoms, const float *D, const float *dtd,
                             const csc_solve_opts *opts, int max_jobs, int ctl_slots, int ctas_per_sm,
                             void *device_workspace, size_t device_bytes, void *host_workspace,
                             size_t host_bytes, double run_seconds, csc_stream_t kernel_stream,
                             csc_stream_t side_stream, csc_queue **queue_out);

/* csc_queue_create without starting the kernel: jobs may then be submitted
 * (csc_queue_submit) before csc_queue_start launches it.  With every job
 * published before the launch, the queue needs no concurrency between the
 * host's copies and the running kernel -- it runs the same way when kernels
 * are serialised (a profiler that replays them one at a time).  Same
 * arguments, ownership and errors as csc_queue_create. */
CSC_API int csc_queue_create_deferred(const csc_shape *atoms, const float *D, const float *dtd,
                                      const csc_solve_opts *opts, int max_jobs, int ctl_slots,
                                      int ctas_per_sm, void *device_workspace, size_t device_bytes,
                                      void *host_workspace, size_t host_bytes, double run_seconds,
                                      csc_stream_t kernel_stream, csc_stream_t side_stream,
                                      csc_queue **queue_out);

/* Launch the kernel of a queue made by csc_queue_create_deferred.  drain = 1:
 * the kernel ends by itself once every job submitted before this call is done,
 * and later csc_queue_submit calls return CSC_ERR_INVALID; drain = 0: the
 * kernel keeps taking jobs until csc_queue_close, as after csc_queue_create.
 * CSC_ERR_INVALID for a queue already running or another drain value. */
CSC_API int csc_queue_start(csc_queue *queue, int drain);

/* Queue one image of T0 x T1 samples: beta [K][Z0][Z1] must hold D~ * X (from
 * csc_init_beta, or a consistent warm state with warm_start = 1, in which
 * case Z is kept; otherwise Z is zeroed).  beta and Z belong to the caller and
 * are updated in place until the job completes.  job_out: index for
 * csc_queue_poll.  opts (may be NULL: the queue's) sets this job's tile and
 * sub-domain sizes, mode, stop margin and timeout; the image is cut into at
 * most opts.max_workers tiles (default: 7/8 of the grid, so that small jobs
 * start beside a large one).
 * CSC_ERR_WORKSPACE when max_jobs or ctl_slots is used up (poll finished
 * jobs to free control slots). */
CSC_API int csc_queue_submit(csc_queue *queue, int T0, int T1, float *beta, float *Z, float lambda,
                             float tol, int warm_start, const csc_solve_opts *opts, int *job_out);

/* 1 when the job has completed (stats filled: status, updates, iterations,
 * rejected, messages, device time in kernel_ms), 0 while it runs, negative
 * status on a bad argument.  Host-only, no CUDA call. */
CSC_API int csc_queue_poll(csc_queue *queue, int job, csc_solve_stats *stats);

/* The device-side state of a job, for diagnosing a stalled queue: out[8] =
 * {first slot, tiles W, tiles taken, tiles finished, jobs published, next
 * slot, grid size, completion word}.  Synchronises the side stream. */
CSC_API int csc_queue_inspect(csc_queue *queue, int job, long long *out);

/* No more jobs: wait until the queue drains, stop the kernel, release the
 * handle (a queue that was never started: just the handle). */
CSC_API int csc_queue_close(csc_queue *queue);

/* FP64 variants of csc_init_beta and csc_lgcd_solve (same layouts, double
 * elements).  They exist to verify the tiled schedule exactly against an FP64
 * reference; they are slow on GB300, whose FP64 rate is low. */
CSC_API int csc_init_beta_f64(const csc_shape *shape, const double *X, const double *D, double *beta,
                      double *dtd, double *lambda_max_out, void *workspace,
                      size_t workspace_bytes, csc_stream_t stream);
CSC_API int csc_lgcd_solve_f64(const csc_shape *shape, const double *X, const double *D,
                       const double *dtd, double *beta, double *Z, double lambda, double tol,
                       const csc_solve_opts *opts, void *workspace, size_t workspace_bytes,
                       csc_solve_stats *stats, csc_stream_t stream);

/* cdl_dict_stats for callers that cannot allocate device memory.  The paper
 * has no counterpart to this call; it exists for embedders that cannot give
 * the library a workspace at the time they need the statistics -- for example
 * a plugin inside an application that owns every device allocation, or a
 * service that reserves all of its device memory at start-up and allocates
 * nothing afterwards.
 *   Same arguments, layouts and results as cdl_dict_stats, without the
 *   workspace: the scratch is a fixed array of CSC_NOALLOC_SCRATCH_BYTES that
 *   the library keeps on every GPU that loads it until the process exits.
 *   The call allocates nothing (no cudaMalloc/cudaFree, no allocating library
 *   routine).
 *   Returns CSC_ERR_WORKSPACE when the problem needs more scratch than the
 *   array holds: the FP64 accumulators of phi and psi and a control block
 *   take their share, and the rest of the array holds the nonzero list of Z
 *   (12 bytes per nonzero, about 690,000 nonzeros for small atoms); a Z with
 *   more nonzeros than that is refused after the count.
 *   The first call on a device (and the first after that device's context
 *   was reset or created anew) looks up the array's device address; make that
 *   first call before any stream capture.  All calls share the one array:
 *   calls whose work overlaps on the GPU (different streams, different host
 *   threads) race and must be serialised by the caller.  Like cdl_dict_stats,
 *   it synchronises `stream` once to check the nonzero count. */
#define CSC_NOALLOC_SCRATCH_BYTES (8u << 20)
CSC_API int cdl_dict_stats_noalloc(const csc_shape *shape, const float *Z, const float *X, float *phi,
                                   float *psi, csc_stream_t stream);

/* The sparse code: the nonzeros of Z (the activations of Eq. csc) as a list
 * in (position, atom) order -- positions ascending, atoms ascending within a
 * position.  Entry i is atom k_out[i], position s_out[i] in atom k's plane
 * (i0 * Z1 + i1 in 2-D, the time index in 1-D) and value val_out[i].
 *   Z: device, K x Z0 x Z1 FP32.  k_out, s_out, val_out: device arrays of cap
 *   entries owned by the caller (may be NULL when cap = 0).  nnz_out: host,
 *   receives the number of nonzeros.  workspace: at least
 *   csc_workspace_size bytes (block counts and the header).
 * Synchronises `stream` once to read the count.  Returns CSC_ERR_WORKSPACE,
 * with *nnz_out set and nothing written, when the count exceeds cap (call
 * again with a larger cap, or with cap = 0 to count only). */
CSC_API int csc_sparse_code(const csc_shape *shape, const float *Z, int *k_out, int *s_out, float *val_out,
                            long long cap, long long *nnz_out, void *workspace, size_t workspace_bytes,
                            csc_stream_t stream);

/* Human-readable name of a status code (static storage). */
CSC_API const char *csc_status_string(int status);

/* The last CUDA error code seen by this library on this thread (0 if none). */
CSC_API int csc_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DICODILE_GB_H */
