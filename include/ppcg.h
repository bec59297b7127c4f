/*
 * ppcg.h -- C ABI of a single-GPU pipelined preconditioned conjugate gradient solver
 * for sparse SPD systems A x = b (NVIDIA B300, sm_103a).
 *
 * Method: Algorithm 2 (pipelined PCG, Ghysels-Vanroose form) of Tiwari & Vadhiyar,
 * "Efficient executions of Pipelined Conjugate Gradient Method on Heterogeneous
 * Architectures", arXiv 2105.06176, Sec. III-B, with the Jacobi preconditioner
 * M = diag(A) and the CSR input format of Sec. V-A.  Every iteration runs on the GPU:
 * one fused pass computes n = A M^-1 w for its rows and updates z, q, s, p, x, r, u, w
 * (the algorithm's vector updates, preconditioner and SpMV), emitting block partials of
 * gamma = (r, u), delta = (w, u) and the stopping norm; alpha and beta are
 * formed on the device, so the host never waits inside a solve.
 *
 * Conventions shared by every call:
 *   - Indices are 0-based.  Matrices are full (not triangular) CSR with int64 row
 *     pointers, int32 column indices and FP64 values.  Symmetry is assumed, not checked.
 *   - Pointers marked "host or device" may be either; the library detects which
 *     (cudaPointerGetAttributes) and stages host data through its own device buffers.
 *   - Calls that take a cudaStream_t are stream-ordered and asynchronous: argument errors
 *     are returned immediately; numerical results (ppcg_info) become valid once the stream
 *     has been synchronised.  A NULL stream means the legacy default stream.
 *   - A handle is not thread-safe; its solves must be ordered on one stream (or the caller
 *     must synchronise between streams).  Server calls are thread-safe.
 *   - The library owns every device buffer it allocates and frees it in the matching
 *     destroy call.  It never frees caller memory.
 */
#ifndef PPCG_H
#define PPCG_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ppcg_ctx* ppcg_handle;
typedef struct ppcg_srv* ppcg_server;

typedef enum {
  PPCG_OK = 0,
  PPCG_PENDING = 1,            /* ppcg_poll: request not finished yet */
  PPCG_ERR_ARG = -1,           /* invalid argument (sizes, NULL pointers, unsorted row_ptr, column out of range) */
  PPCG_ERR_NOT_SPD = -2,       /* a diagonal entry is missing or not positive (Jacobi needs a_ii > 0) */
  PPCG_ERR_BREAKDOWN = -3,     /* gamma <= 0 or alpha denominator (delta - beta*gamma/alpha_prev) <= 0 */
  PPCG_ERR_NOT_CONVERGED = -4, /* maxit reached; x holds the last iterate */
  PPCG_ERR_NONFINITE = -5,     /* gamma or delta became NaN/Inf */
  PPCG_ERR_OOM = -6,           /* device allocation failed or the server's HBM budget is too small */
  PPCG_ERR_CUDA = -7,          /* a CUDA runtime call failed (message via ppcg_last_error) */
  PPCG_ERR_TIMEOUT = -8,       /* a device-side barrier wait exceeded its time limit */
  PPCG_ERR_BUSY = -9,          /* server queue full */
  PPCG_ERR_UNKNOWN_TICKET = -10
} ppcg_status;

typedef enum {
  PPCG_FP64 = 0,     /* every vector and the matrix in FP64 */
  PPCG_FP32_IR = 1,  /* FP32 inner solves inside FP64 iterative refinement (restarted per step) */
  PPCG_FP32_RU = 2   /* FP32 recurrences with FP64 reliable updates (one Krylov sequence) */
} ppcg_precision;
typedef enum {
  PPCG_FMT_AUTO = 0,  /* SELL-C-sigma; a constant-coefficient box stencil on the grid path is
                         detected and run matrix-free (see PPCG_FMT_BOX) */
  PPCG_FMT_CSR = 1,   /* SELL-C-sigma with sigma = 1 (CSR row order kept) */
  PPCG_FMT_SELL = 2,  /* SELL-C-sigma, never matrix-free */
  PPCG_FMT_BOX = 3    /* matrix-free: A = c_d I + c_o (adjacency of the (2R+1)^3 box, R <= 3, on a
                         g^3 grid, truncated at the boundary, rows in grid order, x fastest) -- the
                         125-point Poisson family of Table II for R = 2.  A v is formed from axis-wise
                         box sums of v, no matrix is read.  FP64 Alg. 2 on the grid path; a matrix of
                         another form gives PPCG_ERR_ARG */
} ppcg_format;
typedef enum {
  PPCG_NORM_REL_R = 0,      /* ||r||_2 <= tol * ||b||_2 on the recursive residual, then a true-residual check */
  PPCG_NORM_PAPER_U_ABS = 1 /* sqrt((u, u)) <= tol, the absolute preconditioned norm of Alg. 2 / Sec. VI */
} ppcg_norm;
typedef enum {
  PPCG_PATH_AUTO = 0,
  PPCG_PATH_GRID = 1,     /* one cooperative persistent launch over the whole GPU */
  PPCG_PATH_CLUSTER = 2,  /* one 8-CTA thread-block cluster, vectors in global memory */
  PPCG_PATH_ONCHIP = 3    /* one 8-CTA cluster holding the whole system (vectors and matrix) in its
                             distributed shared memory; FP64 Alg. 2 only, systems up to about
                             11-12 thousand rows of a 3-D 7-point stencil */
} ppcg_path;
typedef enum {
  PPCG_VARIANT_ALG2 = 0,          /* Alg. 2 as printed: u and q carried by their recurrences */
  PPCG_VARIANT_JACOBI_SCALED = 1  /* Jacobi elimination: with M = diag(A), u = M^-1 r and q = M^-1 s hold
                                     exactly, so the solver runs the same iteration on D^-1/2 A D^-1/2
                                     (u = r, q = s, m = w there): six vectors per row instead of eight,
                                     no M^-1 stream, fewer FP64 operations; alpha, beta and x are those
                                     of Alg. 2 up to rounding.  FP64 precision only. */
} ppcg_variant;

/* Solver options.  Obtain defaults with ppcg_opts_default and override fields. */
typedef struct {
  int32_t precision;        /* ppcg_precision.  FP32_IR: FP32 matrix values and vectors inside an
                               FP64 iterative-refinement loop (FP64 outer residual and solution);
                               a refinement step that does not halve the FP64 residual is undone
                               and the solve continues with the FP64 iteration.
                               FP32_RU: one pipelined iteration whose vectors and matrix values
                               are FP32; the solution is accumulated in FP64, and a reliable
                               update (FP64 residual b - A x, FP32 recurrences restarted from it,
                               search direction kept) runs every rr_period iterations, whenever
                               the recursive residual has fallen by inner_tol since the last one,
                               and whenever it passes the stopping test, which the FP64 residual
                               then decides.  Three updates in a row where the recursion claims
                               a 4x fall and the FP64 residual does not halve, a non-finite
                               value, or a breakdown past max_restarts switch to the FP64
                               iteration from the last updated x.  REL_R norm only. */
  int32_t format;           /* ppcg_format.  The matrix is converted to SELL-C-sigma (C = 32) on the
                               device; FMT_CSR forces sigma = 1 (CSR row order kept); FMT_BOX and
                               AUTO's detection use the matrix-free box product instead. */
  int32_t norm;             /* ppcg_norm */
  int32_t path;             /* ppcg_path.  AUTO: ONCHIP when the system fits (FP64 Alg. 2), else
                               CLUSTER up to cluster_max_rows rows, else GRID.  ONCHIP for a system
                               that does not fit gives PPCG_ERR_ARG. */
  int32_t sigma;            /* SELL sorting window in rows (1 = no sorting; 0 = autotune over
                               {1, 256, 2048}: padded matrix bytes plus a gather-locality cost
                               for sorted windows, whose chunks mix rows from all over the window) */
  int32_t rr_period;        /* residual replacement every rr_period iterations.  FP64: 0 = only when the
                               recursive residual passes but the true residual does not.  FP32_IR: the
                               period inside each inner solve, 0 = 25.  FP32_RU: the iterations
                               between reliable updates, 0 = 15 */
  double inner_tol;         /* FP32_IR: relative residual reduction asked of each inner solve.
                               FP32_RU: the fall of the recursive residual that triggers a
                               reliable update */
  int32_t inner_maxit;      /* FP32_IR: iteration cap of one inner solve */
  int32_t max_outer;        /* FP32_IR: cap on refinement steps */
  int64_t spin_limit_ns;    /* time limit of one device-side barrier wait (ns); exceeded -> TIMEOUT */
  int32_t cluster_max_rows; /* PATH_AUTO: systems with at most this many rows take the CLUSTER path */
  int32_t epoch_iters;      /* server: iterations per epoch of a 131072-row solve; a solve of n rows
                               advances epoch_iters * 131072 / n (clamped to [2, 64 epoch_iters]) */
  int32_t max_restarts;     /* restarts after a breakdown (alpha denominator <= 0 past the first
                               iteration): true residuals, direction recurrences reset, beta = 0.
                               0 = report PPCG_ERR_BREAKDOWN instead.  FP32_IR: per inner solve
                               (an inner breakdown past the restarts ends that inner solve) */
  int32_t variant;          /* ppcg_variant */
  double gap_theta;         /* FP64 iteration (also the FP32 forms' FP64 fallback): measured-gap
                               residual replacement, from the accuracy criterion of the pipelined-CG
                               literature (not in the paper).  Whenever gamma = (r, M^-1 r) has fallen
                               by the factor gap_fall since the residuals were last measured or
                               replaced, one extra pass measures ||(b - A x) - r||, the deviation of
                               the recursive residual from the true one; when it exceeds
                               gap_theta * ||r||, the residuals are replaced (r, u, w, s, q, z
                               recomputed from x and p; alpha and beta keep their recurrences).
                               Replacing while that deviation is small keeps the recurrences
                               consistent: a replacement made only once the recursive residual has
                               passed the stopping test can change r by a percent or more, after which
                               the iteration can grow until the alpha denominator breaks down.
                               0 = 1e-6; negative = off */
  int32_t gap_fall;         /* the fall of gamma between two measurements; 0 = 100 (the residual
                               norm about 10x) */
  int32_t cluster_ctas;     /* CLUSTER path: CTAs per system (thread-block cluster size 2, 4, 8 or 16;
                               default 8).  0 = tuned at create: a few iterations of the system are
                               timed on the device with 2, 4 and 8 CTAs and the size with the least
                               CTA-time per iteration wins (the largest within 10% of it), cached per
                               family signature and size bucket.  Fixed for the handle, so a system's
                               result is the same solo and in a batch.  A batch runs one launch per
                               cluster size among its handles: batches of small systems gain from
                               tuning (1e3-3e3 rows: 1.36x FP64, 1.46x FP32_RU on B300), a batch that
                               mixes sizes gains nothing (it is bandwidth-bound and one launch of one
                               size serves it best).  The server uses 8 */
} ppcg_opts;

/* Per-solve results.  Filled asynchronously; valid after the solve's stream is synchronised. */
typedef struct {
  int32_t status;            /* ppcg_status */
  int32_t iters;             /* iterations of Alg. 2 (executions of the vector-update block); FP32_IR:
                                summed over inner solves */
  int32_t outer_iters;       /* FP32_IR refinement steps; FP32_RU FP64 residual evaluations (0 for FP64) */
  int32_t rr_count;          /* residual replacements performed (restarts included) */
  double rel_res_recursive;  /* stopping norm at exit, divided by ||b|| (REL_R) or absolute (PAPER_U_ABS) */
  double rel_res_true;       /* ||b - A x||_2 / ||b||_2 at exit, FP64 (0 when b = 0) */
  double seconds;            /* device time of the solve (globaltimer), setup and final residual included */
  double bytes_per_iter;     /* algorithmic bytes of one iteration, v = 8 (FP64) or 4 (FP32 modes):
                                (v+4) nnz + 4 (N+1) + 17 v N (matrix values and columns, row
                                pointers, 17 vector streams); Jacobi-scaled: (v+4)(nnz - N) +
                                4 (N+1) + 13 v N; matrix-free box stencil: 21 v N (17 vector
                                streams and two stage arrays).  SELL padding is not counted. */
  double bnorm;              /* ||b||_2 */
  int32_t fp64_fallback;     /* FP32_IR: 1 when a refinement step failed to halve the FP64 residual and
                                the solve finished with the FP64 iteration from the previous x;
                                FP32_RU: 1 when the solve finished with the FP64 iteration */
  int32_t reserved;
} ppcg_info;

/* Fill *opts with defaults: FP64, AUTO format/path, REL_R, sigma autotune, rr_period 0,
 * inner_tol 1e-2, inner_maxit 2000, max_outer 100, spin_limit 10 s, cluster_max_rows 16384,
 * epoch_iters 256, max_restarts 8. */
void ppcg_opts_default(ppcg_opts* opts);

/*
 * Create a solver for the n x n SPD matrix given in CSR (Sec. V-A).
 *   row_ptr [n+1] int64, col [nnz] int32, val [nnz] FP64: host or device, caller-owned;
 *   copied during the call, so the caller may free them when it returns.
 *   opts may be NULL (defaults).  stream orders the conversion work; the call synchronises
 *   that stream before returning, so the handle is ready to use on any stream.
 * The matrix is validated (monotone row_ptr, columns in range), the Jacobi diagonal
 * extracted (missing or non-positive -> PPCG_ERR_NOT_SPD), and the values pre-scaled
 * column-wise to A D^-1 and converted to SELL-C-sigma on the device.  The execution path
 * (opts->path) is fixed here for every later solve of the handle.
 * Errors: PPCG_ERR_ARG, PPCG_ERR_NOT_SPD, PPCG_ERR_OOM, PPCG_ERR_CUDA; *handle is then NULL.
 */
ppcg_status ppcg_create(ppcg_handle* handle, int64_t n, int64_t nnz, const int64_t* row_ptr,
                        const int32_t* col, const double* val, const ppcg_opts* opts,
                        cudaStream_t stream);

/*
 * Solve A x = b with Alg. 2 (Sec. III-B) to the stopping test of opts.norm with tolerance
 * tol, at most maxit iterations.
 *   b [n]  host or device, read only.  b = 0 gives x = 0, 0 iterations, PPCG_OK (REL_R).
 *   x0 [n] host or device initial guess, or NULL for zero.  May alias x.
 *   x [n]  host or device output.  Written on every outcome except argument errors.
 *   info   host pointer or NULL; valid after the stream is synchronised.  A non-NULL info is
 *          filled by a host function enqueued on the stream, which holds the stream for tens
 *          to hundreds of microseconds; with NULL the solve's record is only copied into the
 *          handle's pinned staging buffer, and ppcg_last_info reads it after the sync.
 * Returns PPCG_OK when the work was enqueued (numerical status goes to info->status), or
 * PPCG_ERR_ARG / PPCG_ERR_OOM / PPCG_ERR_CUDA immediately.
 * With host b/x the call copies through device staging buffers on the stream.
 */
ppcg_status ppcg_solve(ppcg_handle handle, const double* b, const double* x0, double* x,
                       double tol, int32_t maxit, cudaStream_t stream, ppcg_info* info);

/*
 * The result record of the handle's most recent solve (ppcg_solve or ppcg_batch_solve), read
 * from the pinned staging buffer that solve's stream-ordered copies wrote: call it after that
 * stream has been synchronised (it makes no CUDA call and does not wait).  For solves
 * enqueued with info == NULL this is how the caller gets the status, iteration count and
 * residuals without the stream-held host function.
 *   info   host pointer, written with the same fields ppcg_solve's info would hold.
 * Returns PPCG_OK, or PPCG_ERR_ARG for a NULL handle or info or a handle that has not
 * solved yet.
 */
ppcg_status ppcg_last_info(ppcg_handle handle, ppcg_info* info);

/*
 * Solve count independent systems, each with its own handle, in as few launches as the
 * handles' paths allow: every CLUSTER-path system runs inside one persistent launch of
 * thread-block clusters (a host-side longest-first schedule spreads them over the
 * clusters); ONCHIP-path systems run in one launch of on-chip clusters on a side stream,
 * overlapping it; GRID-path systems run one after another over the whole GPU.
 * b[i], x0[i] (or NULL, or x0 == NULL for all zero), x[i]: DEVICE pointers.
 * tol[i], maxit[i] per system; infos[count] host array or NULL.
 * Each result is bitwise identical to ppcg_solve on the same handle: a system's
 * partition over CTAs and its reduction order depend only on its handle.
 * The handles must be distinct.  Returns after enqueueing; infos valid after stream sync.
 * CLUSTER-path handles with different cluster sizes (ppcg_opts.cluster_ctas) run one launch
 * per size, largest first, the later ones on library side streams joined back into
 * `stream`; ON-CHIP members run on another side stream.  Those side streams and their
 * events are per device, so calls of ppcg_batch_solve on one device from several host
 * threads must not overlap.
 */
ppcg_status ppcg_batch_solve(int32_t count, const ppcg_handle* handles, const double* const* b,
                             const double* const* x0, double* const* x, const double* tol,
                             const int32_t* maxit, cudaStream_t stream, ppcg_info* infos);

/* The execution plan ppcg_create chose for a handle (fixed for the handle's lifetime). */
typedef enum {
  PPCG_COLS_SELL = 0,      /* SELL-C-sigma, 4-byte column per slot */
  PPCG_COLS_DICT = 1,      /* SELL-C-sigma; the iteration pass reads a one-byte index per slot into the
                              matrix's few distinct col - row offsets */
  PPCG_COLS_PATTERN = 2,   /* offset pattern: every row's off-diagonal columns are an ascending subset of
                              row + pat[0..pattern_k); pattern_k slots per row (zeros where a neighbour is
                              absent), and every pass forms the columns instead of reading them */
  PPCG_COLS_MATRIX_FREE = 3  /* the constant-coefficient box stencil of PPCG_FMT_BOX: no matrix is read */
} ppcg_columns;
typedef struct {
  int32_t path;             /* ppcg_path taken (never AUTO) */
  int32_t columns;          /* ppcg_columns of the kernel running the iteration (the pattern and the
                               dictionary have grid-path kernels; a pattern matrix is also a valid SELL
                               matrix, whose stored columns the cluster and on-chip kernels read) */
  int32_t sigma;            /* SELL sorting window (1 = rows in CSR order) */
  int32_t pattern_k;        /* offsets in the pattern (0: none) */
  int32_t dict_size;        /* offsets in the column dictionary (0: none) */
  int32_t ctas;             /* CTAs of one solve's launch (grid path), or of its cluster */
  int64_t slots;            /* SELL slots stored, padding included */
  double padding;           /* padded slots / off-diagonal nonzeros */
  double convert_seconds;   /* CSR -> SELL conversion on the device (the paper keeps CSR, Sec. V-A, to avoid
                               this cost; it is paid once per handle here) */
  double create_seconds;    /* the whole ppcg_create: staging, validation, conversion, detection, workspace */
  double bytes_per_iter;    /* algorithmic bytes of one iteration, as in ppcg_info */
} ppcg_plan;

/*
 * Report the plan of a handle (host only, no CUDA call).  Returns PPCG_OK, or PPCG_ERR_ARG
 * for a NULL handle or plan.  The paper has no counterpart: it describes the conversion
 * cost that its CSR choice avoids (Sec. V-A); this is where the library states its own.
 */
ppcg_status ppcg_plan_info(ppcg_handle handle, ppcg_plan* plan);

/* Destroy a handle (synchronises its last stream first).  NULL is ignored. */
void ppcg_destroy(ppcg_handle handle);

/*
 * Continuous-batching server.  Admission runs on two background threads, one for requests
 * of up to cluster_max_rows rows and one for larger ones.  Each takes its requests in
 * arrival order while their device footprint fits in hbm_budget bytes (0 = 90% of free HBM
 * at creation); an older request of the other class that is waiting for memory keeps its
 * turn.  Admitted requests keep their vectors and scalars resident on the device and
 * advance together in epochs of a bounded number of iterations, so requests that arrive
 * while others run join at the next epoch.  opts may be NULL.  With opts->path ==
 * PPCG_PATH_AUTO and the default cluster_max_rows, requests of up to 131,072 rows run on
 * the CLUSTER path (all of them share one launch per epoch) and larger ones on the GRID
 * path (the two oldest advance each epoch by a slice of about 5-10 ms); the ONCHIP path is
 * not used by the server.  Each epoch runs the cluster launch first and then those slices.
 * A small request therefore never waits for a large solve to finish, nor for the copy and
 * conversion of a large request's matrix: once admitted, it waits at most for the slices
 * of the epoch in progress.  A solve's result equals ppcg_solve on a handle created with
 * the same options and that path.
 */
ppcg_status ppcg_server_create(ppcg_server* server, size_t hbm_budget, const ppcg_opts* opts);

/*
 * Queue one solve and return at once with a ticket.  All pointers are HOST pointers
 * (copied before the call returns): CSR as in ppcg_create, b [n], x0 [n] or NULL.
 * Errors: PPCG_ERR_ARG, PPCG_ERR_BUSY (queue full), PPCG_ERR_OOM (larger than the budget).
 */
ppcg_status ppcg_submit(ppcg_server server, int64_t n, int64_t nnz, const int64_t* row_ptr,
                        const int32_t* col, const double* val, const double* b, const double* x0,
                        double tol, int32_t maxit, uint64_t* ticket);

/*
 * Poll a ticket.  Returns PPCG_PENDING while queued or running; otherwise the solve's
 * status (also in info->status), copies the solution into x_out [n] (host, may be NULL)
 * and forgets the ticket.  Unknown tickets -> PPCG_ERR_UNKNOWN_TICKET.
 */
ppcg_status ppcg_poll(ppcg_server server, uint64_t ticket, double* x_out, ppcg_info* info);

/* Server counters: completed solves, admitted-but-running, queued, bytes of HBM in use. */
ppcg_status ppcg_server_stats(ppcg_server server, int64_t* completed, int64_t* running,
                              int64_t* queued, int64_t* hbm_in_use);

/* Stop the server thread, drop unfinished requests and free everything.  NULL is ignored. */
void ppcg_server_destroy(ppcg_server server);

/*
 * Failure-detection self test.  The paper has no counterpart: it checks the bounded wait
 * of the device-side grid barrier that separates the passes of a GRID-path solve.  Runs
 * that barrier over `grid` co-resident CTAs (cooperative launch) with CTA `drop_rank`
 * exiting without arriving; every other CTA must stop waiting after limit_ns and report a
 * timeout instead of hanging.  Synchronous.  *timed_out receives the number of CTAs that
 * reported the timeout (grid - 1 when the barrier behaves).  Returns PPCG_OK when the
 * launch ran, PPCG_ERR_ARG for bad sizes, PPCG_ERR_CUDA on a launch failure.
 */
ppcg_status ppcg_selftest_barrier_timeout(int32_t grid, int32_t drop_rank, int64_t limit_ns,
                                          int32_t* timed_out);

/*
 * Allocation-free solve.  The paper has no counterpart: this entry point exists for callers
 * that may not allocate device memory while solving -- code whose device memory is owned by
 * a framework pool, real-time loops where cudaMalloc/cudaFree (which can synchronise the
 * whole device) are not allowed, or plug-ins whose host forbids allocation after start-up.
 * It runs pipelined preconditioned CG with a Jacobi (diagonal) preconditioner straight from
 * the caller's device CSR on one thread-block cluster, keeping every working vector in a
 * statically sized device array of the library (4.5 MiB on each GPU that loads the
 * library, held until the process exits).  It calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *   n <= 65536 rows; larger n returns PPCG_ERR_ARG (use ppcg_create/ppcg_solve instead).
 *   row_ptr [n+1] int64, col [nnz] int32, val [nnz], b [n], x [n]: DEVICE pointers, caller-owned.
 *   x0: device initial guess or NULL for zero; may alias x.  Stopping test: REL_R (||r|| <=
 *   tol ||b||), maxit as in ppcg_solve; no residual replacement.
 *   The matrix is checked on the device before it is used: row pointers outside [0, nnz],
 *   decreasing, or with row_ptr[0] != 0 or row_ptr[n] != nnz, or a column outside [0, n),
 *   end the solve with status PPCG_ERR_ARG (nothing is gathered through them); a missing or
 *   non-positive diagonal entry with PPCG_ERR_NOT_SPD.
 *   Return value: argument and launch errors only (PPCG_OK once the solve is enqueued).  The
 *   solve's own status -- OK, NOT_CONVERGED, BREAKDOWN, NONFINITE, NOT_SPD, or ERR_ARG for a
 *   malformed matrix -- is reported only through info: with info non-NULL the call waits for
 *   the solve (it synchronises `stream`) and fills it; with info NULL it only enqueues the
 *   work and the status is not available.
 * Set-up: the first call on a device (any call, including one with n = 0) looks up the
 * scratch array's device address and loads the library's kernel on that device, with that
 * device current; under lazy module loading this is where the array itself is allocated.
 * Make one call with n = 0 at initialisation, before any stream capture: later calls on
 * that device then allocate nothing.
 * All calls on a device share the scratch array: calls whose GPU work overlaps (other streams
 * or host threads) race on it, so order them.  Each call rewrites the scratch it reads, so
 * earlier calls' contents never affect a result.
 */
ppcg_status ppcg_solve_noalloc(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                               const double* val, const double* b, const double* x0, double* x,
                               double tol, int32_t maxit, cudaStream_t stream, ppcg_info* info);

/* Thread-local text of the last error of this thread's calls ("" if none). */
const char* ppcg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PPCG_H */
