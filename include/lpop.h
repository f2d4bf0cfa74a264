/*
 * lpop.h -- C ABI of the GB300 library for PDHG with online preconditioning
 * (H. Lu and W. Zhang, "Enhanced PDHG for Linear Programming with Online
 * Preconditioning", arXiv 2506.17650).
 *
 * Problem (Eq. (1) of the paper, generalised to row senses and bounds):
 *
 *     min  c^T x   s.t.  A_i x (= | <= | >=) b_i  (i < m),   lb <= x <= ub.
 *
 * The library preprocesses the LP (Ruiz equilibration, then Pock-Chambolle or
 * L2 rescaling, Section 2 and Section 4.2), keeps every vector and both CSR
 * copies (A and A^T) resident in device memory, and runs the iteration of
 * Algorithm 1 with the step of Eq. (6): two sparse products fused with the
 * preconditioned primal/dual updates and projections, the online-gradient
 * update of the diagonal preconditioners T and Sigma (Eq. (7), every phi
 * accepted steps, optionally normalised), and KKT / restart reductions.
 *
 * Conventions for every function:
 *  - All pointer arguments are HOST pointers unless stated otherwise.  Input
 *    arrays are caller-owned and only read during the call (copied to the
 *    device); output arrays are caller-allocated.
 *  - The library owns all device memory of a problem and frees it in
 *    lp_destroy() (through options.device_free when the caller supplied an
 *    allocator).
 *  - Every function returns an lp_err code (LP_OK = 0 on success); no C++
 *    exception crosses the ABI.  On failure lp_last_error() describes it.
 *  - The solve outcome (optimal, iteration limit, ...) is an lp_status,
 *    returned through an out-parameter, not as the error code.
 *  - Infinite bounds are IEEE +-INFINITY.  nnz must be below 2^31.
 *  - A problem is not thread-safe: calls on one handle must not overlap.
 */
#ifndef LPOP_H
#define LPOP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lp_problem lp_problem; /* opaque handle, owned by the library */

/* error codes (function return values) */
enum {
  LP_OK = 0,
  LP_ERR_INVALID_ARG = -1,   /* NULL pointer, bad size or bad option */
  LP_ERR_INVALID_INPUT = -2, /* NaN/Inf data, index out of range, lb > ub, ... */
  LP_ERR_CUDA = -3,          /* a CUDA runtime call failed */
  LP_ERR_OOM = -4,           /* device allocation failed */
  LP_ERR_NOT_SOLVED = -5     /* lp_result() before any lp_solve() */
};

/* solve outcome (lp_solve status_out, lp_stats.status) */
enum {
  LP_STATUS_NONE = 0,
  LP_OPTIMAL = 1,          /* relative KKT error within the tolerance */
  LP_ITERATION_LIMIT = 2,  /* iteration limit reached first */
  LP_TIME_LIMIT = 3,       /* options.time_limit seconds elapsed first */
  LP_NUMERICAL_ERROR = 4   /* a KKT quantity became NaN or Inf */
};

/* options.mode */
enum {
  LP_MODE_PLAIN = 0, /* vanilla PDHG (Section 4.2): fixed step 0.9/||A~||_2, no restarts */
  LP_MODE_PDLP = 1   /* Eq. (6): adaptive step size, primal weight, restarts (Section 3.2) */
};

/* options.precision */
enum {
  LP_PREC_FP64 = 0,  /* every kernel in FP64 */
  LP_PREC_MIXED = 1  /* FP32 matrix values, vectors and row arithmetic; FP64 KKT / step-size /
                        normalisation reductions and scalars; FP64 refinement phase */
};

/* options.scheduler: learning-rate rule of the online update (Section 4.1 names AdaGrad) */
enum {
  LP_SCHED_ADAGRAD = 0,      /* per-coordinate AdaGrad */
  LP_SCHED_ADAGRAD_NORM = 1, /* one AdaGrad accumulator per side */
  LP_SCHED_CONST = 2         /* constant learning rate */
};

/* Optional allocator for a problem's device buffers, for callers whose device
 * memory belongs to a framework (for example a caching allocator).  alloc
 * returns at least `bytes` bytes of device memory on the problem's device,
 * aligned to 256 bytes, or NULL (lp_create then fails with LP_ERR_OOM); a
 * block that is not 256-byte aligned is handed straight back to free and
 * lp_create fails with LP_ERR_INVALID_ARG.  free returns a block alloc gave,
 * with the same size.  Both are called only from
 * lp_create and lp_destroy, on the calling thread; lp_destroy synchronises the
 * problem's stream before it frees. */
typedef void* (*lp_device_alloc_fn)(size_t bytes, void* ctx);
typedef void (*lp_device_free_fn)(void* ptr, size_t bytes, void* ctx);

typedef struct lp_options {
  int32_t mode;              /* LP_MODE_*; default LP_MODE_PDLP */
  int32_t scheduler;         /* LP_SCHED_*; default LP_SCHED_ADAGRAD */
  double alpha;              /* online learning rate; 0 keeps T = Sigma = I (vanilla) */
  int32_t phi;               /* update period phi (Section 3.2); <= 0 never updates; default 20 */
  int32_t normalize;         /* normalised online loss (Algorithm 1); default 1 */
  double precond_floor;      /* projection floor for T and Sigma; default 1e-6 */
  int32_t ruiz_iters;        /* Ruiz rounds (Section 2); default 10 */
  double pc_beta;            /* Pock-Chambolle exponent beta in [0, 2] (pdlp mode); default 1 */
  int32_t check_every;       /* attempts between KKT / restart checks, 1..65536 (one check period is
                                captured as one CUDA graph); default 64 */
  int32_t restart;           /* adaptive restarts in pdlp mode; default 1 */
  int32_t power_iters;       /* power iterations for ||A~||_2 (plain mode); default 200 */
  double plain_step_factor;  /* plain mode step = factor / ||A~||_2; default 0.9 */
  double time_limit;         /* seconds per lp_solve call; <= 0 means none; default 0 */
  int32_t use_graph;         /* replay one check period as a CUDA graph; default 1 */
  int32_t kernel_timing;     /* time sampled launches of the hot kernels with CUDA events: 0 off (default),
                                1 one attempt in 8, k >= 2 one attempt in k of each check period */
  int32_t device;            /* CUDA device ordinal; -1 = the calling thread's current device */
  void* stream;              /* cudaStream_t every launch and copy goes to; NULL = default stream */
  int32_t precision;         /* LP_PREC_*; default LP_PREC_FP64 */
  double refine_tol;         /* mixed: the FP32 phase hands over to FP64 once the relative KKT
                                error is at most this (or after refine_stall checks without a
                                10% gain, below); default 1e-6 */
  lp_device_alloc_fn device_alloc; /* NULL: cudaMalloc.  A problem takes its buffers from one block of
                                      lp_memory_bytes() bytes (the per-device step-size table, 16 MiB,
                                      shared by all problems, always comes from cudaMalloc) */
  lp_device_free_fn device_free;   /* required exactly when device_alloc is set */
  void* alloc_ctx;                 /* passed to device_alloc and device_free */
  int32_t refine_stall;            /* mixed: the FP32 phase also hands over after this many checks in a
                                      row without a 10% drop of its best relative KKT error; >= 1,
                                      default 16 */
  int32_t log_every;               /* > 0: lp_solve writes one line to stderr every log_every KKT checks
                                      (attempts, accepted steps, restarts, the three relative KKT errors,
                                      objectives, eta, omega, precision phase); 0 (default): silent */
} lp_options;

typedef struct lp_stats {
  double pobj;               /* c^T x of the returned point (user units) */
  double dobj;               /* dual objective of the returned point */
  double rel_pres;           /* ||primal residual|| / (1 + ||b||) */
  double rel_dres;           /* ||dual residual|| / (1 + ||c||) */
  double rel_gap;            /* |pobj - dobj| / (1 + |pobj| + |dobj|) */
  int64_t iterations;        /* step attempts since create/reset (accepted or not) */
  int64_t accepted;          /* accepted steps k */
  int64_t restarts;
  double eta;                /* current step size */
  double omega;              /* current primal weight */
  double solve_ms;           /* wall time of the last lp_solve call */
  int32_t status;            /* lp_status of the last lp_solve call */
  int32_t reserved;
} lp_stats;

/* Fill *opt with the defaults listed above.  Never fails. */
void lp_options_default(lp_options* opt);

/*
 * Create a problem from the CSR form of A (Eq. (1); problem statement of
 * Section 2) and preprocess it on the device.
 *   m, n          rows (constraints) and columns (variables), m >= 0, n >= 1
 *   nnz           number of stored entries, == row_ptr[m], < 2^31
 *   row_ptr       int64[m+1], non-decreasing, row_ptr[0] == 0
 *   col_idx       int32[nnz], each in [0, n); any order within a row;
 *                 repeated (row, col) entries are summed
 *   val           double[nnz], finite
 *   b             double[m], finite
 *   c             double[n], finite
 *   lb, ub        double[n]; lb < +inf, ub > -inf, lb <= ub; +-INFINITY allowed
 *   sense         char[m]: 'E' (=), 'L' (<=) or 'G' (>=)
 *   opt           options (NULL = defaults); opt->stream is kept for all later calls
 *   out           receives the handle on success, NULL on failure
 * Errors: LP_ERR_INVALID_ARG, LP_ERR_INVALID_INPUT (data checked on the host
 * before any device work), LP_ERR_CUDA, LP_ERR_OOM.
 * The arrays are copied to the device once (rows with repeated entries or out
 * of column order are first merged on the host); the bin-ordered copies of A
 * and A^T are built there, with scratch taken from the problem's block of
 * lp_memory_bytes() bytes (or, where it does not fit, from short-lived
 * allocations of the same kind, freed before the call returns).
 * The call returns after the preprocessing has finished on the device.
 */
int lp_create(int32_t m, int32_t n, int64_t nnz,
              const int64_t* row_ptr, const int32_t* col_idx, const double* val,
              const double* b, const double* c,
              const double* lb, const double* ub, const char* sense,
              const lp_options* opt, lp_problem** out);

/*
 * Run the iteration (Algorithm 1 with Eq. (6)) until the relative KKT error
 * (Section 4.1 tolerance) is at most rel_kkt_tol at a check, or until
 * iter_limit step attempts have been made since create/reset (the limit is
 * cumulative, so a second call continues), or until options.time_limit.
 * A check runs before the first attempt and after every check_every-th
 * attempt.  *status_out (may be NULL) receives an lp_status.
 * Errors: LP_ERR_INVALID_ARG (NULL handle, tol < 0), LP_ERR_CUDA.
 */
int lp_solve(lp_problem* p, double rel_kkt_tol, int64_t iter_limit, int32_t* status_out);

/*
 * Copy the current point, in user units and the caller's row/column order,
 * to x (double[n], may be NULL) and y (double[m], may be NULL; the paper's
 * lambda), and fill *st (may be NULL) with the KKT statistics of the last
 * check.  Errors: LP_ERR_INVALID_ARG, LP_ERR_NOT_SOLVED, LP_ERR_CUDA.
 */
int lp_result(lp_problem* p, double* x, double* y, lp_stats* st);

/*
 * Debug / parity access to the iterate in the PREPROCESSED (scaled) space, in
 * the caller's row/column order: x~ (double[n]), y~ (double[m]), T (double[n]),
 * Sigma (double[m]); any may be NULL.  A pending preconditioner update is
 * applied first.  scal (double[8], may be NULL) receives
 * {eta, omega, k, attempts, wsum, restarts, last_eta_max, last_accept}.
 * Errors: LP_ERR_INVALID_ARG, LP_ERR_CUDA.
 */
int lp_get_iterate(lp_problem* p, double* x, double* y, double* T, double* Sigma, double* scal);

/*
 * Scaled-space vectors of the preprocessing, caller's order: dr (double[m]),
 * dc (double[n]) with A~ = diag(dr) A diag(dc), and scal (double[8], may be
 * NULL) = {eta_0, omega_0, ||A~||_2 estimate (plain mode, else 0), max|A~_ij|,
 * blocks of the A-row kernels, blocks of the A^T-row kernels, work units of A,
 * work units of A^T}.
 * Errors: LP_ERR_INVALID_ARG, LP_ERR_CUDA.
 */
int lp_get_scaling(lp_problem* p, double* dr, double* dc, double* scal);

/*
 * Checkpoint / resume: the complete iteration state in the PREPROCESSED space,
 * caller's order.  A pending preconditioner update is applied before export.
 *   vec_n  double[5 n]: x, xbar (eta-weighted sum since the last restart),
 *          T, AdaGrad accumulator of T, x at the last restart
 *   vec_m  double[6 m]: y, ybar, A x, Sigma, AdaGrad accumulator of Sigma,
 *          y at the last restart
 *   scal   double[16]: eta, omega, wsum, scalar AdaGrad accumulators (primal,
 *          dual), weighted-KKT parts at the last restart (||pres||^2,
 *          ||dres||^2, gap^2), weighted KKT of the previous check, k,
 *          attempts, attempt of the last restart, restarts, restart reference
 *          recorded (0/1), initial check done (0/1), 0
 * lp_set_state takes the same layout (all three arrays required) and makes it
 * the state the next lp_solve continues from; the iteration limit of lp_solve
 * stays cumulative in `attempts`.  Errors: LP_ERR_INVALID_ARG, LP_ERR_CUDA,
 * LP_ERR_INVALID_INPUT (lp_set_state: eta or omega not finite and positive).
 */
int lp_get_state(lp_problem* p, double* vec_n, double* vec_m, double* scal);
int lp_set_state(lp_problem* p, const double* vec_n, const double* vec_m, const double* scal);

/*
 * Return the problem to its initial state (x_0 = proj(0), y_0 = 0, T = Sigma = I,
 * eta_0, omega_0, counters zero) without redoing the preprocessing.
 * Errors: LP_ERR_INVALID_ARG, LP_ERR_CUDA.
 */
int lp_reset(lp_problem* p);

/*
 * Kernel timing (options.kernel_timing >= 1): accumulated CUDA-event time in
 * milliseconds and sample counts of the sampled launches, for up to n_kernels
 * kernels in the order {primal step, dual step}.  launches (may be NULL)
 * receives the number of kernel launches issued since create/reset.
 * Errors: LP_ERR_INVALID_ARG.
 */
int lp_kernel_times(lp_problem* p, double* ms, int64_t* samples, int32_t n_kernels, int64_t* launches);

/*
 * No-allocation variant of the power iteration that lp_create runs in plain
 * mode (||A||_2 estimate for the vanilla step 0.9 / ||A||_2).  The paper has
 * no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- code inside a framework that has reserved device memory for
 * its own pool, a real-time loop that must not allocate, or a caller whose
 * buffers come from another allocator -- and that already hold the matrix on
 * the device.  It allocates nothing: its scratch (three work vectors and the
 * reduction's partial sums) is one fixed device array of 2^20 doubles (8 MiB)
 * that every GPU which loads this library holds until the process exits.
 *   m, n        rows and columns, m >= 1, n >= 1, and 2 n + m + 1025 <= 2^20
 *               (larger sizes are rejected with LP_ERR_INVALID_ARG)
 *   a_*         DEVICE pointers: CSR of A (int32 row_ptr[m+1], int32
 *               col_idx[nnz], double val[nnz])
 *   at_*        DEVICE pointers: CSR of A^T (n rows) holding the same entries
 *   iters       power iterations on A^T A from the all-ones direction, >= 1
 *   stream      cudaStream_t for all work (NULL = default stream); the call
 *               waits for this stream before returning
 *   norm_out    HOST pointer receiving sqrt(||A^T A v||) of the last round
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  The cached address does not survive cudaDeviceReset (the
 * module and its array may then move): do not call this entry point again in
 * a process after resetting the device.  All calls share the one array and leave their data in it;
 * nothing in it needs to start at zero.  Calls whose work overlaps on the GPU
 * (other threads or streams) race on the array: serialise them.
 * Errors: LP_ERR_INVALID_ARG (sizes, NULL pointers), LP_ERR_CUDA; the message
 * is returned by lp_last_error(NULL).
 */
int lp_power_norm_noalloc(int32_t m, int32_t n, const int32_t* a_row_ptr, const int32_t* a_col_idx,
                          const double* a_val, const int32_t* at_row_ptr, const int32_t* at_col_idx,
                          const double* at_val, int32_t iters, void* stream, double* norm_out);

/*
 * Batched solves (many LPs advancing together in one persistent launch).
 *
 * A batch references existing problems (the members keep ownership of their
 * data and state; destroy the batch before its members).  lp_batch_round runs
 * every open member for up to `attempts` step attempts of Algorithm 1 with
 * Eq. (6) -- checks, restarts and the online preconditioner updates included
 * -- in ONE kernel launch.  Members with at least wide_nnz nonzeros are solved
 * by a thread-block cluster of cluster_size CTAs, the others by one CTA each;
 * members are assigned longest-first by nonzero count.  After each round the
 * members' host views are refreshed, so lp_result / lp_get_state work on them
 * as after lp_solve.  All members must live on one device.  The batch runs on
 * its own stream, created on the members' device; each member's pending work
 * on its own stream has finished before the batch first reads that member.
 * Errors: LP_ERR_INVALID_ARG, LP_ERR_CUDA.
 */
typedef struct lp_batch lp_batch;

int lp_batch_create(int32_t count, lp_problem* const* members, lp_batch** out);

/* Replace the member list between rounds (serving: retire finished problems,
 * admit new ones).  Members keep their state. */
int lp_batch_set_members(lp_batch* b, int32_t count, lp_problem* const* members);

/* Team schedule: cluster_size in {1, 2, 4, 8}; members with >= wide_nnz
 * nonzeros get a whole cluster (default: cluster_size 1, no wide teams). */
int lp_batch_set_schedule(lp_batch* b, int32_t cluster_size, int64_t wide_nnz);

/* One round: every member with fewer than iter_limit attempts that is not yet
 * finished under rel_kkt_tol runs up to `attempts` more (members finished
 * under another tolerance are re-opened).  *active_out (may be NULL) receives
 * the number of members still open afterwards. */
int lp_batch_round(lp_batch* b, double rel_kkt_tol, int32_t attempts, int64_t iter_limit, int32_t* active_out);

/* Rounds of round_attempts attempts until no member is open; *n_optimal (may
 * be NULL) receives how many members reached the tolerance.  With a handoff
 * (lp_batch_set_handoff), a member still open at a round boundary after at
 * least that many attempts leaves the batch and finishes with lp_solve (its
 * own full-grid kernels, on its own stream, from a pool of at most 16 host
 * threads of this call) while the batch goes on with the rest; the call
 * returns when all are done.
 * The rule depends only on the member's own attempts, so a member's result
 * does not depend on the rest of the batch. */
int lp_batch_solve(lp_batch* b, double rel_kkt_tol, int64_t iter_limit, int32_t round_attempts, int32_t* n_optimal);

/* Handoff threshold of lp_batch_solve in attempts (0 = never, the default).
 * No counterpart in the paper: it bounds the batch's tail, where a few slow
 * members would otherwise run on a single CTA or cluster each.
 * Errors: LP_ERR_INVALID_ARG (NULL batch, negative value). */
int lp_batch_set_handoff(lp_batch* b, int64_t attempts);

/* Schedule autotuner: for cluster sizes {1, 2, 4, 8} and wide thresholds at
 * the 50/80/95/99th percentiles of the members' nonzero counts, reset every
 * member (lp_reset) and time a whole lp_batch_solve to rel_kkt_tol with an
 * attempt limit of trial_attempts per member, rounds of 256 attempts and the
 * batch's handoff (host clock: handed-off members run on their own streams),
 * so that the trial sees the slowest members, the tail the schedule must
 * hide; keep the fastest schedule and reset the members again.  A trial
 * limit at least as large as the real solve's measures exactly what that
 * solve will take.  Outputs (may be NULL): the chosen cluster size and
 * threshold, its trial time in ms. */
int lp_batch_autotune(lp_batch* b, double rel_kkt_tol, int32_t trial_attempts, int32_t* cluster_size,
                      int64_t* wide_nnz, double* trial_ms);

/* Per member (arrays of the batch's member count, either may be NULL): lp_status
 * (0 while open) and step attempts so far. */
int lp_batch_status(lp_batch* b, int32_t* status, int64_t* iterations);

/* Kernel launches issued by the batch (rounds and state read-backs). */
int lp_batch_launches(const lp_batch* b, int64_t* launches);

/* Free the batch (not its members).  NULL is ignored. */
void lp_batch_destroy(lp_batch* b);

/* Device bytes lp_create allocates for a problem of this size with these
 * options (after merging repeated entries nnz can only shrink), for callers
 * that admit problems by free memory: lp_create takes all of a problem's
 * device buffers from one allocation of this size (the per-device step-size
 * table, 16 MiB, is shared by all problems on a device and not included).
 * Writes *bytes; LP_ERR_INVALID_ARG on bad sizes or NULL bytes. */
int lp_memory_bytes(int32_t m, int32_t n, int64_t nnz, const lp_options* opt, int64_t* bytes);

/* Free all device and host memory of the problem.  NULL is ignored. */
void lp_destroy(lp_problem* p);

/* Last error message of p, or of the calling thread when p is NULL. */
const char* lp_last_error(const lp_problem* p);

#ifdef __cplusplus
}
#endif

#endif /* LPOP_H */
