/*
 * pdlp.h -- C ABI of the GB300 restarted-PDHG (PDLP) linear-programming solver.
 *
 * Problem (cuPDLP.jl paper, Sec. 2, eq. (lp) and eq. (primal-dual)):
 *
 *     min  c'x   s.t.   A x = b,   G x >= h,   l <= x <= u,
 *
 * passed as one CSR matrix K = (A; G) with m rows and n columns whose first
 * n_eq rows are the equalities and the remaining m - n_eq rows the ">="
 * constraints, and one right-hand side q = (b; h).  The paper lists G first;
 * the order is only a permutation of the same problem.  Bounds may be
 * -INFINITY / +INFINITY.  The dual variable y is free on equality rows and
 * y >= 0 on ">=" rows (Lagrangian L(x,y) = c'x - y'Kx + q'y).
 *
 * Method: restarted PDHG of Algorithm 1 with the adaptive step of Algorithm 2
 * (eq. (pdhg), eq. (step-size)), the KKT-error restart of Sec. 3.4 (eq. kkt),
 * primal-weight initialisation / update of Sec. 2.2, Ruiz + Pock-Chambolle
 * diagonal preconditioning of Sec. 2.2 (done on the GPU at create time), and
 * termination on the relative KKT error of the ORIGINAL problem (Sec. 4.1).
 * Every step of the iteration runs in this library's CUDA kernels on one GPU;
 * the host only launches CUDA graphs and polls a status word.
 *
 * Conventions for every function below:
 *   - Return value: PDLP_OK (0) or a negative PDLP_ERR_* code.  No function
 *     aborts the process.  On error pdlp_last_error() returns a message for
 *     the calling thread.
 *   - Pointers named *_out are caller-allocated HOST buffers of the stated
 *     length; inputs are HOST arrays copied during the call (the caller keeps
 *     ownership and may free them on return).  Functions ending in _device
 *     take DEVICE pointers instead (see their comments).
 *   - A solver object is not thread-safe: use one host thread per object.
 *   - Requires a CUDA device of compute capability 10.3 (GB300 / sm_103a).
 */
#ifndef PDLP_GB300_H
#define PDLP_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define PDLP_OK 0
#define PDLP_ERR_INVALID (-1) /* bad argument or malformed LP; nothing was done */
#define PDLP_ERR_CUDA (-2)    /* a CUDA call failed (no device, launch error, ...) */
#define PDLP_ERR_OOM (-3)     /* device or host allocation failed */

/* ---- solve status (the `status` out-argument) ---- */
#define PDLP_OPTIMAL 0    /* all three Sec. 4.1 inequalities hold with eps = tol */
#define PDLP_ITER_LIMIT 1 /* max_iter accepted PDHG steps taken first */
#define PDLP_TIME_LIMIT 2 /* params.time_limit_s wall-clock seconds elapsed first */
#define PDLP_NUMERICAL 3  /* a NaN / Inf appeared in the step-size test */
/* Infeasibility detection (Sec. 2.2, last bullet; params.eps_infeas > 0): at
 * a check, the difference of the last two accepted iterates, or the current
 * iterate minus the epoch's first, unscaled to the original LP, is an
 * approximate certificate (pdlp_info.ray_obj > 0 and ray_res <= eps_infeas *
 * ray_obj; definitions at pdlp_info).  The ray is returned in place of the
 * iterate it concerns. */
#define PDLP_PRIMAL_INFEASIBLE 4 /* y_out holds a dual ray yr: yr_i >= 0 on ">=" rows, lambda =
                                    proj_Lambda(-K'yr), q'yr + l'lambda+ - u'lambda- > 0 */
#define PDLP_DUAL_INFEASIBLE 5   /* x_out holds a primal ray xr: K_E xr = 0, K_G xr >= 0, xr in the
                                    recession cone of the bounds, c'xr < 0 (unbounded if feasible) */

typedef struct pdlp_solver pdlp_solver; /* opaque */

/* Algorithm parameters.  Defaults (pdlp_default_params) are the paper's
 * constants where it prints them (beta = 0.2 / 0.8 / 0.36, Sec. 3.4; step
 * exponents 0.3 / 0.6 are fixed, Algorithm 2) and this library's readings
 * where it is silent (10 Ruiz passes, Pock-Chambolle alpha = 1, theta = 0.5,
 * eps_zero = 1e-10, restart/termination check every 64 accepted steps). */
typedef struct {
  int32_t check_period;   /* P: restart + termination check after every P accepted steps (>= 1) */
  int32_t ruiz_iters;     /* Ruiz l_inf passes at create (>= 0) */
  double pc_alpha;        /* Pock-Chambolle exponent in [0, 2]; < 0 disables the pass */
  double theta;           /* primal-weight smoothing, [0, 1] */
  double eps_zero;        /* InitializePrimalWeight / PrimalWeightUpdate threshold */
  double beta_suff;       /* restart criterion (i) */
  double beta_nec;        /* restart criterion (ii) */
  double beta_art;        /* restart criterion (iii) */
  double time_limit_s;    /* wall-clock limit per solve; <= 0 means none */
  int32_t value_bits;     /* 64: K values stored FP64; 32: the PDHG steps read FP32 copies of the
                             scaled K (FP64 gathers, accumulation and iterates); the restart /
                             termination checks take their own products (K'y, K'ybar, K xbar) with
                             the FP64 K and reuse the dual step's K x of the current iterate */
  int32_t f32_polish;     /* with value_bits = 32: switch the steps to the FP64 K when the original-
                             space relative KKT error stalls over two restarts above tol (1 = on) */
  double eps_infeas;      /* relative tolerance of the infeasibility certificates (default 1e-8);
                             0 turns infeasibility detection off (single-LP and batched solvers) */
} pdlp_params;

/* Summary of the last solve (pdlp_get_info). */
typedef struct {
  int32_t status;   /* PDLP_* status of the last solve, -1 while running / never solved */
  int32_t which;    /* 0: the returned point is the current iterate, 1: the epoch average;
                       infeasible: 2: the certificate is the difference of the last two accepted
                       iterates, 3: the current iterate minus the epoch's first */
  int64_t iters;    /* accepted PDHG steps (k of Algorithm 1) */
  int64_t attempts; /* Algorithm 2 trials, accepted + rejected */
  int64_t restarts; /* restarts taken (n of Algorithm 1) */
  int64_t checks;   /* restart / termination checks evaluated */
  double pobj, dobj;      /* c'x and q'y + l'lambda+ - u'lambda- on the original LP at the last check */
  double rp_norm, rd_norm; /* ||(Ax-b, [h-Gx]+)||_2 and ||c - K'y - lambda||_2 (original LP) */
  double q_norm, c_norm;  /* ||q||_2, ||c||_2 of the original LP */
  double omega, eta_hat;  /* primal weight and next trial step size (scaled LP) */
  double setup_ms;        /* pdlp_create device work (transfer + transpose + scaling) */
  double solve_ms;        /* wall time of the last solve call */
  int64_t graph_launches; /* CUDA-graph launches in the last solve */
  int64_t f64_switch_iter; /* value_bits = 32 only: k at which the steps moved to FP64 K, -1 never */
  /* infeasible statuses only (else 0), on the original LP: PDLP_PRIMAL_INFEASIBLE: ray_obj =
     q'yr + l'lambda+ - u'lambda-, ray_res = ||(-K'yr - lambda, min(yr_G, 0))||_2;
     PDLP_DUAL_INFEASIBLE: ray_obj = -c'xr, ray_res = ||(K_E xr, min(K_G xr, 0), v)||_2 with v
     the distance of xr to the bounds' recession cone (xr_j >= 0 where l_j is finite, <= 0 where
     u_j is finite) */
  double ray_obj, ray_res;
} pdlp_info;

/* One restart / termination check that did not end the solve
 * (pdlp_get_trace): the Sec. 3.4 quantities on the scaled LP and the
 * Sec. 4.1 measures of the current iterate on the original LP. */
typedef struct {
  int64_t k;          /* accepted steps when the check ran */
  int64_t attempts;   /* Algorithm 2 trials so far (rejected steps = attempts - k) */
  int64_t restarts;   /* restarts so far (n in Algorithm 1), this check's included */
  int32_t restart;    /* bit 0: criterion (i), bit 1: (ii), bit 2: (iii); 0 = no restart */
  int32_t cand_avg;   /* 1 if GetRestartCandidate picked the average */
  double kkt_cur;     /* KKT_omega(current iterate), eq. (kkt) */
  double kkt_avg;     /* KKT_omega(average iterate) */
  double kkt_start;   /* KKT_omega(z^{n,0}) after the check (recomputed with the new omega) */
  double omega;       /* primal weight after the check */
  double eta_hat;     /* next trial step size */
  double rel_gap;     /* |c'x - dual objective| / (1 + |c'x| + |dual objective|) */
  double rel_primal;  /* primal residual / (1 + ||q||) */
  double rel_dual;    /* dual residual / (1 + ||c||) */
} pdlp_check;

/* Fills *p with the defaults listed above.  p must be non-NULL. */
void pdlp_default_params(pdlp_params *p);

/* Builds a solver for the LP: validates the CSR (row_ptr[0] = 0,
 * non-decreasing, 0 <= col_idx < n, finite values / c / q, no NaN bounds,
 * l <= u, l != +inf, u != -inf), copies everything to the GPU, builds K',
 * runs the Sec. 2.2 Ruiz + Pock-Chambolle scaling on the device, and stores
 * the scaled K and K' a second time in the sliced-ELL layout the iteration
 * reads (rows renumbered by length; see pdlp_get_layout).  The sliced-ELL
 * copy needs fewer than 2^31 stored entries (padding included).  With the
 * environment variable PDLP_DEBUG_CHECKS=1 create also checks that copy on
 * the device (column indices, padding, work items, row coverage) and fails
 * with PDLP_ERR_INVALID and the violation counts if it is malformed.
 *   m >= 0 rows, n >= 1 columns, 0 <= n_eq <= m, nnz = row_ptr[m] < 2^31.
 *   c: n, row_ptr: m+1, col_idx / val: nnz (int32 / float64), q: m, l / u: n.
 * Errors: PDLP_ERR_INVALID (bad input; *out untouched), PDLP_ERR_CUDA,
 * PDLP_ERR_OOM.  On success *out owns device memory until pdlp_destroy. */
int pdlp_create(pdlp_solver **out, int32_t m, int32_t n, int32_t n_eq, const double *c,
                const int32_t *row_ptr, const int32_t *col_idx, const double *val, const double *q,
                const double *l, const double *u);

/* As pdlp_create with explicit parameters (NULL = defaults) and a CUDA stream
 * (a cudaStream_t passed as void*; NULL = the library creates its own
 * non-blocking stream).  All device work of the solver is ordered on it. */
int pdlp_create_ex(pdlp_solver **out, int32_t m, int32_t n, int32_t n_eq, const double *c,
                   const int32_t *row_ptr, const int32_t *col_idx, const double *val, const double *q,
                   const double *l, const double *u, const pdlp_params *params, void *stream);

/* Cold solve from x = 0, y = 0 (Sec. 4.1, "Initialization") to the relative
 * KKT tolerance tol (> 0) or max_iter (>= 1) accepted steps.  Writes the
 * solution of the ORIGINAL LP to x_out (n) and y_out (m; may be NULL when
 * m = 0), the PDLP_* status to *status and the accepted step count to *iters
 * (either pointer may be NULL).  Blocks until done. */
int pdlp_solve(pdlp_solver *s, double tol, int64_t max_iter, double *x_out, double *y_out, int *status,
               int64_t *iters);

/* pdlp_create_ex for an LP whose arrays are already in DEVICE memory (the
 * same layout and meaning as pdlp_create's host arrays: c, l, u of n; q of m;
 * CSR row_ptr m+1, col_idx / val nnz; all on the current device).  The
 * caller keeps ownership; the solver copies what it needs into its own
 * memory, so the arrays may be freed or reused once the call returns.  The
 * row starts and the n- and m-vectors are read back to the host (the layout
 * of K and the input checks need them); the nonzeros are checked and copied
 * on the device and never cross to the host, except for an LP with a column
 * of more than 4096 nonzeros, whose K' is then built on the host.  Work is
 * ordered on `stream` (cudaStream_t as void*, NULL = a new stream), which
 * becomes the solver's stream as in pdlp_create_ex.  The solver is the one
 * pdlp_create_ex builds from the same values: every later result is bitwise
 * the same.  Errors: PDLP_ERR_INVALID for the input faults pdlp_create
 * rejects (found on the host or by the device check, before any solver
 * memory is allocated), PDLP_ERR_CUDA / PDLP_ERR_OOM as pdlp_create_ex. */
int pdlp_create_device(pdlp_solver **out, int32_t m, int32_t n, int32_t n_eq, const double *c,
                       const int32_t *row_ptr, const int32_t *col_idx, const double *val, const double *q,
                       const double *l, const double *u, const pdlp_params *params, void *stream);

/* QP extension (the paper's introduction names the extension of the method
 * to quadratic programs; this is the case of a diagonal Hessian): from the
 * next solve on, the objective is x'Qx/2 + c'x with Q = diag(qdiag), qdiag a
 * HOST array of n finite, non-negative entries in the original column order
 * (copied; NULL returns to the LP).  The primal step becomes the exact
 * proximal step x' = proj_X((x - tau (c - K'y)) / (1 + tau Q_jj)), the KKT
 * error and Sec. 4.1 termination use the objective's gradient c + Qx in the
 * reduced cost and the QP's objectives (primal c'x + x'Qx/2, dual
 * q'y + l'lambda+ - u'lambda- - x'Qx/2), Q is scaled with the columns
 * (D2 Q D2), and infeasibility detection is off (its certificates are the
 * LP's).  Everything else (Algorithms 1-2, restarts, primal weight) is
 * unchanged.  Errors: PDLP_ERR_INVALID for a null solver or a negative or
 * non-finite entry; PDLP_ERR_CUDA. */
int pdlp_set_quadratic(pdlp_solver *s, const double *qdiag);

/* As pdlp_solve but starting from (x0, y0) given in the ORIGINAL space
 * (host arrays of n and m; either may be NULL = zeros).  The point is used as
 * given (the first PDHG step projects it). */
int pdlp_solve_warm(pdlp_solver *s, const double *x0, const double *y0, double tol, int64_t max_iter,
                    double *x_out, double *y_out, int *status, int64_t *iters);

/* Non-blocking pieces of pdlp_solve, for callers that overlap work or time
 * the iteration:  pdlp_begin resets the state (warm point as in
 * pdlp_solve_warm, NULLs = cold) and evaluates KKT(z^{0,0});
 * pdlp_run_periods enqueues n_periods CUDA-graph launches (each covers P
 * accepted steps plus one restart / termination check, or stops early once
 * the solve has ended) without waiting; pdlp_poll waits for the enqueued work
 * and returns the status (-1 = still running); pdlp_finish writes the outputs
 * like pdlp_solve and waits. */
int pdlp_begin(pdlp_solver *s, const double *x0, const double *y0, double tol, int64_t max_iter);
int pdlp_run_periods(pdlp_solver *s, int32_t n_periods);
int pdlp_poll(pdlp_solver *s, int *status, int64_t *iters);
int pdlp_finish(pdlp_solver *s, double *x_out, double *y_out, int *status, int64_t *iters);

/* Checkpoint and resume of a solve: the state of Algorithm 1 (the iterate
 * z^{n,t}, the epoch's step-weighted sums behind the average z-bar^{n,t},
 * the restart point z^{n,0}, the step size eta-hat, the primal weight
 * omega^n, the counters k, t, n, the KKT references of the Sec. 3.4
 * criteria, the restart candidate) together with the cached products K x and
 * K'y the steps reuse and the infeasibility-detection references (Sec. 2.2).
 * The vectors are the scaled-space values in the ORIGINAL order of rows and
 * columns (stored exactly, nothing is rounded).
 *   pdlp_get_state: with buf = NULL, writes the blob's size to *bytes;
 *   otherwise copies the state into buf (cap bytes available) once the
 *   solver's stream is idle.  Take it between check periods: after
 *   pdlp_begin, pdlp_run_periods + pdlp_poll, or a finished solve.
 *   pdlp_set_state: loads a blob from pdlp_get_state of a solver built from
 *   the same LP with the same parameters (possibly another solver object,
 *   in another process, on a GPU with the same number of SMs), replacing
 *   the current state; the check trace is not part of the state (the
 *   solver's trace restarts: pdlp_get_trace then reports the checks made
 *   since the load).
 *   pdlp_resume: continues the loaded (or begun) solve like pdlp_solve,
 *   to the tolerance, iteration limit and time limit of the original solve
 *   (the time limit counts from pdlp_set_state).
 * Solving N + M steps equals solving N, moving the state, and resuming, bit
 * for bit.  Errors: PDLP_ERR_INVALID for a too-small buffer, a blob of
 * another size, library version, LP or parameter set, one not taken
 * between check periods, or one whose counters and flags are out of range
 * (check period, trace position, negative step counts, FP32 values on a
 * solver without them), all rejected on the host before any device work;
 * PDLP_ERR_CUDA for CUDA failures. */
int pdlp_get_state(const pdlp_solver *s, void *buf, size_t cap, size_t *bytes);
int pdlp_set_state(pdlp_solver *s, const void *buf, size_t bytes);
int pdlp_resume(pdlp_solver *s, double *x_out, double *y_out, int *status, int64_t *iters);

/* Enqueues n_periods periods like pdlp_run_periods but launches each kernel
 * directly (no graph) between CUDA events on the solver's stream, then waits
 * and adds each kernel class's event-measured device time to ms[i] and its
 * launch count to launches[i] (arrays of pdlp_kernel_count() entries, caller
 * zeroes them).  Same arithmetic as the graph path. */
int pdlp_time_kernels(pdlp_solver *s, int32_t n_periods, double *ms, int64_t *launches);
int32_t pdlp_kernel_count(void);
const char *pdlp_kernel_name(int32_t i);

/* Reports on the last solve.  info: see pdlp_info.  trace: the solver keeps
 * the records of the last 65536 checks in a device ring buffer (written by
 * the check kernel, no per-check transfer); pdlp_get_trace copies up to cap
 * of the retained records, oldest first, into trace and stores the number
 * of checks recorded since the solve began or its state was loaded (which
 * may exceed 65536) in *count. */
int pdlp_get_info(const pdlp_solver *s, pdlp_info *info);
int pdlp_get_trace(const pdlp_solver *s, pdlp_check *trace, int32_t cap, int32_t *count);

/* The Sec. 2.2 scaling computed at create: D1 (m), D2 (n) and the scaled
 * values of K~ = D1 K D2 in the input's CSR order (nnz).  Any pointer may be
 * NULL. */
int pdlp_get_scaling(const pdlp_solver *s, double *D1, double *D2, double *val_scaled);

/* Shapes of the sliced-ELL copies of K and K' the step and check kernels
 * read (pdlp_get_layout).  Rows are renumbered by length inside their group
 * (equality rows of K first); rows of at most long_threshold entries sit in
 * slices of 32 rows padded to the slice's longest row, longer rows are stored
 * whole, padded to a multiple of 32 entries.  Every stored entry costs one
 * FMA per SpMV, each slice one epilogue per SpMV. */
typedef struct {
  int64_t K_stored, K_slices, K_long_rows;    /* stored entries (padding included), slices, long rows */
  int64_t KT_stored, KT_slices, KT_long_rows; /* the same for K' */
  int32_t long_threshold, pad_;
} pdlp_layout_info;
int pdlp_get_layout(const pdlp_solver *s, pdlp_layout_info *info);

/* Measures this GPU's rate of random 8-byte gathers from a 16 MB vector
 * (2e7 gathers with coalesced 32-bit indices, 8 in flight per thread) and
 * of FP64 fused multiply-adds (lane operations per second), with CUDA
 * events on a private stream: the ceilings of the two on-chip resources an
 * SpMV half-step uses besides HBM (one gather and one FMA per nonzero).  Not
 * part of the method; allocates ~100 MB for the duration of the call.
 * Errors: PDLP_ERR_INVALID for null arguments, PDLP_ERR_CUDA. */
int pdlp_probe_rates(double *gathers_per_s, double *dfma_per_s);

/* The same random gathers with an SpMV's matrix stream beside them: per
 * entry a coalesced 4-byte index, a coalesced 8-byte value, the gather and
 * one FP64 FMA (the bytes a sliced-ELL SpMV moves per stored nonzero), 2e7
 * entries; gathers per second.  The ceiling a step kernel's SpMV meets on
 * an LP whose columns give the gathers no reuse.  Not part of the method;
 * allocates ~260 MB for the duration of the call.  Errors as
 * pdlp_probe_rates. */
int pdlp_probe_stream_gathers(double *gathers_per_s);

/* The CUDA stream (cudaStream_t as void*) all work of `s` is ordered on. */
void *pdlp_get_stream(const pdlp_solver *s);

/* Bytes of device memory the solver holds. */
size_t pdlp_device_bytes(const pdlp_solver *s);

/* Frees the solver's device and host memory (NULL is a no-op). */
void pdlp_destroy(pdlp_solver *s);

/* Message for the last error on the calling thread ("" if none). */
const char *pdlp_last_error(void);

/* ---- batched solves ---------------------------------------------------------
 * Many independent LPs solved together in one persistent launch: one CTA
 * runs the whole restarted PDHG of one LP (Algorithms 1-2, Sec. 3.4 restarts,
 * Sec. 4.1 termination, Sec. 2.2 scaling) with its own step size, primal
 * weight, restart and termination state, taking LPs from a device queue in
 * decreasing order of size.  Intended for many small and medium LPs (each
 * solve is confined to one SM). */

/* One LP of a batch, as in pdlp_create (HOST arrays). */
typedef struct {
  int32_t m, n, n_eq, pad_;
  const double *c;
  const int32_t *row_ptr;
  const int32_t *col_idx;
  const double *val;
  const double *q, *l, *u;
} pdlp_lp;

typedef struct pdlp_batch pdlp_batch; /* opaque */

typedef struct {
  int32_t count;           /* LPs in the batch */
  int32_t grid;            /* persistent CTAs launched */
  int64_t sum_m, sum_n, sum_nnz;
  double setup_ms;         /* create: validation, transposes, copies, batched scaling */
  double tune_ms;          /* create: schedule autotuning */
  double solve_ms;         /* last pdlp_batch_solve call, wall time */
  double entries_per_lane; /* the SpMV schedule most LPs were given by the per-LP autotuner: lanes
                              per row = smallest power of two g <= 32 with (mean row length) / g <=
                              entries_per_lane, from {4, 8, 16}; each LP's own choice is in
                              pdlp_batch_lanes.  Row sums have one order for every choice, so the
                              results do not depend on it */
  size_t device_bytes;
  int32_t resident;        /* LPs small enough to be solved from the CTA's shared memory */
  int32_t resident_max_bytes; /* shared-memory budget per CTA for such an LP */
  int32_t team_lps;        /* LPs large enough to be solved by a team of CTAs */
  int32_t team_size;       /* CTAs (SMs) per team */
  int32_t team_min_nnz;    /* nonzeros from which an LP goes to a team */
} pdlp_batch_stats;

/* Validates every LP (same rules as pdlp_create; errors name the LP), copies
 * the batch to the GPU, builds each K', scales every LP on the device and
 * autotunes the SpMV schedule by timing short solves of the whole batch with
 * a few candidate schedules.  Each LP is solved by one CTA; an LP whose K,
 * K' and vectors fit in the CTA's shared-memory budget is copied there and
 * solved from shared memory; an LP with at least 32768 nonzeros is solved by
 * a team of four CTAs on as many SMs, which meet at bounded global-memory
 * barriers (the batch's CTAs must all be resident: a barrier that waits more
 * than 2 s fails the solve with PDLP_ERR_CUDA).  params: NULL = defaults; value_bits must be 64.
 * stream: cudaStream_t as void* (NULL = own stream). */
int pdlp_batch_create(pdlp_batch **out, int32_t count, const pdlp_lp *lps, const pdlp_params *params,
                      void *stream);

/* Solves every LP of the batch to tol / max_iter (as pdlp_solve_warm).
 * x0 / y0: packed HOST warm starts (LP i's block follows LP i-1's; lengths
 * sum of n / sum of m) or NULL for cold starts.  Outputs are packed the same
 * way: x_out (sum of n), y_out (sum of m), status and iters (count each);
 * any output pointer may be NULL.  An LP certified infeasible gets
 * PDLP_PRIMAL_INFEASIBLE / PDLP_DUAL_INFEASIBLE with its ray in its y / x
 * block, as in pdlp_solve.  Blocks until done. */
int pdlp_batch_solve(pdlp_batch *b, const double *x0, const double *y0, double tol, int64_t max_iter,
                     double *x_out, double *y_out, int32_t *status, int64_t *iters);
int pdlp_batch_info(const pdlp_batch *b, pdlp_batch_stats *stats);
/* When each LP of the last pdlp_batch_solve started and finished (device
 * global timer), in seconds after the earliest start (count entries each;
 * NULL ok): the schedule behind the batch's makespan. */
int pdlp_batch_times(const pdlp_batch *b, double *start_s, double *end_s);
/* Lanes per row chosen for each LP's K and K' (count entries each; NULL ok):
 * 32 is a warp per row, smaller values put 32 / g rows on a warp.  The
 * autotuner at create times each candidate schedule on the whole batch and
 * keeps, per LP, the fastest; it changes speed, not results. */
int pdlp_batch_lanes(const pdlp_batch *b, int32_t *lanes_K, int32_t *lanes_KT);
void pdlp_batch_destroy(pdlp_batch *b);

/* ---- learned warm start: BF16 MLP -----------------------------------------
 * in -> hidden -> ReLU -> hidden -> ReLU -> out, mapping the parameters of a
 * parametric LP family to a start point (x, y) for pdlp_solve_warm /
 * pdlp_batch_solve.  Not in the paper.  Weights and activations enter the
 * GEMMs as BF16 with FP32 accumulation on the tensor cores; the output layer,
 * loss, gradients and Adam state (FP32 master weights) stay FP32.  The loss
 * is the mean squared error on targets standardised per output with the
 * mean / standard deviation of the data set given to pdlp_mlp_set_data;
 * pdlp_mlp_predict returns values in target units.  All arrays below are
 * HOST arrays, row-major. */
typedef struct pdlp_mlp pdlp_mlp; /* opaque */

/* max_batch (1..65535) bounds the mini-batch of train / gradients and the
 * chunk of predict; each weight matrix must stay below 2^31 entries, else
 * PDLP_ERR_INVALID.  Parameters start at zero: set them with
 * pdlp_mlp_set_params. */
int pdlp_mlp_create(pdlp_mlp **out, int32_t in_dim, int32_t hidden, int32_t out_dim, int32_t max_batch,
                    void *stream);
/* Number of FP32 parameters: layout W1 (in x hidden), b1 (hidden),
 * W2 (hidden x hidden), b2, W3 (hidden x out), b3 (out); W row-major [in][out]. */
int64_t pdlp_mlp_param_count(const pdlp_mlp *net);
/* Sets / reads the FP32 master weights (setting also resets Adam's moments). */
int pdlp_mlp_set_params(pdlp_mlp *net, const float *params);
int pdlp_mlp_get_params(const pdlp_mlp *net, float *params);
/* Copies the training set (X: samples x in, T: samples x out) to the GPU and
 * computes the per-output standardisation there. */
int pdlp_mlp_set_data(pdlp_mlp *net, int32_t samples, const float *X, const float *T);
/* `steps` Adam steps; step s uses rows idx[s * batch .. s * batch + batch)
 * of the data set (the caller draws them).  losses: per-step mean squared
 * error before the update (NULL ok). */
int pdlp_mlp_train(pdlp_mlp *net, int32_t steps, int32_t batch, const int32_t *idx, float lr, float beta1,
                   float beta2, float eps, float *losses);
/* Y (count x out) for inputs X (count x in), in target units. */
int pdlp_mlp_predict(pdlp_mlp *net, int32_t count, const float *X, float *Y);
/* One forward / backward pass on data-set rows idx[0 .. batch) without an
 * update: the loss and the gradient of every parameter (param_count floats,
 * layout as for set_params).  For checking the backward pass. */
int pdlp_mlp_gradients(pdlp_mlp *net, int32_t batch, const int32_t *idx, float *loss, float *grads);
/* Per-output standardisation in use (out floats each; NULL ok). */
int pdlp_mlp_stats(const pdlp_mlp *net, float *mean, float *std_dev);
void pdlp_mlp_destroy(pdlp_mlp *net);

/* Allocation-free Ruiz + Pock-Chambolle scaling of a matrix the caller keeps
 * in DEVICE memory.  This entry point has no counterpart in the paper; it is
 * the same scaling pdlp_create applies, with the same correctly rounded
 * divisions in the same order (row by row here, entry by entry in
 * pdlp_create, where each quotient comes from the factor's reciprocal and one
 * exact correction step; l_inf maxima and the fixed-order Pock-Chambolle row
 * sums do not depend on that), so D1, D2 and the scaled values are bitwise
 * equal to pdlp_get_scaling's.  It is offered
 * for callers
 * that cannot call cudaMalloc or cudaFree: code that must take every byte of
 * device memory from its own pool (a framework's caching allocator, a
 * service with a fixed memory budget) and code that must not stall the device,
 * which cudaFree does.  It allocates nothing: the per-pass row and column
 * factors live in a fixed 4 MiB device array inside this library, held by
 * every GPU that loads the library until the process exits.
 *   K (m x n CSR: K_ptr m+1, K_idx / K_val nnz) and its transpose K' (n x m
 *   CSR: KT_ptr n+1, KT_idx / KT_val nnz, entries of each row in increasing
 *   order of K's row index) are DEVICE arrays; K_val and KT_val are scaled in
 *   place to D1 K D2 (and its transpose); D1 (m) and D2 (n) are DEVICE
 *   outputs.  ruiz_iters >= 0 l_inf passes, then one Pock-Chambolle pass with
 *   exponent pc_alpha <= 2 (pc_alpha < 0 skips it), as in pdlp_params.
 *   stream: a cudaStream_t as void* (NULL = the legacy default stream); the
 *   work is enqueued there and the call returns without waiting.
 * Limits and errors: 0 <= m <= 262144 and 1 <= n <= 262144, else
 * PDLP_ERR_INVALID with a message naming the limit.  A null KT_ptr or D2, or
 * (when m > 0) a null K_ptr, K_idx, K_val, KT_idx, KT_val or D1, gives
 * PDLP_ERR_INVALID before any CUDA call.  The first call on each device looks up the device
 * address of the internal array (with that device current), so make that
 * first call before any stream capture begins.  All calls share the one
 * array: calls whose work overlaps on the GPU (different streams, or several
 * host threads) race and corrupt each other's factors.  Every factor is fully
 * rewritten in each pass, so nothing is left over from an earlier call. */
int pdlp_scale_device_noalloc(int32_t m, int32_t n, const int32_t *K_ptr, const int32_t *K_idx, double *K_val,
                              const int32_t *KT_ptr, const int32_t *KT_idx, double *KT_val, int32_t ruiz_iters,
                              double pc_alpha, double *D1, double *D2, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PDLP_GB300_H */
