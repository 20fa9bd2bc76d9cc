/*
 * ensemble_solve.h - C ABI of libensemble_solve.so, the GB300 (sm_103a) hot path of the
 * multiple-ensemble method of Krasnopolsky, arXiv 1711.10622: pressure-Poisson solves for m
 * simultaneous flow realizations that share one sparse matrix.
 *
 * Conventions used by every entry point
 *   - Blocks of m vectors (X, Y, B, solutions) are n x m, stored row-wise in one array, element
 *     (k, l) at index k*m + l ("row-interleaved"; Section 2.3, the storage assumed by Fig. GSpMV).
 *   - CSR matrices use int32 row pointers and column indices and float64 values (Section 2.3).
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream). Unless stated
 *     otherwise a call only enqueues work on that stream and returns.
 *   - Device pointers are owned by the caller and must stay valid until the enqueued work ends.
 *     The library owns what it allocates (matrix copies, workspaces) and frees it in
 *     ens_destroy_matrix.
 *   - Errors: every call returns an ens_status; on failure nothing is enqueued and a message is
 *     available from ens_last_error() (per host thread). Sizes and pointers are validated on the
 *     host before any launch.
 *   - Threads: ens_gspmv, ens_solve_block and ens_solve_batch keep their scratch per call and may
 *     run concurrently on one matrix from several host threads / streams. ens_gspmv_host,
 *     ens_autotune, ens_set_f64_mode and ens_set_native_share change per-matrix state: call them
 *     from one host thread at a time per matrix, not concurrently with other calls on it.
 */
#ifndef ENSEMBLE_SOLVE_H
#define ENSEMBLE_SOLVE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ens_matrix ens_matrix;

typedef enum {
  ENS_OK = 0,
  ENS_ERR_INVALID = 1,     /* bad argument: size, pointer, CSR structure, unsupported m */
  ENS_ERR_OOM = 2,         /* device allocation failed */
  ENS_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed */
  ENS_ERR_TIMEOUT = 4,     /* a bounded device-side wait ran out */
  ENS_ERR_BUDGET = 5,      /* the request does not fit the memory budget */
  ENS_ERR_UNSUPPORTED = 6  /* valid request the library does not implement */
} ens_status;

/* Per-column outcome of a solve; the numeric values are part of the ABI. */
typedef enum {
  ENS_COL_CONVERGED = 0,   /* ||b - A x||_2 / ||b||_2 <= tol (b = 0 gives x = 0, 0 iterations) */
  ENS_COL_MAXITER = 1,     /* iteration limit reached */
  ENS_COL_BREAKDOWN = 2,   /* BiCGStab breakdown: rho ~ 0, (rhat, v) = 0, (t, t) = 0, omega = 0 or a
                              non-finite step length (x keeps its last finite iterate) */
  ENS_COL_NONFINITE = 3,   /* NaN/Inf met in b, x0 or the iteration */
  ENS_COL_INCOMPATIBLE = 4 /* singular operator and sum(b) != 0 */
} ens_col_status;

typedef enum { ENS_F64 = 0, ENS_F32 = 1 } ens_dtype;

/* ens_create_matrix flags */
#define ENS_MATRIX_SINGULAR 0x1u /* constants span the null space (pure Neumann/periodic) */

/* FP64 GSpMV arithmetic (ens_set_f64_mode): how the float64 path computes its products. */
typedef enum {
  ENS_F64_AUTO = 0,   /* library choice (split-float arithmetic where values allow) */
  ENS_F64_NATIVE = 1, /* native double-precision FMA for every product */
  ENS_F64_SPLIT = 2,  /* double-float products on the FP32 pipe, native FP64 fallback per row
                         segment whose values fall outside the split range */
  ENS_F64_HYBRID = 3  /* per lane, one column with native DFMA and one with split-float arithmetic,
                         so the FP64 and FP32/integer pipes work at once (even m; odd m: native) */
} ens_f64_mode;

/*
 * Create a device-resident CSR matrix from HOST arrays (copied; the caller keeps ownership).
 *   n        rows = columns, 1 <= n <= 2^31 - 1
 *   nnz      nonzeros, 0 <= nnz <= 2^31 - 1
 *   row_ptr  int32[n+1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz
 *   col_idx  int32[nnz], 0 <= col_idx[j] < n
 *   val      float64[nnz]
 *   flags    ENS_MATRIX_SINGULAR or 0
 * The library also keeps a float32 copy of val (for ENS_F32 products), the inverse diagonal
 * (Jacobi scaling of the Chebyshev preconditioner) and a split-float copy of val.
 * Synchronous: returns after the copies end. *out receives the handle.
 * Errors: ENS_ERR_INVALID (structure), ENS_ERR_OOM, ENS_ERR_CUDA.
 */
ens_status ens_create_matrix(int64_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                             const double *val, uint32_t flags, void *stream, ens_matrix **out);

/* Free the matrix and every workspace it owns. Synchronises the device first. NULL is a no-op. */
ens_status ens_destroy_matrix(ens_matrix *A);

/* n, nnz and the largest row length of A (any pointer may be NULL). */
ens_status ens_matrix_info(const ens_matrix *A, int64_t *n, int64_t *nnz, int32_t *max_row_len);

/* Select the FP64 GSpMV arithmetic for A (default ENS_F64_AUTO). */
ens_status ens_set_f64_mode(ens_matrix *A, int32_t mode);

/*
 * Split-float FP64 products only: the share, in 32nds of the row sweeps, that is computed with
 * native DFMA instead (0 = all split, 32 = all native; -1 = the library's table by block width).
 * GB300's FP64 pipe is idle in the split path, so a hybrid share adds its throughput. Tuning knob
 * used by the autotuner; results stay within the FP64 accuracy bound either way.
 */
ens_status ens_set_native_share(ens_matrix *A, int32_t share);

/*
 * Autotuner: time the GSpMV launch candidates for block width m (1..64) and dtype on this matrix
 * (lanes per row, i.e. rows per warp and column-tile width; tiled or untiled rows; for FP64 also native
 * DFMA vs split-float with native shares 0, 8, 12, 16, 24 of 32, and the column hybrid) and keep the fastest for later
 * ens_gspmv calls and for the solver's products of that width. Uses temporary device blocks of
 * n x m (stream-ordered, freed before return). Synchronous. Optional outputs: chosen lanes, chosen
 * share (32 = native, 64 = column hybrid), and the best time per launch in microseconds. A share
 * set with ens_set_native_share, or ENS_F64_HYBRID / ENS_F64_SPLIT modes, still take priority.
 */
ens_status ens_autotune(ens_matrix *A, int32_t m, int32_t dtype, void *stream, int32_t *lanes, int32_t *share,
                        double *best_us);

/*
 * Row traversal of ens_gspmv / ens_gspmv_host on A: -1 (default) the autotuner's choice per width
 * (tiled without tuning), 0 always shared-memory row tiles, 1 always untiled rows (read straight from
 * global memory; the column hybrid arithmetic always uses tiles). Results stay within the accuracy
 * bound either way. ENS_ERR_INVALID for other values.
 */
ens_status ens_set_untiled(ens_matrix *A, int32_t mode);

/*
 * The launch the autotuner chose for width m and dtype (-1 in every output where it has not run):
 * lanes per row, native share (as ens_autotune reports it) and untiled = 1 when the rows are read
 * straight from global memory instead of through shared-memory row tiles (both forms are timed).
 */
ens_status ens_tuned_variant(const ens_matrix *A, int32_t m, int32_t dtype, int32_t *lanes, int32_t *share,
                             int32_t *untiled);

/*
 * Generalised SpMV Y = A X (Section 2.3, Fig. GSpMV): for every row i and column l,
 *   Y[i*m + l] = sum_{j = row_ptr[i]}^{row_ptr[i+1]-1} val[j] * X[col_idx[j]*m + l].
 * m >= 1 columns (any m; m in {1,2,4,8,16,32} have specialised kernels). X and Y are DEVICE
 * pointers to n*m elements of the dtype (float64 for ENS_F64, float32 for ENS_F32; ENS_F32 uses
 * the float32 copy of val). X and Y must not overlap. Asynchronous on `stream`.
 * Accuracy (ENS_F64): each output is within 1e-12 of the exact sum relative to sum_j |val||x|.
 */
ens_status ens_gspmv(const ens_matrix *A, int32_t m, int32_t dtype, const void *X, void *Y, void *stream);

/*
 * The same product with HOST buffers X (n*m, read) and Y (n*m, written). The library copies X to
 * a device staging buffer it owns, runs the product and copies Y back; synchronous (returns after
 * Y is written). Page-locked host memory gives the full copy bandwidth. On matrices of more than
 * one 256-row tile the three stages overlap: X arrives in blocks of rows on a library-owned copy
 * stream, in the order the row chunks (up to 16) first need them, each row chunk is computed on
 * `stream` once the X blocks its column indices reach have arrived (periodic couplings included),
 * and its Y rows are copied back on a second library-owned stream. The overlap needs
 * page-locked X and Y: with pageable buffers each copy call returns only when it is done, so the
 * copies and kernels then run largely one after another. Y holds the same
 * values as ens_gspmv's to within the accuracy bound below (the FP64 split/native assignment of
 * rows can differ with the chunking). X and Y may overlap (an in-place product): the stages then
 * run one after the other.
 */
ens_status ens_gspmv_host(ens_matrix *A, int32_t m, int32_t dtype, const void *X, void *Y, void *stream);

/*
 * ens_gspmv_host without device allocation. (The paper has no counterpart: this is a deployment
 * variant of ens_gspmv_host.) For callers that cannot let a library allocate device memory during
 * a call: applications that reserve all device memory for their own pool up front, real-time loops
 * that cannot afford an allocation's latency or implicit synchronisation, and hosts that forbid
 * plug-in libraries from allocating. It calls no cudaMalloc, cudaFree or other allocating routine:
 * X and Y are staged through one array compiled into the library, 2 x 16 MiB, which every GPU that
 * loads the array holds until the process exits.
 *   Same arguments, semantics and accuracy as ens_gspmv_host (host X read, host Y written;
 *   synchronous). n * m * sizeof(dtype) must not exceed 16 MiB (16,777,216 bytes; e.g. n*m <= 2,097,152
 *   for float64); larger requests return ENS_ERR_INVALID. The matrix's device must be current.
 *   The first call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 *   device current. With CUDA's lazy module loading (the default since CUDA 12.2) that lookup is
 *   also what loads the array's module, so the 32 MiB (plus a small module overhead) are reserved on
 *   the device by that FIRST call, not when the library is loaded. Make the first call once per
 *   device at start-up: before the application reserves its own device-memory pool, and before any
 *   stream capture. Every later call reserves nothing.
 *   All calls share the array and it keeps the last call's contents; nothing in it needs to start at
 *   zero (each call overwrites the staged X and all of Y). Calls whose GPU work overlapped would race
 *   on it; this entry point serialises its callers with a lock and returns only after its own copies
 *   finish, so calls made through it do not overlap within a process.
 */
ens_status ens_gspmv_host_noalloc(const ens_matrix *A, int32_t m, int32_t dtype, const void *X, void *Y, void *stream);

/* ---------------------------------------------------------------- multi-RHS BiCGStab solve */

typedef enum { ENS_PRECOND_NONE = 0, ENS_PRECOND_CHEBYSHEV = 1, ENS_PRECOND_AMG = 2 } ens_precond;
typedef enum { ENS_PREC_F64 = 0, ENS_PREC_MIXED = 1 } ens_precision;

typedef struct {
  int32_t max_iter;    /* BiCGStab iterations per column (FP64 mode); default 10000 */
  int32_t precond;     /* ENS_PRECOND_NONE (default), ENS_PRECOND_CHEBYSHEV, or ENS_PRECOND_AMG (one
                          V-cycle of the hierarchy built by ens_amg_setup on the matrix) */
  int32_t cheb_steps;  /* Chebyshev updates per application, >= 1 (default 4 = 3 GSpMVs; polynomial
                          of degree cheb_steps - 1 in D^-1 A) */
  double cheb_lo;      /* eigenvalue interval [cheb_lo, cheb_hi] of D^-1 A, 0 < lo < hi */
  double cheb_hi;      /* (default [2/30, 2]; 2 bounds D^-1 A of diagonally dominant M-matrices) */
  int32_t precision;   /* ENS_PREC_F64 (default) or ENS_PREC_MIXED: FP32 inner BiCGStab with FP32
                          reductions, FP64 outer residual r = b - A x and correction x += d */
  double inner_tol;    /* mixed: relative residual of each FP32 inner solve (default 1e-3; FP32
                          cannot resolve much below cond(A) * 6e-8, and each refinement step only
                          needs a reliable reduction) */
  int32_t max_outer;   /* mixed: refinement steps (default 50) */
  int32_t inner_max_iter; /* mixed: BiCGStab iterations per inner solve (default 100); a stagnating
                             inner solve is cut short and the next refinement step restarts it */
  int32_t check_every; /* host-driven loop only: iterations between reads of the convergence flags
                          (default 1) */
  int32_t x0_zero;     /* nonzero: ignore X on input and start from x0 = 0 */
  int32_t use_graph;   /* nonzero (default): the iteration loop runs on the device as a CUDA graph
                          with a conditional WHILE node; 0: host-driven loop */
  void *workspace;     /* NULL (default): the solve's scratch (internal copies of B and X, the Krylov
                          blocks, the preconditioner's blocks, per-column scalars) is allocated
                          stream-ordered for the call. Otherwise caller-owned DEVICE memory, 256-byte
                          aligned, that holds all of it: nothing is allocated, so a server can keep
                          its solvers' state in memory reserved once (Section 4.2's M = alpha + gamma m:
                          gamma m is this workspace). One call at a time per workspace. */
  uint64_t workspace_bytes; /* its size; a call that needs more returns ENS_ERR_BUDGET (the size it
                               needed at least is then ens_last_workspace_bytes()) */
} ens_solve_opts;

/* Host arrays of m entries each, filled on return; any pointer may be NULL. */
typedef struct {
  int32_t *iters;  /* BiCGStab iterations (summed over the inner solves in mixed mode) */
  double *relres;  /* true relative residual ||b - A x||_2 / ||b||_2 at exit (0 if b = 0, NaN for
                      NONFINITE / INCOMPATIBLE columns rejected before iterating) */
  int32_t *status; /* ens_col_status */
  int32_t *outer;  /* refinement steps (mixed mode), 0 otherwise */
} ens_solve_stats;

/* Fill *o with the defaults listed above. */
void ens_default_solve_opts(ens_solve_opts *o);

/*
 * Solve A x_l = b_l for the m columns of B at once (Section 2.2: the m pressure solves of the
 * ensemble share the matrix, only the right-hand sides differ; Section 4.1: BiCGStab). Each
 * column runs its own BiCGStab recurrence (van der Vorst 1992; right preconditioning, per-column
 * alpha, beta, omega, rho) and every iteration shares one GSpMV over the whole block; converged
 * columns are frozen. Stops column l when ||b_l - A x_l||_2 / ||b_l||_2 <= tol[l] (the recursive
 * residual, checked after each half step), then reports the true residual.
 *   B    DEVICE, n x m row-interleaved float64 (read)
 *   X    DEVICE, n x m row-interleaved float64: initial guess in (unless opts->x0_zero), solution out
 *   tol  HOST, m finite values >= 0
 *   opts may be NULL (defaults); stats may be NULL.
 * With ENS_MATRIX_SINGULAR the operator's null space is the constants: a column whose sum exceeds
 * 1e-10 sqrt(n) ||b_l|| is rejected (ENS_COL_INCOMPATIBLE) and every solution is returned with
 * zero mean. Supports 1 <= m <= 64. Synchronous: returns when X and stats are written.
 * Workspace (about 8-13 n x m blocks) is allocated stream-ordered for the call and released, or taken
 * from opts->workspace when given (then nothing is allocated).
 */
ens_status ens_solve_block(const ens_matrix *A, int32_t m, const double *B, double *X, const double *tol,
                           const ens_solve_opts *opts, ens_solve_stats *stats, void *stream);

/*
 * Coupled block-Krylov variant of ens_solve_block: block BiCGStab (Guennouni, Jbilou and Sadok
 * 2003), standing in for the multiple right-hand-side extension of the paper's solver library that
 * Section 3 names without describing. The m columns build ONE Krylov space: alpha and beta are
 * m x m matrices (R~^T V)^-1 (R~^T R) and -(R~^T V)^-1 (R~^T T) with the shadow block R~ = R_0,
 * solved by LU with partial pivoting on the host, and omega = <T, S>_F / <T, T>_F is one scalar per
 * block; right preconditioning M^-1 (ENS_PRECOND_NONE, _CHEBYSHEV or _AMG) on every column.
 * Arguments as ens_solve_block; float64 only (ENS_ERR_UNSUPPORTED for ENS_PREC_MIXED or a caller
 * workspace), 1 <= m <= 32. The block stops when every column's recursive residual meets its tol
 * (after a half or a full step) or after max_iter iterations; every column reports the block's
 * iteration count; a column is CONVERGED when its recursive residual meets its tolerance at exit,
 * else MAXITER. Columns with b = 0, non-finite data or an incompatible b (singular operators) leave
 * before the first iteration, as in ens_solve_block. BREAKDOWN for every remaining column: a zero
 * pivot in R~^T V (e.g. two equal right-hand sides), <T, T>_F = 0, omega = 0 or a non-finite step.
 * Gram products and updates cost O(n m^2) float64 multiply-adds per iteration (the FP64 pipe).
 * Synchronous.
 */
ens_status ens_solve_block_coupled(const ens_matrix *A, int32_t m, const double *B, double *X, const double *tol,
                                   const ens_solve_opts *opts, ens_solve_stats *stats, void *stream);

/* One system of a batched solve. */
typedef struct {
  const ens_matrix *A;    /* its matrix */
  int32_t m;              /* its block width, 1..64 */
  const double *B;        /* DEVICE n x m right-hand sides */
  double *X;              /* DEVICE n x m: initial guess in (unless opts->x0_zero), solution out */
  const double *tol;      /* HOST [m] */
  ens_solve_stats *stats; /* HOST arrays of m entries each, or NULL */
} ens_batch_item;

/*
 * Solve several systems of uneven n and m at once (Section 2.2's shared-matrix solves, for several
 * matrices). Each system runs exactly the ens_solve_block algorithm with the shared opts; all of
 * them are recorded as branches of ONE CUDA graph whose iteration loops are conditional WHILE
 * nodes (nested outer/inner loops in mixed precision), so a single graph launch runs every system
 * concurrently and each loop stops on the device when its columns are done or its limit is hit.
 * The items' buffers must not overlap. Synchronous. Errors name the offending item.
 */
ens_status ens_solve_batch(int32_t nsys, const ens_batch_item *items, const ens_solve_opts *opts, void *stream);

/*
 * Aggregation multigrid preconditioner ("AMG-lite"). The paper's solver is BiCGStab with algebraic
 * multigrid (Section 4.1); this is a lighter stand-in built once per matrix:
 *   strength   j != i is a strong neighbour of i when |a_ij| >= theta sqrt(|a_ii| |a_jj|);
 *   aggregates plain aggregation in three greedy phases (Vanek, Mandel, Brezina 1996): rows in
 *              increasing order start an aggregate with their strong neighbours when all of them
 *              are free; left-over rows join the phase-1 aggregate of their strongest aggregated
 *              strong neighbour (largest |a_ij|, then the smallest j); rows still free start
 *              aggregates with their free strong neighbours;
 *   transfer   piecewise constant P, restriction P^T; coarse operators A_c = P^T A P;
 *   levels     coarsen while n > coarse_size (at most max_levels, each level <= n / 1.5 rows);
 *   V-cycle    z = S(r); z += P V(P^T (r - A z)); z += S(r - A z), S = the Jacobi-scaled Chebyshev
 *              iteration on the level's matrix (smooth_steps updates, interval [cheb_lo, cheb_hi]
 *              of D^-1 A_l); the coarsest level runs coarse_steps Chebyshev updates.
 * The V-cycle is one fixed linear operator, applied to all m columns of a block at once (every
 * level's products are GSpMVs); ens_solve_block with ENS_PRECOND_AMG uses it as M^-1. Each smoothed
 * level also keeps the column-scaled copy A_l D_l^-1, so a two-update smoothing is one pass.
 */
typedef struct {
  double theta;          /* strength threshold (default 0.08) */
  int32_t max_levels;    /* levels including the fine one, 2..16 (default 8) */
  int32_t coarse_size;   /* stop coarsening at or below this many rows (default 512) */
  int32_t smooth_steps;  /* Chebyshev updates per smoothing, >= 1 (default 2 = 1 GSpMV) */
  int32_t coarse_steps;  /* Chebyshev updates on the coarsest level, >= 1 (default 16) */
  double cheb_lo;        /* smoother interval of D^-1 A_l (default [2/30, 2]: diagonal dominance */
  double cheb_hi;        /* is kept by P^T A P, so 2 bounds every level) */
} ens_amg_opts;

/* Fill *o with the defaults listed above. */
void ens_default_amg_opts(ens_amg_opts *o);

/* Build the hierarchy of A and attach it (replacing any previous one). Reads A back to the host,
 * aggregates and forms the coarse operators there, and uploads them as matrices of their own.
 * opts may be NULL (defaults). Synchronises `stream`. ENS_ERR_INVALID for bad options; on a
 * device error nothing is attached. Not concurrent with other calls on A. */
ens_status ens_amg_setup(ens_matrix *A, const ens_amg_opts *opts, void *stream);

/* Level count of A's hierarchy (0 if none) and, if the arrays are not NULL, the rows and nonzeros
 * of each level (host arrays of at least that many entries). */
ens_status ens_amg_info(const ens_matrix *A, int32_t *levels, int64_t *rows, int64_t *nnz);

/* Host copies of level `level`: its CSR (row_ptr [rows+1], col_idx and val [nnz]) and, except on the
 * coarsest level, agg [rows] (next-level row of each row). Any pointer may be NULL. Synchronous. */
ens_status ens_amg_level(const ens_matrix *A, int32_t level, int32_t *row_ptr, int32_t *col_idx, double *val,
                         int32_t *agg);

/* Z = V(R): one V-cycle on an n x m row-interleaved DEVICE block (dtype ENS_F64 or ENS_F32; the
 * float32 cycle uses the float32 copies of every level), 1 <= m <= 64. Workspace is allocated
 * stream-ordered for the call. Synchronous. ENS_ERR_INVALID without a hierarchy. */
ens_status ens_amg_apply(const ens_matrix *A, int32_t m, int32_t dtype, const void *R, void *Z, void *stream);

/* Human-readable message of the last failed call on this host thread ("" if none). */
const char *ens_last_error(void);

/* Scratch bytes the last ens_solve_block / ens_solve_batch call on this host thread took from its
 * workspace (or allocated stream-ordered when it had none); after ENS_ERR_BUDGET, the bytes it needed
 * up to the request that did not fit. The per-solve part of the memory model M = alpha + gamma m
 * (Section 4.2, Tables 6/7) is fitted from these values. */
uint64_t ens_last_workspace_bytes(void);

/* Library version string. */
const char *ens_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ENSEMBLE_SOLVE_H */
