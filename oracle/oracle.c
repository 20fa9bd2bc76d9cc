/*
 * CPU FP64 oracle for the multi-RHS pressure-Poisson hot path (arXiv 1711.10622).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the CUDA path is
 * checked against. Only the tests, the smoke check and the bench's CPU-baseline leg may load
 * it; the product library never calls it and shares no code with it.
 *
 * Built with -O2 -ffp-contract=off (no FMA contraction, no fast-math) so every sum below is
 * evaluated exactly in the order written.
 *
 * Contents
 *   oracle_spmv        y = A x for one column of a row-interleaved block (Section 2.3, Fig. GSpMV
 *                      with m = 1: per row, sum initialised to 0, j ascending in CSR order)
 *   oracle_gspmv       Y = A X for an n x m row-interleaved block, computed column by column as
 *                      m independent SpMVs (the definition of GSpMV in Section 2.3)
 *   oracle_chebyshev   z = p(D^-1 A) D^-1 r: Chebyshev iteration on the Jacobi-scaled system from
 *                      a zero start (Saad, Iterative Methods for Sparse Linear Systems, 2nd ed.,
 *                      Alg. 12.1); the preconditioner is not in the paper.
 *   oracle_bicgstab    BiCGStab (van der Vorst 1992, cited in Section 1; SLAE solver of Section 4.1)
 *                      for ONE right-hand side, right-preconditioned, x0 given.
 *   oracle_solve_block m independent BiCGStab solves, one per column (Section 2.2: m pressure
 *                      solves share the matrix; only the right-hand sides differ).
 *   oracle_gspmv_rowwise  the same Y = A X with the column loop inside the row loop (the form of
 *                      Fig. GSpMV); every element is summed in the same order, so the result is
 *                      bit-identical to oracle_gspmv.
 *   oracle_lu_solve    dense LU with partial pivoting (textbook), used to pin the solver.
 * The aggregation multigrid preconditioner (precond 2) lives in amg.c.
 *
 * The same source builds twice: serially (the test oracle) and with -fopenmp (the CPU baseline
 * timed on all host cores). The OpenMP pragmas split only independent work, rows of a product and
 * columns of a block solve, and every value is computed by the same serial code in the same order,
 * so both builds give the same bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads an OpenMP region of this build may use (1 in the serial build). */
int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Per-column outcome codes; the CUDA library uses the same numeric values. */
#define OR_CONVERGED 0
#define OR_MAXITER 1
#define OR_BREAKDOWN 2
#define OR_NONFINITE 3
#define OR_INCOMPATIBLE 4

/* Section 2.3, Fig. GSpMV, m = 1. X element k of the column lives at x[k*incx]. */
void oracle_spmv(int64_t n, const int32_t *row, const int32_t *col, const double *val,
                 const double *x, int64_t incx, double *y, int64_t incy) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double sum = 0.0;
    for (int64_t j = row[i]; j < row[i + 1]; ++j) sum += val[j] * x[(int64_t)col[j] * incx];
    y[i * incy] = sum;
  }
}

/* Section 2.3: Y = A X with X, Y stored row-wise (element (k, l) at k*m + l); one SpMV per column. */
void oracle_gspmv(int64_t n, const int32_t *row, const int32_t *col, const double *val, int m,
                  const double *X, double *Y) {
  for (int l = 0; l < m; ++l) oracle_spmv(n, row, col, val, X + l, m, Y + l, m);
}

/* Section 2.3, Fig. GSpMV: Y = A X with the m columns of a row computed together; each matrix entry
 * is read once per row and applied to the whole row of X. Element (i, l) is still the sum over j
 * ascending from 0, as in oracle_gspmv. */
void oracle_gspmv_rowwise(int64_t n, const int32_t *row, const int32_t *col, const double *val, int m,
                          const double *X, double *Y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double *y = Y + i * m;
    for (int l = 0; l < m; ++l) y[l] = 0.0;
    for (int64_t j = row[i]; j < row[i + 1]; ++j) {
      const double a = val[j];
      const double *x = X + (int64_t)col[j] * m;
      for (int l = 0; l < m; ++l) y[l] += a * x[l];
    }
  }
}

static double dot(int64_t n, const double *a, const double *b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static double diag_of_row(const int32_t *row, const int32_t *col, const double *val, int64_t i) {
  for (int64_t j = row[i]; j < row[i + 1]; ++j)
    if (col[j] == i) return val[j];
  return 0.0;
}

/*
 * Chebyshev iteration for A z = r with Jacobi scaling D = diag(A), zero initial guess, on the
 * eigenvalue interval [lo, hi] of D^-1 A. With theta = (hi+lo)/2, delta = (hi-lo)/2,
 * sigma = theta/delta:
 *   d_0 = D^-1 r / theta,  z_1 = d_0,  res_1 = r - A d_0,  rho_0 = 1/sigma
 *   for k = 1 .. steps-1:
 *     rho_k = 1 / (2 sigma - rho_{k-1})
 *     d_k   = rho_k rho_{k-1} d_{k-1} + (2 rho_k / delta) D^-1 res_k
 *     z_{k+1} = z_k + d_k,  res_{k+1} = res_k - A d_k   (the last residual is not needed)
 * `steps` counts the updates of z; it costs steps-1 SpMVs and z = p(D^-1 A) D^-1 r with p of
 * degree steps-1. The residual recurrence res_{k+1} = res_k - A d_k is Saad's form; it equals
 * r - A z_{k+1} in exact arithmetic.
 */
void oracle_chebyshev(int64_t n, const int32_t *row, const int32_t *col, const double *val,
                      const double *r, double *z, double lo, double hi, int steps) {
  double *dinv = (double *)malloc(sizeof(double) * n);
  double *d = (double *)malloc(sizeof(double) * n);
  double *res = (double *)malloc(sizeof(double) * n);
  double *ad = (double *)malloc(sizeof(double) * n);
  for (int64_t i = 0; i < n; ++i) dinv[i] = 1.0 / diag_of_row(row, col, val, i);
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  for (int64_t i = 0; i < n; ++i) {
    d[i] = dinv[i] * r[i] / theta;
    z[i] = d[i];
    res[i] = r[i];
  }
  double rho_prev = 1.0 / sigma;
  for (int k = 1; k < steps; ++k) {
    oracle_spmv(n, row, col, val, d, 1, ad, 1);
    for (int64_t i = 0; i < n; ++i) res[i] = res[i] - ad[i];
    const double rho = 1.0 / (2.0 * sigma - rho_prev);
    const double c1 = rho * rho_prev, c2 = 2.0 * rho / delta;
    for (int64_t i = 0; i < n; ++i) {
      d[i] = c1 * d[i] + c2 * (dinv[i] * res[i]);
      z[i] = z[i] + d[i];
    }
    rho_prev = rho;
  }
  free(dinv);
  free(d);
  free(res);
  free(ad);
}

typedef struct {
  int max_iter;
  int precond;   /* 0 none, 1 Chebyshev, 2 aggregation V-cycle (amg.c) */
  int cheb_steps;
  double cheb_lo, cheb_hi;
  int singular;  /* 1: constants span the null space; check compatibility, zero-mean x at exit */
  const void *amg; /* precond 2: the hierarchy from oracle_amg_setup for this matrix */
} oracle_opts;

void oracle_amg_vcycle(const void *h, const double *r, double *z);

static void apply_prec(const oracle_opts *o, int64_t n, const int32_t *row, const int32_t *col,
                       const double *val, const double *in, double *out) {
  if (o->precond == 1)
    oracle_chebyshev(n, row, col, val, in, out, o->cheb_lo, o->cheb_hi, o->cheb_steps);
  else if (o->precond == 2)
    oracle_amg_vcycle(o->amg, in, out);
  else
    memcpy(out, in, sizeof(double) * n);
}

static int all_finite(int64_t n, const double *a) {
  for (int64_t i = 0; i < n; ++i)
    if (!isfinite(a[i])) return 0;
  return 1;
}

/*
 * BiCGStab for one right-hand side b (contiguous, length n), x in: initial guess, out: solution.
 * Right preconditioning x = M^-1 u. Stops when ||r||_2 / ||b||_2 <= tol (checked after the
 * half step on s and after the full step on r). Returns the per-column status; *iters is the
 * number of iterations begun; *relres the TRUE relative residual ||b - A x|| / ||b|| at exit.
 * Breakdown: |rho| <= 1e-300 * ||rhat|| ||r||, (rhat, v) == 0, (t, t) == 0, omega == 0, or a
 * non-finite alpha or omega (detected before x is updated, so x keeps its last finite iterate).
 */
int oracle_bicgstab(int64_t n, const int32_t *row, const int32_t *col, const double *val,
                    const double *b, double *x, double tol, const oracle_opts *o, int *iters,
                    double *relres) {
  *iters = 0;
  const double bnorm = sqrt(dot(n, b, b));
  if (!all_finite(n, b) || !all_finite(n, x)) {
    *relres = NAN;
    return OR_NONFINITE;
  }
  if (bnorm == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    *relres = 0.0;
    return OR_CONVERGED;
  }
  if (o->singular) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += b[i];
    if (fabs(s) > 1e-10 * sqrt((double)n) * bnorm) {
      *relres = NAN;
      return OR_INCOMPATIBLE;
    }
  }
  double *r = (double *)calloc(n, sizeof(double)), *rh = (double *)calloc(n, sizeof(double));
  double *p = (double *)calloc(n, sizeof(double)), *v = (double *)calloc(n, sizeof(double));
  double *ph = (double *)calloc(n, sizeof(double)), *s = (double *)calloc(n, sizeof(double));
  double *sh = (double *)calloc(n, sizeof(double)), *t = (double *)calloc(n, sizeof(double));

  oracle_spmv(n, row, col, val, x, 1, r, 1);
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
  memcpy(rh, r, sizeof(double) * n);
  const double rhnorm = sqrt(dot(n, rh, rh));
  double rho_old = 1.0, alpha = 1.0, omega = 1.0;
  int status = OR_MAXITER;
  if (sqrt(dot(n, r, r)) / bnorm <= tol) status = OR_CONVERGED;

  for (int k = 1; status == OR_MAXITER && k <= o->max_iter; ++k) {
    *iters = k;
    const double rho = dot(n, rh, r);
    if (!isfinite(rho)) { status = OR_NONFINITE; break; }
    if (fabs(rho) <= 1e-300 * rhnorm * sqrt(dot(n, r, r))) { status = OR_BREAKDOWN; break; }
    const double beta = (rho / rho_old) * (alpha / omega);
    for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
    apply_prec(o, n, row, col, val, p, ph);
    oracle_spmv(n, row, col, val, ph, 1, v, 1);
    const double rhv = dot(n, rh, v);
    /* breakdown: (rhat, v) = 0, or a step length that is not finite (x keeps its last iterate) */
    if (rhv == 0.0 || !isfinite(rho / rhv)) { status = OR_BREAKDOWN; break; }
    alpha = rho / rhv;
    for (int64_t i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
    if (sqrt(dot(n, s, s)) / bnorm <= tol) {
      for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * ph[i];
      status = OR_CONVERGED;
      break;
    }
    apply_prec(o, n, row, col, val, s, sh);
    oracle_spmv(n, row, col, val, sh, 1, t, 1);
    const double tt = dot(n, t, t);
    if (tt == 0.0 || !isfinite(dot(n, t, s) / tt)) { status = OR_BREAKDOWN; break; }
    omega = dot(n, t, s) / tt;
    for (int64_t i = 0; i < n; ++i) {
      x[i] = x[i] + alpha * ph[i] + omega * sh[i];
      r[i] = s[i] - omega * t[i];
    }
    rho_old = rho;
    const double rn = sqrt(dot(n, r, r));
    if (!isfinite(rn)) { status = OR_NONFINITE; break; }
    if (rn / bnorm <= tol) status = OR_CONVERGED;
    if (omega == 0.0 && status != OR_CONVERGED) { status = OR_BREAKDOWN; break; }
  }

  if (o->singular) { /* the solution of a singular system is fixed only up to a constant */
    double mean = 0.0;
    for (int64_t i = 0; i < n; ++i) mean += x[i];
    mean /= (double)n;
    for (int64_t i = 0; i < n; ++i) x[i] -= mean;
  }
  oracle_spmv(n, row, col, val, x, 1, r, 1);
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
  *relres = sqrt(dot(n, r, r)) / bnorm;
  free(r); free(rh); free(p); free(v); free(ph); free(s); free(sh); free(t);
  return status;
}

/* Section 2.2: the m pressure solves share A; each column is solved on its own. B, X: n x m
 * row-interleaved. tol, iters, relres, status: arrays of length m. */
void oracle_solve_block(int64_t n, const int32_t *row, const int32_t *col, const double *val, int m,
                        const double *B, double *X, const double *tol, const oracle_opts *o,
                        int *iters, double *relres, int *status) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int l = 0; l < m; ++l) {
    double *b = (double *)malloc(sizeof(double) * n), *x = (double *)malloc(sizeof(double) * n);
    for (int64_t i = 0; i < n; ++i) { b[i] = B[i * m + l]; x[i] = X[i * m + l]; }
    status[l] = oracle_bicgstab(n, row, col, val, b, x, tol[l], o, &iters[l], &relres[l]);
    for (int64_t i = 0; i < n; ++i) X[i * m + l] = x[i];
    free(b);
    free(x);
  }
}

/* Dense LU with partial pivoting on a row-major N x N matrix (overwritten); b is overwritten with
 * the solution. Returns 0, or 1 if a zero pivot is met. */
int oracle_lu_solve(int N, double *a, double *b) {
  for (int k = 0; k < N; ++k) {
    int piv = k;
    double best = fabs(a[(int64_t)k * N + k]);
    for (int i = k + 1; i < N; ++i) {
      const double v = fabs(a[(int64_t)i * N + k]);
      if (v > best) { best = v; piv = i; }
    }
    if (best == 0.0) return 1;
    if (piv != k) {
      for (int j = 0; j < N; ++j) {
        const double tmp = a[(int64_t)k * N + j];
        a[(int64_t)k * N + j] = a[(int64_t)piv * N + j];
        a[(int64_t)piv * N + j] = tmp;
      }
      const double tb = b[k]; b[k] = b[piv]; b[piv] = tb;
    }
    for (int i = k + 1; i < N; ++i) {
      const double f = a[(int64_t)i * N + k] / a[(int64_t)k * N + k];
      a[(int64_t)i * N + k] = f;
      for (int j = k + 1; j < N; ++j) a[(int64_t)i * N + j] -= f * a[(int64_t)k * N + j];
      b[i] -= f * b[k];
    }
  }
  for (int i = N - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < N; ++j) s -= a[(int64_t)i * N + j] * b[j];
    b[i] = s / a[(int64_t)i * N + i];
  }
  return 0;
}
