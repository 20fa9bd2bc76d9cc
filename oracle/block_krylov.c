/*
 * CPU FP64 oracle of the coupled block-Krylov solve (block BiCGStab).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.c): the plain reference the CUDA path is checked against.
 *
 * The paper's solver library has a multiple right-hand-side extension (Section 3) that it does not
 * describe. The independent recurrences of oracle_solve_block share every matrix product between
 * the m columns but keep the Krylov spaces apart. A block method instead builds ONE Krylov space from
 * all m columns: the step lengths are m x m matrices and every column's update mixes all columns.
 * This is the block BiCGStab of Guennouni, Jbilou and Sadok (2003), with right preconditioning
 * x = M^-1 u (M^-1 applied column by column). With R~ = R_0 (the shadow block), P_0 = R_0:
 *   V = A M^-1 P                                      (block product)
 *   alpha = (R~^T V)^-1 (R~^T R)                        (m x m, dense LU with partial pivoting)
 *   S = R - V alpha
 *   T = A M^-1 S
 *   omega = <T, S>_F / <T, T>_F                         (one scalar for the whole block)
 *   X += M^-1 P alpha + omega M^-1 S,   R = S - omega T
 *   beta = -(R~^T V)^-1 (R~^T T)
 *   P = R + (P - omega V) beta
 * For m = 1 these are the scalar BiCGStab recurrences (beta = -(r~, t)/(r~, v) equals
 * (rho_new/rho)(alpha/omega) in exact arithmetic).
 *
 * Stopping: the block stops when every column's recursive residual ||r_l|| <= tol_l ||b_l|| (after
 * the half step on S or after the full step on R), or after max_iter iterations; a column then is
 * CONVERGED if its recursive residual meets its tolerance, MAXITER otherwise. Columns with b = 0
 * (x = 0), non-finite data or, for singular operators, an incompatible right-hand side leave the
 * block before the first iteration, as in oracle_bicgstab. Breakdown (every remaining column gets
 * BREAKDOWN, x keeps its last iterate): a zero pivot in the LU of R~^T V, <T, T>_F = 0, omega = 0,
 * or a non-finite step.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_CONVERGED 0
#define OR_MAXITER 1
#define OR_BREAKDOWN 2
#define OR_NONFINITE 3
#define OR_INCOMPATIBLE 4

typedef struct {
  int max_iter;
  int precond;
  int cheb_steps;
  double cheb_lo, cheb_hi;
  int singular;
  const void *amg;
} oracle_opts;

void oracle_spmv(int64_t n, const int32_t *row, const int32_t *col, const double *val, const double *x,
                 int64_t incx, double *y, int64_t incy);
void oracle_chebyshev(int64_t n, const int32_t *row, const int32_t *col, const double *val, const double *r,
                      double *z, double lo, double hi, int steps);
void oracle_amg_vcycle(const void *h, const double *r, double *z);
int oracle_lu_solve(int N, double *a, double *b);

/* Z = M^-1 Y column by column (k columns of an n x k row-interleaved block). */
static void block_prec(const oracle_opts *o, int64_t n, const int32_t *row, const int32_t *col, const double *val,
                       int k, const double *Y, double *Z, double *tin, double *tout) {
  for (int l = 0; l < k; ++l) {
    for (int64_t i = 0; i < n; ++i) tin[i] = Y[i * k + l];
    if (o->precond == 1)
      oracle_chebyshev(n, row, col, val, tin, tout, o->cheb_lo, o->cheb_hi, o->cheb_steps);
    else if (o->precond == 2)
      oracle_amg_vcycle(o->amg, tin, tout);
    else
      memcpy(tout, tin, sizeof(double) * n);
    for (int64_t i = 0; i < n; ++i) Z[i * k + l] = tout[i];
  }
}

/* W = A Z column by column. */
static void block_spmv(int64_t n, const int32_t *row, const int32_t *col, const double *val, int k, const double *Z,
                       double *W) {
  for (int l = 0; l < k; ++l) oracle_spmv(n, row, col, val, Z + l, k, W + l, k);
}

/* C (k x k, row-major C[i*k + j]) = U^T W: C_ij = sum over rows of U[., i] W[., j], rows ascending. */
static void gram(int64_t n, int k, const double *U, const double *W, double *C) {
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      double s = 0.0;
      for (int64_t r = 0; r < n; ++r) s += U[r * k + i] * W[r * k + j];
      C[i * k + j] = s;
    }
}

/* Solve G Y = F (k x k each, row-major), G unchanged; 1 on a zero pivot. Column by column. */
static int small_solve(int k, const double *G, const double *F, double *Y, double *work) {
  double *a = work, *b = work + k * k;
  for (int j = 0; j < k; ++j) {
    memcpy(a, G, sizeof(double) * k * k);
    for (int i = 0; i < k; ++i) b[i] = F[i * k + j];
    if (oracle_lu_solve(k, a, b)) return 1;
    for (int i = 0; i < k; ++i) Y[i * k + j] = b[i];
  }
  return 0;
}

static int finite_all(int64_t count, const double *a) {
  for (int64_t i = 0; i < count; ++i)
    if (!isfinite(a[i])) return 0;
  return 1;
}

/*
 * B, X: n x m row-interleaved (X in: initial guess, out: solution); tol, iters, relres, status: m.
 * Returns the number of block iterations.
 */
int oracle_block_bicgstab(int64_t n, const int32_t *row, const int32_t *col, const double *val, int m,
                          const double *B, double *X, const double *tol, const oracle_opts *o, int *iters,
                          double *relres, int *status) {
  double *tin = (double *)malloc(sizeof(double) * n), *tout = (double *)malloc(sizeof(double) * n);
  double *bn = (double *)calloc(m, sizeof(double));
  int *act = (int *)calloc(m, sizeof(int)), *idx = (int *)calloc(m, sizeof(int));
  /* per-column start checks (as oracle_bicgstab) */
  int k = 0;
  for (int l = 0; l < m; ++l) {
    double s2 = 0.0, sum = 0.0;
    int fin = 1;
    for (int64_t i = 0; i < n; ++i) {
      const double b = B[i * m + l];
      s2 += b * b;
      sum += b;
      if (!isfinite(b) || !isfinite(X[i * m + l])) fin = 0;
    }
    bn[l] = sqrt(s2);
    iters[l] = 0;
    relres[l] = NAN;
    status[l] = OR_CONVERGED;
    if (!fin) {
      status[l] = OR_NONFINITE;
    } else if (bn[l] == 0.0) {
      for (int64_t i = 0; i < n; ++i) X[i * m + l] = 0.0;
      relres[l] = 0.0;
    } else if (o->singular && fabs(sum) > 1e-10 * sqrt((double)n) * bn[l]) {
      status[l] = OR_INCOMPATIBLE;
    } else {
      act[l] = 1;
      idx[k++] = l;
    }
  }
  int it = 0;
  if (k > 0) {
    const size_t blk = (size_t)n * k;
    double *Xb = (double *)malloc(sizeof(double) * blk), *Bb = (double *)malloc(sizeof(double) * blk);
    double *R = (double *)malloc(sizeof(double) * blk), *Rt = (double *)malloc(sizeof(double) * blk);
    double *P = (double *)malloc(sizeof(double) * blk), *Ph = (double *)malloc(sizeof(double) * blk);
    double *V = (double *)malloc(sizeof(double) * blk), *S = (double *)malloc(sizeof(double) * blk);
    double *Sh = (double *)malloc(sizeof(double) * blk), *T = (double *)malloc(sizeof(double) * blk);
    double *G = (double *)malloc(sizeof(double) * k * k), *H = (double *)malloc(sizeof(double) * k * k);
    double *al = (double *)malloc(sizeof(double) * k * k), *be = (double *)malloc(sizeof(double) * k * k);
    double *work = (double *)malloc(sizeof(double) * (k * k + k));
    double *tk = (double *)malloc(sizeof(double) * k);
    for (int64_t i = 0; i < n; ++i)
      for (int q = 0; q < k; ++q) {
        Xb[i * k + q] = X[i * m + idx[q]];
        Bb[i * k + q] = B[i * m + idx[q]];
      }
    block_spmv(n, row, col, val, k, Xb, R);
    for (size_t e = 0; e < blk; ++e) R[e] = Bb[e] - R[e];
    memcpy(Rt, R, sizeof(double) * blk);
    memcpy(P, R, sizeof(double) * blk);
    int state = OR_MAXITER; /* the block's outcome so far */
    /* converged at the start? */
    {
      int all = 1;
      for (int q = 0; q < k; ++q) {
        double s2 = 0.0;
        for (int64_t i = 0; i < n; ++i) s2 += R[i * k + q] * R[i * k + q];
        if (sqrt(s2) > tol[idx[q]] * bn[idx[q]]) all = 0;
      }
      if (all) state = OR_CONVERGED;
    }
    for (int kk = 1; state == OR_MAXITER && kk <= o->max_iter; ++kk) {
      it = kk;
      block_prec(o, n, row, col, val, k, P, Ph, tin, tout);
      block_spmv(n, row, col, val, k, Ph, V);
      gram(n, k, Rt, V, G);
      gram(n, k, Rt, R, H);
      if (small_solve(k, G, H, al, work) || !finite_all((int64_t)k * k, al)) {
        state = OR_BREAKDOWN;
        break;
      }
      for (int64_t i = 0; i < n; ++i)
        for (int q = 0; q < k; ++q) {
          double s = R[i * k + q];
          for (int p = 0; p < k; ++p) s -= V[i * k + p] * al[p * k + q];
          S[i * k + q] = s;
        }
      int all = 1;
      for (int q = 0; q < k; ++q) {
        double s2 = 0.0;
        for (int64_t i = 0; i < n; ++i) s2 += S[i * k + q] * S[i * k + q];
        if (sqrt(s2) > tol[idx[q]] * bn[idx[q]]) all = 0;
      }
      if (all) { /* half step: X += M^-1 P alpha */
        for (int64_t i = 0; i < n; ++i)
          for (int q = 0; q < k; ++q) {
            double s = Xb[i * k + q];
            for (int p = 0; p < k; ++p) s += Ph[i * k + p] * al[p * k + q];
            Xb[i * k + q] = s;
          }
        memcpy(R, S, sizeof(double) * blk);
        state = OR_CONVERGED;
        break;
      }
      block_prec(o, n, row, col, val, k, S, Sh, tin, tout);
      block_spmv(n, row, col, val, k, Sh, T);
      double ts = 0.0, tt = 0.0;
      for (size_t e = 0; e < blk; ++e) {
        ts += T[e] * S[e];
        tt += T[e] * T[e];
      }
      if (tt == 0.0 || !isfinite(ts / tt)) {
        state = OR_BREAKDOWN;
        break;
      }
      const double om = ts / tt;
      for (int64_t i = 0; i < n; ++i)
        for (int q = 0; q < k; ++q) {
          double s = Xb[i * k + q];
          for (int p = 0; p < k; ++p) s += Ph[i * k + p] * al[p * k + q];
          Xb[i * k + q] = s + om * Sh[i * k + q];
          R[i * k + q] = S[i * k + q] - om * T[i * k + q];
        }
      all = 1;
      int fin = 1;
      for (int q = 0; q < k; ++q) {
        double s2 = 0.0;
        for (int64_t i = 0; i < n; ++i) s2 += R[i * k + q] * R[i * k + q];
        if (!isfinite(s2)) fin = 0;
        if (sqrt(s2) > tol[idx[q]] * bn[idx[q]]) all = 0;
      }
      if (!fin) {
        state = OR_NONFINITE;
        break;
      }
      if (all) {
        state = OR_CONVERGED;
        break;
      }
      if (om == 0.0) {
        state = OR_BREAKDOWN;
        break;
      }
      gram(n, k, Rt, T, H);
      for (int e = 0; e < k * k; ++e) H[e] = -H[e];
      if (small_solve(k, G, H, be, work) || !finite_all((int64_t)k * k, be)) {
        state = OR_BREAKDOWN;
        break;
      }
      /* (the row's new P entries depend on its old ones: written after the row is complete) */
      for (int64_t i = 0; i < n; ++i) {
        for (int q = 0; q < k; ++q) {
          double s = R[i * k + q];
          for (int p = 0; p < k; ++p) s += (P[i * k + p] - om * V[i * k + p]) * be[p * k + q];
          tk[q] = s;
        }
        for (int q = 0; q < k; ++q) P[i * k + q] = tk[q];
      }
    }
    /* per-column outcome from the recursive residual at exit */
    for (int q = 0; q < k; ++q) {
      const int l = idx[q];
      iters[l] = it;
      if (state == OR_MAXITER) {
        double s2 = 0.0;
        for (int64_t i = 0; i < n; ++i) s2 += R[i * k + q] * R[i * k + q];
        status[l] = sqrt(s2) <= tol[l] * bn[l] ? OR_CONVERGED : OR_MAXITER;
      } else {
        status[l] = state;
      }
    }
    for (int64_t i = 0; i < n; ++i)
      for (int q = 0; q < k; ++q) X[i * m + idx[q]] = Xb[i * k + q];
    free(Xb); free(Bb); free(R); free(Rt); free(P); free(Ph); free(V); free(S); free(Sh); free(T);
    free(G); free(H); free(al); free(be); free(work); free(tk);
  }
  /* singular operators: zero-mean solutions (columns that entered the block); true residuals */
  for (int l = 0; l < m; ++l) {
    if (!act[l]) continue;
    if (o->singular) {
      double mean = 0.0;
      for (int64_t i = 0; i < n; ++i) mean += X[i * m + l];
      mean /= (double)n;
      for (int64_t i = 0; i < n; ++i) X[i * m + l] -= mean;
    }
    oracle_spmv(n, row, col, val, X + l, m, tin, 1);
    double s2 = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      const double r = B[i * m + l] - tin[i];
      s2 += r * r;
    }
    relres[l] = sqrt(s2) / bn[l];
  }
  free(tin); free(tout); free(bn); free(act); free(idx);
  return it;
}
