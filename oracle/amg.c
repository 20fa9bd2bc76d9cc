/*
 * CPU FP64 oracle for an aggregation multigrid preconditioner ("AMG-lite") for the multi-RHS
 * pressure solve. The paper's solver is BiCGStab with classical algebraic multigrid (Section 4.1);
 * this is the lighter stand-in that replaces the Chebyshev polynomial by a V-cycle whose levels
 * are built by plain aggregation and smoothed by the same Chebyshev iteration.
 *
 * TEST INFRASTRUCTURE ONLY, like oracle.c: loaded by the tests, the smoke check and the bench's
 * CPU leg; the product library shares no code with it.
 *
 * Method (Vanek, Mandel, Brezina 1996, plain aggregation; every step written out in the order
 * below, no reordering):
 *   strength   j != i is a strong neighbour of i when |a_ij| >= theta sqrt(|a_ii| |a_jj|).
 *   aggregates phase 1: rows in increasing order; a row whose strong neighbours are all free
 *              starts an aggregate with them. Phase 2: every row still free joins the phase-1
 *              aggregate of its strongest aggregated strong neighbour (largest |a_ij|, then the
 *              smallest j), judged on the phase-1 assignment. Phase 3: rows still free, in order,
 *              start an aggregate with their free strong neighbours. Aggregates are numbered in
 *              order of creation.
 *   transfer   P = piecewise constant (P_iI = 1 when row i is in aggregate I), R = P^T.
 *   coarse     A_c = P^T A P: entry (I, J) sums a_ij over i in I, j in J; every structural entry is
 *              kept; columns ascending.
 *   levels     coarsen while n > coarse_size, the level count stays below max_levels and the
 *              coarse level has at most n / 1.5 rows.
 *   smoother   the Jacobi-scaled Chebyshev iteration of oracle_chebyshev on that level's matrix
 *              (interval [lo, hi] of D^-1 A_l, `smooth` updates from a zero start).
 *   V-cycle    z = V_l(r): on the coarsest level z = Chebyshev with `coarse` updates; otherwise
 *                z = S(r); z += P V_{l+1}(R (r - A z)); z += S(r - A z)     (S = the smoother)
 *              a fixed linear operator in r.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

void oracle_spmv(int64_t n, const int32_t *row, const int32_t *col, const double *val, const double *x, int64_t incx,
                 double *y, int64_t incy);
void oracle_chebyshev(int64_t n, const int32_t *row, const int32_t *col, const double *val, const double *r,
                      double *z, double lo, double hi, int steps);

#define AMG_MAX_LEVELS 16

typedef struct {
  int64_t n;
  int32_t *row, *col;
  double *val;
  int32_t *agg; /* [n] aggregate of each row (to level + 1), NULL on the coarsest level */
  int64_t nc;   /* rows of the next level */
} amg_level;

typedef struct {
  int nlev;
  amg_level lev[AMG_MAX_LEVELS];
  double lo, hi;
  int smooth, coarse;
} oracle_amg;

static double diag_entry(const amg_level *L, int64_t i) {
  for (int32_t j = L->row[i]; j < L->row[i + 1]; ++j)
    if (L->col[j] == i) return L->val[j];
  return 0.0;
}

static int is_strong(const amg_level *L, const double *diag, int64_t i, int32_t j, double a, double theta) {
  return j != i && fabs(a) >= theta * sqrt(fabs(diag[i]) * fabs(diag[j]));
}

/* Aggregation of level L; returns the aggregate count, fills agg[n]. */
static int64_t aggregate(const amg_level *L, double theta, int32_t *agg) {
  const int64_t n = L->n;
  double *diag = (double *)malloc(sizeof(double) * n);
  for (int64_t i = 0; i < n; ++i) diag[i] = diag_entry(L, i);
  for (int64_t i = 0; i < n; ++i) agg[i] = -1;
  int64_t na = 0;
  /* phase 1 */
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    int all_free = 1;
    for (int32_t k = L->row[i]; k < L->row[i + 1]; ++k)
      if (is_strong(L, diag, i, L->col[k], L->val[k], theta) && agg[L->col[k]] >= 0) all_free = 0;
    if (!all_free) continue;
    agg[i] = (int32_t)na;
    for (int32_t k = L->row[i]; k < L->row[i + 1]; ++k)
      if (is_strong(L, diag, i, L->col[k], L->val[k], theta)) agg[L->col[k]] = (int32_t)na;
    ++na;
  }
  /* phase 2, on the phase-1 assignment */
  int32_t *p1 = (int32_t *)malloc(sizeof(int32_t) * n);
  memcpy(p1, agg, sizeof(int32_t) * n);
  for (int64_t i = 0; i < n; ++i) {
    if (p1[i] >= 0) continue;
    double best = -1.0;
    int32_t bestj = -1;
    for (int32_t k = L->row[i]; k < L->row[i + 1]; ++k) {
      const int32_t j = L->col[k];
      if (!is_strong(L, diag, i, j, L->val[k], theta) || p1[j] < 0) continue;
      const double a = fabs(L->val[k]);
      if (a > best || (a == best && j < bestj)) {
        best = a;
        bestj = j;
      }
    }
    if (bestj >= 0) agg[i] = p1[bestj];
  }
  free(p1);
  /* phase 3 */
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    agg[i] = (int32_t)na;
    for (int32_t k = L->row[i]; k < L->row[i + 1]; ++k)
      if (is_strong(L, diag, i, L->col[k], L->val[k], theta) && agg[L->col[k]] < 0) agg[L->col[k]] = (int32_t)na;
    ++na;
  }
  free(diag);
  return na;
}

/* A_c = P^T A P for piecewise-constant P: per coarse row, a small list of (column, sum). */
static void galerkin(const amg_level *L, const int32_t *agg, int64_t nc, amg_level *C) {
  int64_t *cnt = (int64_t *)calloc(nc + 1, sizeof(int64_t));
  /* rows of each aggregate */
  int64_t *start = (int64_t *)calloc(nc + 1, sizeof(int64_t));
  for (int64_t i = 0; i < L->n; ++i) start[agg[i] + 1]++;
  for (int64_t I = 0; I < nc; ++I) start[I + 1] += start[I];
  int64_t *members = (int64_t *)malloc(sizeof(int64_t) * (L->n ? L->n : 1));
  int64_t *fill = (int64_t *)calloc(nc, sizeof(int64_t));
  for (int64_t i = 0; i < L->n; ++i) members[start[agg[i]] + fill[agg[i]]++] = i;
  /* first pass: distinct columns per coarse row (linear search in a scratch list) */
  int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * 64);
  double *sums = (double *)malloc(sizeof(double) * 64);
  int64_t cap = 64;
  int64_t nnz = 0;
  int32_t **rc = (int32_t **)malloc(sizeof(int32_t *) * (nc ? nc : 1));
  double **rv = (double **)malloc(sizeof(double *) * (nc ? nc : 1));
  for (int64_t I = 0; I < nc; ++I) {
    int64_t k = 0;
    for (int64_t t = start[I]; t < start[I + 1]; ++t) {
      const int64_t i = members[t];
      for (int32_t q = L->row[i]; q < L->row[i + 1]; ++q) {
        const int32_t J = agg[L->col[q]];
        int64_t s = 0;
        while (s < k && cols[s] != J) ++s;
        if (s == k) {
          if (k == cap) {
            cap *= 2;
            cols = (int32_t *)realloc(cols, sizeof(int32_t) * cap);
            sums = (double *)realloc(sums, sizeof(double) * cap);
          }
          cols[k] = J;
          sums[k] = 0.0;
          ++k;
        }
        sums[s] += L->val[q];
      }
    }
    /* sort by column (insertion sort: rows are short) */
    for (int64_t a = 1; a < k; ++a) {
      const int32_t c = cols[a];
      const double v = sums[a];
      int64_t b = a - 1;
      while (b >= 0 && cols[b] > c) {
        cols[b + 1] = cols[b];
        sums[b + 1] = sums[b];
        --b;
      }
      cols[b + 1] = c;
      sums[b + 1] = v;
    }
    cnt[I + 1] = k;
    rc[I] = (int32_t *)malloc(sizeof(int32_t) * (k ? k : 1));
    rv[I] = (double *)malloc(sizeof(double) * (k ? k : 1));
    memcpy(rc[I], cols, sizeof(int32_t) * k);
    memcpy(rv[I], sums, sizeof(double) * k);
    nnz += k;
  }
  C->n = nc;
  C->row = (int32_t *)malloc(sizeof(int32_t) * (nc + 1));
  C->col = (int32_t *)malloc(sizeof(int32_t) * (nnz ? nnz : 1));
  C->val = (double *)malloc(sizeof(double) * (nnz ? nnz : 1));
  C->row[0] = 0;
  for (int64_t I = 0; I < nc; ++I) {
    C->row[I + 1] = (int32_t)(C->row[I] + cnt[I + 1]);
    memcpy(C->col + C->row[I], rc[I], sizeof(int32_t) * cnt[I + 1]);
    memcpy(C->val + C->row[I], rv[I], sizeof(double) * cnt[I + 1]);
    free(rc[I]);
    free(rv[I]);
  }
  C->agg = NULL;
  C->nc = 0;
  free(rc);
  free(rv);
  free(cols);
  free(sums);
  free(cnt);
  free(start);
  free(members);
  free(fill);
}

oracle_amg *oracle_amg_setup(int64_t n, const int32_t *row, const int32_t *col, const double *val, double theta,
                             int max_levels, int64_t coarse_size, double lo, double hi, int smooth, int coarse) {
  oracle_amg *h = (oracle_amg *)calloc(1, sizeof(oracle_amg));
  h->lo = lo;
  h->hi = hi;
  h->smooth = smooth;
  h->coarse = coarse;
  if (max_levels > AMG_MAX_LEVELS) max_levels = AMG_MAX_LEVELS;
  amg_level *L = &h->lev[0];
  L->n = n;
  L->row = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
  memcpy(L->row, row, sizeof(int32_t) * (n + 1));
  L->col = (int32_t *)malloc(sizeof(int32_t) * (row[n] ? row[n] : 1));
  memcpy(L->col, col, sizeof(int32_t) * row[n]);
  L->val = (double *)malloc(sizeof(double) * (row[n] ? row[n] : 1));
  memcpy(L->val, val, sizeof(double) * row[n]);
  h->nlev = 1;
  while (h->nlev < max_levels && h->lev[h->nlev - 1].n > coarse_size) {
    amg_level *F = &h->lev[h->nlev - 1];
    int32_t *agg = (int32_t *)malloc(sizeof(int32_t) * F->n);
    const int64_t nc = aggregate(F, theta, agg);
    if ((double)nc > (double)F->n / 1.5) {
      free(agg);
      break;
    }
    F->agg = agg;
    F->nc = nc;
    galerkin(F, agg, nc, &h->lev[h->nlev]);
    h->nlev++;
  }
  return h;
}

void oracle_amg_free(oracle_amg *h) {
  if (!h) return;
  for (int l = 0; l < h->nlev; ++l) {
    free(h->lev[l].row);
    free(h->lev[l].col);
    free(h->lev[l].val);
    free(h->lev[l].agg);
  }
  free(h);
}

/* Level sizes and arrays, for the tests: returns the level count; n[l], nnz[l] filled. */
int oracle_amg_levels(const oracle_amg *h, int64_t *n, int64_t *nnz) {
  for (int l = 0; l < h->nlev; ++l) {
    n[l] = h->lev[l].n;
    nnz[l] = h->lev[l].row[h->lev[l].n];
  }
  return h->nlev;
}

/* Copy level l's CSR and aggregate map (agg may be NULL; the coarsest level has none). */
void oracle_amg_level(const oracle_amg *h, int l, int32_t *row, int32_t *col, double *val, int32_t *agg) {
  const amg_level *L = &h->lev[l];
  memcpy(row, L->row, sizeof(int32_t) * (L->n + 1));
  memcpy(col, L->col, sizeof(int32_t) * L->row[L->n]);
  memcpy(val, L->val, sizeof(double) * L->row[L->n]);
  if (agg && L->agg) memcpy(agg, L->agg, sizeof(int32_t) * L->n);
}

static void vcycle(const oracle_amg *h, int l, const double *r, double *z) {
  const amg_level *L = &h->lev[l];
  const int64_t n = L->n;
  if (l == h->nlev - 1) {
    oracle_chebyshev(n, L->row, L->col, L->val, r, z, h->lo, h->hi, h->coarse);
    return;
  }
  double *res = (double *)malloc(sizeof(double) * n);
  double *az = (double *)malloc(sizeof(double) * n);
  double *dz = (double *)malloc(sizeof(double) * n);
  double *rc = (double *)calloc(L->nc, sizeof(double));
  double *zc = (double *)malloc(sizeof(double) * L->nc);
  /* pre-smoothing from zero */
  oracle_chebyshev(n, L->row, L->col, L->val, r, z, h->lo, h->hi, h->smooth);
  /* restrict the residual: rc_I = sum over i in I of (r - A z)_i */
  oracle_spmv(n, L->row, L->col, L->val, z, 1, az, 1);
  for (int64_t i = 0; i < n; ++i) res[i] = r[i] - az[i];
  for (int64_t i = 0; i < n; ++i) rc[L->agg[i]] += res[i];
  vcycle(h, l + 1, rc, zc);
  /* prolongate: z_i += zc_agg(i) */
  for (int64_t i = 0; i < n; ++i) z[i] += zc[L->agg[i]];
  /* post-smoothing on the new residual */
  oracle_spmv(n, L->row, L->col, L->val, z, 1, az, 1);
  for (int64_t i = 0; i < n; ++i) res[i] = r[i] - az[i];
  oracle_chebyshev(n, L->row, L->col, L->val, res, dz, h->lo, h->hi, h->smooth);
  for (int64_t i = 0; i < n; ++i) z[i] += dz[i];
  free(res);
  free(az);
  free(dz);
  free(rc);
  free(zc);
}

/* z = V(r) on the finest level (one column). */
void oracle_amg_vcycle(const void *h, const double *r, double *z) { vcycle((const oracle_amg *)h, 0, r, z); }
