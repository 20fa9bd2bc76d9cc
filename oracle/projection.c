/*
 * CPU FP64 oracle for the projection step around the pressure solve (arXiv 1711.10622, Section 2.2,
 * Eqs. eq2 and eq3): the right-hand side (1/tau) div u* of the pressure Poisson equation and the
 * correction u~ = u* - tau grad p~, for m flow states at once.
 *
 * TEST INFRASTRUCTURE ONLY, like oracle.c: loaded by the tests, the smoke check and the bench's
 * CPU leg; the product library shares no code with it.
 *
 * Discretisation (the paper names a second-order staggered finite-difference scheme, Section 3,
 * without printing it; this is the reading that matches the finite-volume Poisson operator the
 * inputs are built with):
 *   - cells (i, j, k), i fastest; velocity component d lives on the faces normal to direction d;
 *     face i along d is the low face of cell i (between cells i-1 and i). A periodic direction has
 *     N faces (face 0 joins cell N-1 and cell 0), any other direction N + 1 (faces 0 and N are
 *     boundaries). Face arrays are indexed like the cell array with N replaced by the face count
 *     along d, and hold m values per face, row-interleaved (face f, state l at f*m + l).
 *   - a face is OPEN when both adjacent cells exist and are fluid, or when it is a boundary face of
 *     a Dirichlet (open) direction next to a fluid cell. Every other face (Neumann wall, faces
 *     touching a solid cell) is a WALL: zero flux, never updated.
 *   - divergence of a fluid cell: the outward flux sum over its open faces,
 *       (D u)_c = sum_d area_d(c) (u_{hi face} - u_{lo face}),
 *     area_d = the product of the cell's widths in the other two directions.
 *   - pressure gradient on an open face between fluid cells a (low side) and b (high side):
 *       (G p)_f = (p_b - p_a) / dist_f,  dist_f = distance between the cell centres (across the wrap
 *     of a periodic direction); on an open Dirichlet boundary face the boundary value is p = 0 at
 *     the face, half a cell away: (G p)_f = 2 p_c / width on the low boundary and -2 p_c / width on
 *     the high boundary.
 * With these, D G p = -A p for the operator A = -L assembled from the same face weights
 * area_f / dist_f, so the Poisson equation of Eq. eq3 becomes A p = -(1/tau) D u*.
 *
 * Grid arguments: nx, ny, nz; node coordinates xn[nx+1], yn[ny+1], zn[nz+1]; bc[3] per direction
 * (0 wall/Neumann, 1 periodic, 2 Dirichlet); row_of_cell[nx*ny*nz] = row of each cell, -1 for a
 * solid cell (rows count the fluid cells in cell order).
 */
#include <stdint.h>
#include <stdlib.h>

#define PR_WALL 0
#define PR_PERIODIC 1
#define PR_DIRICHLET 2

typedef struct {
  int64_t N[3];
  const double *nodes[3];
  const int32_t *bc;
  const int64_t *row_of_cell;
} pgrid;

static int64_t nfaces(const pgrid *g, int d) { return g->bc[d] == PR_PERIODIC ? g->N[d] : g->N[d] + 1; }

static double width(const pgrid *g, int d, int64_t i) { return g->nodes[d][i + 1] - g->nodes[d][i]; }

static double centre(const pgrid *g, int d, int64_t i) { return 0.5 * (g->nodes[d][i] + g->nodes[d][i + 1]); }

/* Flat index of cell (c[0], c[1], c[2]). */
static int64_t cell_index(const pgrid *g, const int64_t c[3]) { return c[0] + g->N[0] * (c[1] + g->N[1] * c[2]); }

/* Flat index of the face along d whose position is c (c[d] is the face number). */
static int64_t face_index(const pgrid *g, int d, const int64_t c[3]) {
  int64_t F[3] = {g->N[0], g->N[1], g->N[2]};
  F[d] = nfaces(g, d);
  return c[0] + F[0] * (c[1] + F[1] * c[2]);
}

/* Row of the cell at c, or -1 when c lies outside the grid or in a solid cell. */
static int64_t row_at(const pgrid *g, const int64_t c[3]) {
  for (int d = 0; d < 3; ++d)
    if (c[d] < 0 || c[d] >= g->N[d]) return -1;
  return g->row_of_cell[cell_index(g, c)];
}

/* The face along d at position f (f[d] = face number): adjacent rows (lo: cell f[d]-1 with wrap,
 * hi: cell f[d]) and its kind. Returns 1 for an open interior face (both rows set, *dist set),
 * 2 for an open Dirichlet boundary face (one row set, the other -1, *wid = that cell's width),
 * 0 for a wall. */
static int classify(const pgrid *g, int d, const int64_t f[3], int64_t *lo, int64_t *hi, double *dist,
                    double *wid) {
  const int64_t N = g->N[d];
  int64_t a[3] = {f[0], f[1], f[2]}, b[3] = {f[0], f[1], f[2]};
  a[d] = f[d] - 1;
  b[d] = f[d];
  int wrap = 0;
  if (g->bc[d] == PR_PERIODIC && a[d] < 0) {
    a[d] = N - 1;
    wrap = 1;
  }
  *lo = row_at(g, a);
  *hi = row_at(g, b);
  if (*lo >= 0 && *hi >= 0) {
    const double L = g->nodes[d][N] - g->nodes[d][0];
    *dist = wrap ? centre(g, d, b[d]) + L - centre(g, d, a[d]) : centre(g, d, b[d]) - centre(g, d, a[d]);
    return 1;
  }
  if (g->bc[d] == PR_DIRICHLET && f[d] == 0 && *hi >= 0) {
    *wid = width(g, d, 0);
    return 2;
  }
  if (g->bc[d] == PR_DIRICHLET && f[d] == N && *lo >= 0) {
    *wid = width(g, d, N - 1);
    return 2;
  }
  return 0;
}

/* Area of the face along d of cell c: the product of the cell's widths in the other directions. */
static double area(const pgrid *g, int d, const int64_t c[3]) {
  double a = 1.0;
  for (int e = 0; e < 3; ++e)
    if (e != d) a *= width(g, e, c[e]);
  return a;
}

static void make_grid(pgrid *g, int64_t nx, int64_t ny, int64_t nz, const double *xn, const double *yn,
                      const double *zn, const int32_t *bc, const int64_t *row_of_cell) {
  g->N[0] = nx;
  g->N[1] = ny;
  g->N[2] = nz;
  g->nodes[0] = xn;
  g->nodes[1] = yn;
  g->nodes[2] = zn;
  g->bc = bc;
  g->row_of_cell = row_of_cell;
}

/* D[r*m + l] = scale * (D u)_c for every fluid cell c (row r) and state l; u = (U, V, W). */
void oracle_divergence(int64_t nx, int64_t ny, int64_t nz, const double *xn, const double *yn, const double *zn,
                       const int32_t *bc, const int64_t *row_of_cell, int m, double scale, const double *U,
                       const double *V, const double *W, double *D) {
  pgrid g;
  make_grid(&g, nx, ny, nz, xn, yn, zn, bc, row_of_cell);
  const double *comp[3] = {U, V, W};
  int64_t c[3];
  for (c[2] = 0; c[2] < nz; ++c[2])
    for (c[1] = 0; c[1] < ny; ++c[1])
      for (c[0] = 0; c[0] < nx; ++c[0]) {
        const int64_t r = row_of_cell[cell_index(&g, c)];
        if (r < 0) continue;
        for (int l = 0; l < m; ++l) {
          double s = 0.0;
          for (int d = 0; d < 3; ++d) {
            int64_t flo[3] = {c[0], c[1], c[2]}, fhi[3] = {c[0], c[1], c[2]};
            fhi[d] = c[d] + 1;
            if (g.bc[d] == PR_PERIODIC && fhi[d] == g.N[d]) fhi[d] = 0;
            int64_t lo, hi;
            double dist, wid;
            const double a = area(&g, d, c);
            /* outward flux: + through the high face, - through the low face; walls carry none */
            if (classify(&g, d, fhi, &lo, &hi, &dist, &wid)) s += a * comp[d][face_index(&g, d, fhi) * m + l];
            if (classify(&g, d, flo, &lo, &hi, &dist, &wid)) s -= a * comp[d][face_index(&g, d, flo) * m + l];
          }
          D[r * m + l] = scale * s;
        }
      }
}

/* u -= tau * G p on every open face (Eq. eq2); wall faces are left as they are. */
void oracle_grad_correct(int64_t nx, int64_t ny, int64_t nz, const double *xn, const double *yn, const double *zn,
                         const int32_t *bc, const int64_t *row_of_cell, int m, double tau, const double *P,
                         double *U, double *V, double *W) {
  pgrid g;
  make_grid(&g, nx, ny, nz, xn, yn, zn, bc, row_of_cell);
  double *comp[3] = {U, V, W};
  for (int d = 0; d < 3; ++d) {
    int64_t F[3] = {nx, ny, nz};
    F[d] = nfaces(&g, d);
    int64_t f[3];
    for (f[2] = 0; f[2] < F[2]; ++f[2])
      for (f[1] = 0; f[1] < F[1]; ++f[1])
        for (f[0] = 0; f[0] < F[0]; ++f[0]) {
          int64_t lo, hi;
          double dist = 0.0, wid = 0.0;
          const int kind = classify(&g, d, f, &lo, &hi, &dist, &wid);
          if (kind == 0) continue;
          const int64_t fi = face_index(&g, d, f);
          for (int l = 0; l < m; ++l) {
            double grad;
            if (kind == 1)
              grad = (P[hi * m + l] - P[lo * m + l]) / dist;
            else if (hi >= 0)
              grad = 2.0 * P[hi * m + l] / wid; /* low boundary: (p_c - 0) / (width / 2) */
            else
              grad = -2.0 * P[lo * m + l] / wid; /* high boundary: (0 - p_c) / (width / 2) */
            comp[d][fi * m + l] -= tau * grad;
          }
        }
  }
}
