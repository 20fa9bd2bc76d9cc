/*
 * ensemble_project.h - the projection step around the pressure solve, for m flow states at once
 * (arXiv 1711.10622, Section 2.2, Eqs. eq2 and eq3), in libensemble_solve.so.
 *
 * Each Runge-Kutta substep of the paper's DNS predicts a velocity u*, solves the pressure Poisson
 * equation  lap p~ = (1/tau) div u*  and corrects  u~ = u* - tau grad p~. The matrix is the same
 * for every flow state; only the right-hand sides differ, so m states give one solve with m
 * right-hand sides (ens_solve_block). These calls build those right-hand sides and apply the
 * correction for all m states in one pass each.
 *
 * Grid and discretisation (the paper's staggered second-order scheme, Section 3, read as the
 * finite-volume form that matches the pressure matrix A = -L assembled with face weights
 * area / distance between cell centres):
 *   - nx x ny x nz cells on a tensor-product grid with node coordinates xn[nx+1], yn[ny+1],
 *     zn[nz+1] (strictly increasing); cells numbered x fastest; solid cells (optional mask) are
 *     removed and the fluid cells numbered in cell order give the rows of A and of the pressure.
 *   - bc[d] per direction: ENS_BC_WALL (Neumann pressure, zero normal velocity), ENS_BC_PERIODIC
 *     (at least 3 cells), ENS_BC_DIRICHLET (open boundary, p = 0 on the boundary face).
 *   - velocity component d lives on the faces normal to direction d. Along d there are N_d faces
 *     for a periodic direction (face 0 joins cells N_d-1 and 0) and N_d + 1 otherwise; face i is the
 *     low face of cell i. Component arrays are indexed like the cell array with N_d replaced by
 *     that count, m values per face, row-interleaved (face f, state l at f*m + l).
 *   - a face is open when both adjacent cells are fluid, or when it is a Dirichlet boundary face
 *     of a fluid cell; every other face is a wall (zero flux, never written).
 *   - (D u)_c = sum_d area_d(c) (u_{hi face} - u_{lo face}) over open faces (outward flux);
 *     (G p)_f = (p_hi - p_lo) / dist_f with p = 0 half a cell outside a Dirichlet face. Then
 *     D G = -A, and Eq. eq3 reads  A p = -(1/tau) D u*.
 * Conventions (streams, ownership, errors, threads) are those of ensemble_solve.h.
 */
#ifndef ENSEMBLE_PROJECT_H
#define ENSEMBLE_PROJECT_H

#include <stdint.h>

#include "ensemble_solve.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ens_grid ens_grid;

typedef enum { ENS_BC_WALL = 0, ENS_BC_PERIODIC = 1, ENS_BC_DIRICHLET = 2 } ens_bc;

/* Copy a grid description to the device (geometry, cell <-> row maps, open-face masks).
 * xn, yn, zn: host arrays of nx+1, ny+1, nz+1 node coordinates (finite, strictly increasing).
 * bc: host int32[3]. solid: host uint8[nx*ny*nz] (nonzero = solid cell, x fastest) or NULL.
 * Synchronises `stream` before returning. ENS_ERR_INVALID for bad sizes, coordinates, boundary
 * codes, a periodic direction with fewer than 3 cells, no fluid cell or more than 2^31 - 1 cells;
 * ENS_ERR_OOM / ENS_ERR_CUDA on device failures (nothing is leaked). */
ens_status ens_create_grid(int32_t nx, int32_t ny, int32_t nz, const double *xn, const double *yn, const double *zn,
                           const int32_t *bc, const uint8_t *solid, void *stream, ens_grid **out);

/* Free a grid (synchronises the device first). NULL is accepted. */
ens_status ens_destroy_grid(ens_grid *G);

/* n_rows: fluid cells (= rows of the pressure matrix); n_faces[3]: face count of each velocity
 * component array. */
ens_status ens_grid_info(const ens_grid *G, int64_t *n_rows, int64_t n_faces[3]);

/* D = scale * (D u): the divergence of m staggered velocity fields per fluid-cell row, n_rows x m
 * row-interleaved (device). With scale = -1/tau this is the right-hand side of Eq. eq3 for the
 * matrix A = -L. U, V, W: device, n_faces[d] x m. D must not overlap U, V or W. */
ens_status ens_divergence(const ens_grid *G, int32_t m, double scale, const double *U, const double *V,
                          const double *W, double *D, void *stream);

/* u -= tau * G p on every open face, in place (Eq. eq2). P: device, n_rows x m pressures. U, V, W:
 * device, n_faces[d] x m; wall faces are not written. P must not overlap U, V or W. */
ens_status ens_grad_correct(const ens_grid *G, int32_t m, double tau, const double *P, double *U, double *V,
                            double *W, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ENSEMBLE_PROJECT_H */
