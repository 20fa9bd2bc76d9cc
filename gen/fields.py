"""Staggered-grid velocity fields for the projection step around the pressure solve.

Section 2.2 (Eqs. eq2, eq3): each substep projects a preliminary velocity u* onto the divergence-
free space with the pressure of a Poisson equation whose matrix does not change; m flow states give
m right-hand sides. This module describes the grid an operator was built on (node coordinates,
boundary types, solid cells) and draws seeded preliminary velocity fields on its faces. It holds
none of the method's arithmetic (no divergence, gradient or solve).

Face layout: velocity component d lives on the faces normal to direction d. Along d a periodic
direction has N faces (face 0 joins cells N-1 and 0), any other direction N + 1; the face array of
component d is indexed like the cell array (x fastest) with N replaced by that face count, and
holds m values per face, row-interleaved ((faces, m) C-order).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .operators import DIRICHLET, PERIODIC, Operator

BC_CODES = {"neumann": 0, PERIODIC: 1, DIRICHLET: 2}


@dataclass
class Grid:
    shape: tuple  # (nx, ny, nz)
    nodes: tuple  # node coordinates per direction, lengths N+1
    bcs: tuple  # boundary type per direction
    solid: np.ndarray | None  # bool (nz, ny, nx), True = removed cell
    row_of_cell: np.ndarray  # int64 [nx*ny*nz], -1 for solid cells

    @property
    def n(self) -> int:
        return int((self.row_of_cell >= 0).sum())

    @property
    def bc_codes(self) -> np.ndarray:
        return np.array([BC_CODES[b] for b in self.bcs], dtype=np.int32)

    def face_counts(self) -> tuple:
        """Number of faces along each direction (N for periodic, N + 1 otherwise)."""
        return tuple(N if bc == PERIODIC else N + 1 for N, bc in zip(self.shape, self.bcs))

    def face_shape(self, d: int) -> tuple:
        """(nz', ny', nx') of the face array of component d."""
        dims = list(self.shape)
        dims[d] = self.face_counts()[d]
        return (dims[2], dims[1], dims[0])

    def nfaces(self, d: int) -> int:
        return int(np.prod(self.face_shape(d)))


def grid_of(op: Operator) -> Grid:
    """The grid an operator from fv_poisson was assembled on."""
    nx, ny, nz = op.shape
    ncell = nx * ny * nz
    rows = np.full(ncell, -1, dtype=np.int64)
    cells = np.arange(ncell) if op.cell_of_row is None else op.cell_of_row
    rows[cells] = np.arange(op.n, dtype=np.int64)
    return Grid(op.shape, op.meta["nodes"], op.bcs, op.meta.get("solid"), rows)


def _wall_faces(grid: Grid, d: int) -> np.ndarray:
    """bool over the face array of component d: True where the face is a wall (a Neumann boundary
    or a face touching a solid cell). Used only to zero the synthetic inputs there."""
    nx, ny, nz = grid.shape
    N = grid.shape[d]
    F = grid.face_counts()[d]
    fluid = np.ones((nz, ny, nx), dtype=bool) if grid.solid is None else ~grid.solid
    ax = (2, 1, 0)[d]
    pos = np.arange(F)
    lo = pos - 1
    hi = pos.copy()
    if grid.bcs[d] == PERIODIC:
        lo = lo % N
    lo_ok = (lo >= 0) & (lo < N)
    hi_ok = (hi >= 0) & (hi < N)
    take_lo = np.take(fluid, np.clip(lo, 0, N - 1), axis=ax)
    take_hi = np.take(fluid, np.clip(hi, 0, N - 1), axis=ax)
    shp = [1, 1, 1]
    shp[ax] = F
    lo_f = take_lo & lo_ok.reshape(shp)
    hi_f = take_hi & hi_ok.reshape(shp)
    open_ = lo_f & hi_f
    if grid.bcs[d] == DIRICHLET:
        bnd_lo = (pos == 0).reshape(shp) & hi_f
        bnd_hi = (pos == N).reshape(shp) & lo_f
        open_ = open_ | bnd_lo | bnd_hi
    return ~open_


def predictor_velocity(grid: Grid, m: int, seed: int, noise: float = 0.05):
    """m preliminary velocity fields (U, V, W), each (faces_d, m) row-interleaved.

    The base flow is the channel initial condition of Section 4.3.1, one per flow state i:
    u_i = (1 - eta^2)(3/2 + delta_i sin(2 pi z / L_z)), w_i = delta_i (1 - eta^2) sin(2 pi x / L_x),
    v = 0, with eta in [-1, 1] the normalised wall-normal coordinate and delta_i ~ U[-0.1, 0.1]
    (it is divergence-free). Seeded N(0, noise^2) perturbations on every face stand for the
    non-solenoidal part of a predictor step. Wall faces are zero.
    """
    rng = np.random.default_rng(seed)
    delta = rng.uniform(-0.1, 0.1, size=m)
    xn, yn, zn = grid.nodes
    Lx, Lz = xn[-1] - xn[0], zn[-1] - zn[0]
    yc = 0.5 * (yn[:-1] + yn[1:])
    eta = (yc - 0.5 * (yn[0] + yn[-1])) / (0.5 * (yn[-1] - yn[0]))
    prof = 1.0 - eta**2
    zc = 0.5 * (zn[:-1] + zn[1:])
    xc = 0.5 * (xn[:-1] + xn[1:])
    out = []
    for d in range(3):
        fz, fy, fx = grid.face_shape(d)
        if d == 0:  # u at x faces: position x = xn[i], y = yc[j], z = zc[k]
            base = prof[None, :, None, None] * (1.5 + delta[None, None, None, :] * np.sin(2 * np.pi * (zc - zn[0]) / Lz)[:, None, None, None])
            base = np.broadcast_to(base, (fz, fy, fx, m))
        elif d == 2:  # w at z faces: x = xc[i]
            base = delta[None, None, None, :] * prof[None, :, None, None] * np.sin(2 * np.pi * (xc - xn[0]) / Lx)[None, None, :, None]
            base = np.broadcast_to(base, (fz, fy, fx, m))
        else:
            base = np.zeros((fz, fy, fx, m))
        f = base + noise * rng.standard_normal(size=(fz, fy, fx, m))
        f[_wall_faces(grid, d)] = 0.0
        out.append(np.ascontiguousarray(f.reshape(-1, m)))
    return tuple(out)
