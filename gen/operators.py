"""Cell-centred finite-volume 7-point pressure-Poisson operators on tensor-product grids.

The paper's SLAEs come from the pressure Poisson equation (Section 2.2, Eqs. eq2/eq3) discretised on
structured grids: a plain channel with wall-normal stretching and a channel with wall-mounted
cubes (Section 4). Those matrices are not published, so this module builds synthetic operators of the
same structure: a 7-point stencil (rows of 4..7 nonzeros), int32 CSR indices and float64 values,
the storage the traffic model of Section 2.3 assumes (4-byte integers, 8-byte floats).

Discretisation (a reading, since the paper does not print its scheme for the Poisson matrix):
``A = -L`` in volume-weighted (symmetric) form. Every open face f between cells i and j adds
``w_f = area_f / dist_f`` to ``A[i,i]`` and ``A[j,j]`` and ``-w_f`` to ``A[i,j]`` and ``A[j,i]``;
``dist_f`` is the distance between the two cell centres (wrapping across a periodic boundary).
A Dirichlet boundary face uses a mirrored ghost cell (p_ghost = -p) and adds ``2*area/width`` to
the diagonal only. Neumann walls and faces shared with a solid (removed) cell add nothing.
Each face weight is computed once and read from both sides, so A is exactly symmetric.

Cells are numbered x fastest: ``cell = x + nx*(y + ny*z)``; solid cells get no row and the
fluid cells keep their relative order. Columns inside each row are sorted ascending.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

PERIODIC = "periodic"
NEUMANN = "neumann"
DIRICHLET = "dirichlet"
_BCS = (PERIODIC, NEUMANN, DIRICHLET)


def uniform_nodes(N: int, L: float) -> np.ndarray:
    """N+1 equally spaced node coordinates on [0, L]."""
    return np.linspace(0.0, L, N + 1, dtype=np.float64)


def tanh_nodes(N: int, gamma: float, half_height: float = 1.0) -> np.ndarray:
    """Wall-normal nodes clustered at both walls: y_j = h*tanh(gamma*(2j/N-1))/tanh(gamma), j=0..N.

    The coordinates span [-h, h]; gamma controls the stretching (the ratio of the largest to
    the smallest cell width grows with gamma).
    """
    j = np.arange(N + 1, dtype=np.float64)
    return half_height * np.tanh(gamma * (2.0 * j / N - 1.0)) / np.tanh(gamma)


@dataclass
class Operator:
    """A square CSR matrix with the grid it was built on.

    row_ptr: int32[n+1], col_idx: int32[nnz], val: float64[nnz]. ``singular`` is True when no
    Dirichlet face exists, so the constants span the null space of A (and of A^T, A being
    symmetric); a right-hand side must then have zero sum to be compatible.
    """

    name: str
    shape: tuple  # (nx, ny, nz)
    bcs: tuple  # per direction
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray
    singular: bool
    cell_of_row: np.ndarray | None = None  # flat grid cell of each row (None: identity)
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def row_length_histogram(self) -> dict:
        lengths = np.diff(self.row_ptr)
        vals, counts = np.unique(lengths, return_counts=True)
        return {int(v): int(c) for v, c in zip(vals, counts)}

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col_idx, self.row_ptr), shape=(self.n, self.n))


def _face_geometry(nodes: np.ndarray, bc: str):
    """Cell widths, centres and the centre-to-centre distance across each 'plus' face.

    dist_plus[c] is the distance from cell c to cell c+1 (to cell 0 across a periodic wrap);
    NaN where the plus face is a boundary.
    """
    width = np.diff(nodes)
    centre = 0.5 * (nodes[:-1] + nodes[1:])
    N = width.shape[0]
    dist_plus = np.full(N, np.nan)
    dist_plus[:-1] = centre[1:] - centre[:-1]
    if bc == PERIODIC:
        L = nodes[-1] - nodes[0]
        dist_plus[-1] = centre[0] + L - centre[-1]
    return width, centre, dist_plus


def fv_poisson(
    xn: np.ndarray,
    yn: np.ndarray,
    zn: np.ndarray,
    bcs=(PERIODIC, NEUMANN, PERIODIC),
    solid: np.ndarray | None = None,
    name: str = "fv7",
) -> Operator:
    """Assemble the 7-point FV operator on the grid with node coordinates xn, yn, zn.

    bcs: boundary type per direction (x, y, z), each one of 'periodic', 'neumann', 'dirichlet'.
    solid: optional bool array of shape (nz, ny, nx); True cells are removed from the domain and
    their faces act as Neumann walls for the neighbouring fluid cells.
    """
    for bc in bcs:
        if bc not in _BCS:
            raise ValueError(f"unknown boundary type {bc!r}")
    nodes = (xn, yn, zn)
    dims = tuple(len(a) - 1 for a in nodes)
    nx, ny, nz = dims
    for d, bc in enumerate(bcs):
        if bc == PERIODIC and dims[d] < 3:
            raise ValueError("a periodic direction needs at least 3 cells")
    geo = [_face_geometry(nodes[d], bcs[d]) for d in range(3)]
    wx, wy, wz = geo[0][0], geo[1][0], geo[2][0]

    shape3 = (nz, ny, nx)  # C order: x fastest
    fluid = np.ones(shape3, dtype=bool) if solid is None else ~np.asarray(solid, dtype=bool)
    if fluid.shape != shape3:
        raise ValueError(f"solid mask must have shape {shape3}")
    ncell = nx * ny * nz
    fluid_flat = fluid.reshape(-1)
    n = int(fluid_flat.sum())
    rowmap = np.full(ncell, -1, dtype=np.int64)
    rowmap[fluid_flat] = np.arange(n, dtype=np.int64)

    # Face areas per direction as broadcastable 3D arrays (z, y, x).
    area = [
        (wz[:, None, None] * wy[None, :, None]) * np.ones((1, 1, nx)),  # x faces
        (wz[:, None, None] * wx[None, None, :]) * np.ones((1, ny, 1)),  # y faces
        (wy[None, :, None] * wx[None, None, :]) * np.ones((nz, 1, 1)),  # z faces
    ]
    axis_of = (2, 1, 0)  # array axis of direction d in the (z, y, x) layout
    stride_of = (1, nx, nx * ny)

    idx3 = np.arange(ncell, dtype=np.int64).reshape(shape3)
    diag = np.zeros(shape3)
    slot_cols = []
    slot_vals = []
    for d in range(3):
        ax = axis_of[d]
        width, _, dist_plus = geo[d]
        shp = [1, 1, 1]
        shp[ax] = dims[d]
        # weight of the face between c and c+1 in direction d (NaN: boundary)
        w_plus = area[d] / dist_plus.reshape(shp)
        nb_plus = np.roll(idx3, -1, axis=ax)
        nb_minus = np.roll(idx3, 1, axis=ax)
        w_minus = np.roll(w_plus, 1, axis=ax)
        fl_plus = np.roll(fluid, -1, axis=ax)
        fl_minus = np.roll(fluid, 1, axis=ax)
        pos = np.arange(dims[d]).reshape(shp)
        has_plus = np.broadcast_to(~np.isnan(dist_plus).reshape(shp), shape3) & fl_plus & fluid
        has_minus = (
            np.broadcast_to(np.roll(~np.isnan(dist_plus), 1).reshape(shp), shape3) & fl_minus & fluid
        )
        if bcs[d] != PERIODIC:
            has_minus = has_minus & (pos > 0)
        for has, nb, w in ((has_minus, nb_minus, w_minus), (has_plus, nb_plus, w_plus)):
            wv = np.where(has, w, 0.0)
            diag += wv
            slot_cols.append(np.where(has, nb, -1))
            slot_vals.append(-wv)
        if bcs[d] == DIRICHLET:
            lo = [slice(None)] * 3
            lo[ax] = 0
            hi = [slice(None)] * 3
            hi[ax] = dims[d] - 1
            a_lo = np.broadcast_to(area[d], shape3)[tuple(lo)]
            a_hi = np.broadcast_to(area[d], shape3)[tuple(hi)]
            diag[tuple(lo)] += 2.0 * a_lo / width[0]
            diag[tuple(hi)] += 2.0 * a_hi / width[-1]
    slot_cols.append(np.where(fluid, idx3, -1))
    slot_vals.append(diag)

    cols = np.stack([c.reshape(-1)[fluid_flat] for c in slot_cols], axis=1)  # (n, 7) grid cells
    vals = np.stack([v.reshape(-1)[fluid_flat] for v in slot_vals], axis=1)
    del slot_cols, slot_vals
    valid = cols >= 0
    rcols = np.where(valid, rowmap[np.where(valid, cols, 0)], np.iinfo(np.int64).max)
    order = np.argsort(rcols, axis=1, kind="stable")
    rcols = np.take_along_axis(rcols, order, axis=1)
    vals = np.take_along_axis(vals, order, axis=1)
    valid = np.take_along_axis(valid, order, axis=1)
    counts = valid.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("nnz exceeds int32 indexing")
    col_idx = rcols[valid].astype(np.int32)
    val = vals[valid].astype(np.float64)
    singular = DIRICHLET not in bcs
    op = Operator(
        name=name,
        shape=dims,
        bcs=tuple(bcs),
        row_ptr=row_ptr.astype(np.int32),
        col_idx=col_idx,
        val=val,
        singular=singular,
        cell_of_row=None if solid is None else np.nonzero(fluid_flat)[0].astype(np.int64),
    )
    op.meta["dy_ratio"] = float(wy.max() / wy.min())
    op.meta["nodes"] = tuple(np.array(a, dtype=np.float64) for a in nodes)
    op.meta["solid"] = None if solid is None else ~fluid
    return op
