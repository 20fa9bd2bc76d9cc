"""Multi-GPU forms of the multiple-ensemble solve: one process per GPU.

Two ways to share the work of m simultaneous pressure solves between G ranks:

* Ensemble split: the m right-hand sides are independent (Section 2.2: every realization solves
  its own pressure equation with the same matrix), so each rank takes a contiguous share of the
  columns and solves it on its own copy of the matrix. The solve needs no communication at all;
  the results are gathered at the end. Each rank reuses its matrix reads over fewer columns.
* Row split: the paper's own parallel form, a 3D geometric decomposition (Section 3; MPI in the
  paper). Each rank owns a contiguous block of rows (z-slabs of the grid for the natural cell
  order) and keeps its vectors as an EXTENDED local block [owned rows | halo rows]. Every GSpMV
  first sends to each neighbour the owned rows it reads (one message per neighbour, m values per
  row: Section 4.1's message count, independent of m), computes the interior rows (those reading
  owned rows only) while the halo is in flight, then the boundary rows. Each BiCGStab iteration
  adds the ranks' partial dot products with three allreduces of m, 3 m and 2 m scalars.

The device work of a rank is done by the library (include/ensemble_dist.h: row-block matrices,
block dots, block linear combinations, row gather; ens_solve_block for the ensemble split). The
host side here builds the partition, posts the exchanges and reduces through a communicator:
TorchComm (torch.distributed: NCCL between GPUs, gloo between CPU processes) or any object with
the same three methods. The per-column BiCGStab scalars (alpha, beta, omega and the convergence
and breakdown tests, m values per step) are formed on the host from the allreduced dots, with the
rules of the single-GPU solver.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

CONVERGED, MAXITER, BREAKDOWN, NONFINITE, INCOMPATIBLE = 0, 1, 2, 3, 4


# ----------------------------------------------------------------------------- ensemble split
def column_shares(m: int, size: int):
    """Contiguous column ranges [c0, c1) of the m right-hand sides, one per rank, sizes differing by
    at most one (a rank may get none when m < size)."""
    base, extra = divmod(m, size)
    out, c = [], 0
    for r in range(size):
        w = base + (1 if r < extra else 0)
        out.append((c, c + w))
        c += w
    return out


def solve_ensemble_split(comm, B, solve_fn, gather: bool = True):
    """Ensemble split: this rank solves its share of the columns of B (n x m, every rank holds all
    of B, or at least its own columns) with solve_fn(B_share) -> (X_share, stats), with no
    communication; with gather, every rank then receives the whole n x m solution.

    Returns (X or X_share, stats of this rank's columns, (c0, c1))."""
    n, m = B.shape
    c0, c1 = column_shares(m, comm.size)[comm.rank]
    if c1 > c0:
        X, st = solve_fn(B[:, c0:c1])
    else:
        X, st = B[:, 0:0] * 0, {}
    if not gather:
        return X, st, (c0, c1)
    return comm.allgather_columns(X, column_shares(m, comm.size)), st, (c0, c1)


# ----------------------------------------------------------------------------- row split
def slab_bounds(n: int, size: int, plane: int | None = None):
    """Contiguous row ranges [r0, r1), one per rank, balanced by rows; with `plane` (rows per grid
    plane of the natural cell order) every boundary falls between planes (z-slabs)."""
    units = n // plane if plane and n % plane == 0 else n
    unit = n // units
    base, extra = divmod(units, size)
    out, u = [], 0
    for r in range(size):
        w = base + (1 if r < extra else 0)
        out.append((u * unit, (u + w) * unit))
        u += w
    return out


def _csr_rows(row_ptr, col_idx, val, rows):
    rp = np.asarray(row_ptr, dtype=np.int64)
    starts, ends = rp[rows], rp[rows + 1]
    lens = ends - starts
    ptr = np.zeros(rows.shape[0] + 1, dtype=np.int64)
    np.cumsum(lens, out=ptr[1:])
    idx = np.arange(int(ptr[-1]), dtype=np.int64) - np.repeat(ptr[:-1], lens) + np.repeat(starts, lens)
    return ptr, np.asarray(col_idx)[idx], np.asarray(val)[idx]


@dataclass
class RowBlock:
    """One rank's share of a row-split matrix (every rank builds its own from the global structure,
    deterministically, so no set-up messages are needed).

    Local numbering: positions 0..n_loc-1 are the owned rows, interior rows first (ascending global
    index), then boundary rows; positions n_loc.. are the halo rows (ascending global index, hence
    grouped by owner). `glob[p]` is the global row of local position p < n_loc.
    """

    rank: int
    size: int
    r0: int
    r1: int
    n_loc: int
    n_int: int
    glob: np.ndarray
    halo: np.ndarray
    recv: dict = field(default_factory=dict)  # peer -> (offset into the halo, count)
    send: dict = field(default_factory=dict)  # peer -> local positions to send, in the peer's halo order
    A_int: tuple = ()  # (row_ptr, col_idx, val) of the interior rows, extended numbering
    A_bnd: tuple = ()  # the same for the boundary rows
    n_global: int = 0

    @property
    def n_ext(self) -> int:
        return self.n_loc + int(self.halo.shape[0])


def _owner(bounds, g):
    starts = np.array([b[0] for b in bounds])
    return np.searchsorted(starts, g, side="right") - 1


def _halo_of(row_ptr, col_idx, r0, r1):
    cols = np.asarray(col_idx[row_ptr[r0] : row_ptr[r1]], dtype=np.int64)
    return np.unique(cols[(cols < r0) | (cols >= r1)])


def row_block(row_ptr, col_idx, val, bounds, rank: int) -> RowBlock:
    """Build rank `rank`'s RowBlock of the CSR matrix for the row ranges `bounds`."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col_idx = np.asarray(col_idx)
    n = row_ptr.shape[0] - 1
    r0, r1 = bounds[rank]
    n_loc = r1 - r0
    halo = _halo_of(row_ptr, col_idx, r0, r1)
    # interior: rows reading owned rows only
    rows = np.arange(r0, r1, dtype=np.int64)
    lens = np.diff(row_ptr[r0 : r1 + 1])
    cols = np.asarray(col_idx[row_ptr[r0] : row_ptr[r1]], dtype=np.int64)
    outside = ((cols < r0) | (cols >= r1)).astype(np.int64)
    per_row = np.zeros(n_loc, dtype=np.int64)
    np.add.at(per_row, np.repeat(np.arange(n_loc), lens), outside)
    interior = rows[per_row == 0]
    boundary = rows[per_row > 0]
    glob = np.concatenate([interior, boundary])
    pos = np.empty(n_loc, dtype=np.int64)
    pos[glob - r0] = np.arange(n_loc)

    def renumber(c):
        c = np.asarray(c, dtype=np.int64)
        own = (c >= r0) & (c < r1)
        out = np.empty_like(c)
        out[own] = pos[c[own] - r0]
        out[~own] = n_loc + np.searchsorted(halo, c[~own])
        return out.astype(np.int32)

    def block(rws):
        p, c, v = _csr_rows(row_ptr, col_idx, val, rws)
        return p.astype(np.int32), renumber(c), np.ascontiguousarray(v, dtype=np.float64)

    rb = RowBlock(rank=rank, size=len(bounds), r0=r0, r1=r1, n_loc=n_loc, n_int=int(interior.shape[0]), glob=glob,
                  halo=halo, A_int=block(interior), A_bnd=block(boundary), n_global=n)
    owners = _owner(bounds, halo)
    for q in np.unique(owners):
        sel = np.nonzero(owners == q)[0]
        rb.recv[int(q)] = (int(sel[0]), int(sel.shape[0]))
    # what each other rank reads from me: my rows in its halo, in its (ascending) halo order
    for q in range(len(bounds)):
        if q == rank:
            continue
        qh = _halo_of(row_ptr, col_idx, *bounds[q])
        mine = qh[(qh >= r0) & (qh < r1)]
        if mine.size:
            rb.send[q] = pos[mine - r0].astype(np.int32)
    return rb


# ----------------------------------------------------------------------------- communicators
class TorchComm:
    """torch.distributed communicator (initialised process group): NCCL between GPUs, gloo between
    CPU processes. exchange() posts every send and receive at once and returns the handles."""

    def __init__(self, group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def exchange(self, sends: dict, recvs: dict):
        works = []
        for q, t in recvs.items():
            works.append(self.dist.irecv(t, src=q, group=self.group))
        for q, t in sends.items():
            works.append(self.dist.isend(t, dst=q, group=self.group))
        return works

    def wait(self, works):
        for w in works:
            w.wait()

    def allreduce(self, t):
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t

    def allgather_columns(self, X, shares):
        import torch

        width = max(c1 - c0 for c0, c1 in shares)
        pad = torch.zeros((X.shape[0], width), dtype=X.dtype, device=X.device)
        pad[:, : X.shape[1]] = X
        parts = [torch.empty_like(pad) for _ in range(self.size)]
        self.dist.all_gather(parts, pad.contiguous(), group=self.group)
        return torch.cat([p[:, : c1 - c0] for p, (c0, c1) in zip(parts, shares)], dim=1).contiguous()


# ----------------------------------------------------------------------------- device ops
class CudaOps:
    """The library's device work for one rank (ensemble_dist.h), on PyTorch CUDA tensors."""

    def __init__(self, device=None, stream=None):
        import torch

        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.stream = stream

    def _s(self):
        import ctypes

        st = self.stream or self.torch.cuda.current_stream(self.device)
        return ctypes.c_void_p(st.cuda_stream)

    def matrix(self, csr, n_cols):
        from .api import RectMatrix

        return RectMatrix(*csr, n_cols=n_cols) if len(csr[0]) > 1 else None

    def zeros(self, rows, m):
        return self.torch.zeros((rows, m), dtype=self.torch.float64, device=self.device)

    def from_host(self, a, dtype=None):
        return self.torch.from_numpy(np.ascontiguousarray(a if dtype is None else a.astype(dtype))).to(self.device)

    def to_host(self, t):
        return t.cpu().numpy()

    def gspmv(self, A, X, Y):
        if A is not None:
            from .api import gspmv_rect

            gspmv_rect(A, X, Y, stream=self.stream)

    def dots(self, pairs, rows):
        from .api import block_dots

        return block_dots(pairs, rows, stream=self.stream)

    def lincomb(self, coefs, vecs, out, rows):
        from .api import block_lincomb

        block_lincomb(coefs, vecs, out, rows, stream=self.stream)

    def gather(self, idx, X, out):
        from .api import gather_rows

        gather_rows(idx, X, out, stream=self.stream)

    def synchronize(self):
        (self.stream or self.torch.cuda.current_stream(self.device)).synchronize()


class DistMatrix:
    """A row-split matrix on one rank: its RowBlock, the interior and boundary row blocks on the
    device, the send index lists and the exchange buffers for block width m."""

    def __init__(self, rb: RowBlock, ops, m: int):
        self.rb, self.ops, self.m = rb, ops, m
        self.A_int = ops.matrix(rb.A_int, rb.n_ext)
        self.A_bnd = ops.matrix(rb.A_bnd, rb.n_ext)
        self.send_idx = {q: ops.from_host(ix, np.int32) for q, ix in rb.send.items()}
        self.send_buf = {q: ops.zeros(len(ix), m) for q, ix in rb.send.items()}

    def gspmv(self, comm, X_ext, Y):
        """Y (n_loc x m) = local rows of A X, X_ext (n_ext x m) holding this rank's owned rows; its halo
        rows are filled here. Interior rows are computed while the halo messages are in flight. The
        transport must order its reads after the work already queued on the caller's stream (as
        torch.distributed does for NCCL; gloo on CPU tensors is synchronous)."""
        rb = self.rb
        for q, ix in self.send_idx.items():
            self.ops.gather(ix, X_ext, self.send_buf[q])
        recvs = {q: X_ext[rb.n_loc + off : rb.n_loc + off + cnt] for q, (off, cnt) in rb.recv.items()}
        works = comm.exchange(self.send_buf, recvs)
        self.ops.gspmv(self.A_int, X_ext, Y[: rb.n_int])
        comm.wait(works)
        self.ops.gspmv(self.A_bnd, X_ext, Y[rb.n_int :])
        return Y


@dataclass
class DistResult:
    X_loc: object  # owned rows of the solution, local order (RowBlock.glob)
    iters: np.ndarray
    relres: np.ndarray
    status: np.ndarray
    allreduces: int = 0


def dist_bicgstab(comm, ops, rb: RowBlock, B_loc, tol, max_iter: int = 10000, singular: bool = False,
                  X0_loc=None) -> DistResult:
    """m independent BiCGStab solves (right preconditioning with M = I) on a row-split matrix: the
    per-column recurrences, stopping tests and breakdown rules of the single-GPU solver, with every
    dot product formed as local partial dots plus an allreduce and every product a halo-exchange
    GSpMV. Three allreduces per iteration: (rhat, v) [m scalars]; ||s||^2, (t, s), (t, t) [3 m];
    ||r||^2, (rhat, r) [2 m]. The dots are computed directly (no recurrence-derived norms), so every
    stopping decision is taken on the same quantities as in the single-GPU solver and the oracle.

    B_loc: (n_loc, m) owned rows of B in local order (rows rb.glob). Returns the owned rows of x."""
    m = int(B_loc.shape[1])
    n_loc, n_ext = rb.n_loc, rb.n_ext
    tolv = np.broadcast_to(np.asarray(tol, dtype=np.float64), (m,)).copy()
    D = DistMatrix(rb, ops, m)
    nred = [0]

    def reduce(pairs):
        d = ops.dots(pairs, n_loc)
        comm.allreduce(d)
        nred[0] += 1
        return np.asarray(ops.to_host(d), dtype=np.float64).reshape(len(pairs), m)

    def coef(v):
        return ops.from_host(np.asarray(v, dtype=np.float64))

    b = B_loc
    x_ext = ops.zeros(n_ext, m)  # x as an extended block (its halo is exchanged for r = b - A x)
    if X0_loc is not None:
        x_ext[:n_loc] = X0_loc
    r, rh, v, s, t = (ops.zeros(n_loc, m) for _ in range(5))
    p_ext, s_ext = ops.zeros(n_ext, m), ops.zeros(n_ext, m)
    ones = ops.from_host(np.ones((n_loc, m)))
    status = np.full(m, CONVERGED, dtype=np.int32)
    iters = np.zeros(m, dtype=np.int32)
    active = np.ones(m, dtype=bool)

    # r = b - A x, rhat = r; ||b||^2, ||r||^2 and (singular) sum(b) in one allreduce
    D.gspmv(comm, x_ext, r)
    ops.lincomb([None, coef(-np.ones(m))], [b, r], r, n_loc)
    ops.lincomb([None], [r], rh, n_loc)
    red = reduce([(b, b), (r, r)] + ([(b, ones)] if singular else []))
    bn2, rn2 = red[0], red[1]
    early = np.zeros(m, dtype=bool)
    zero_b = bn2 == 0.0
    nonfinite = ~np.isfinite(bn2) | ~np.isfinite(rn2)
    status[nonfinite] = NONFINITE
    early |= nonfinite | zero_b
    if singular:
        incompat = ~early & (np.abs(red[2]) > 1e-10 * np.sqrt(float(rb.n_global)) * np.sqrt(bn2))
        status[incompat] = INCOMPATIBLE
        early |= incompat
    thr2 = tolv * tolv * bn2
    active &= ~early & ~(rn2 <= thr2)
    rh2 = rn2.copy()
    rho = rn2.copy()
    rho_old = np.ones(m)
    alpha = np.ones(m)
    omega = np.ones(m)
    it = 0
    while active.any() and it < max_iter:
        it += 1
        iters[active] = it
        # p = r + beta (p - omega v) (converged columns: coefficients 0, p unused)
        beta = np.where(active, (rho / rho_old) * (alpha / np.where(omega == 0, 1.0, omega)), 0.0)
        ops.lincomb([None, coef(beta), coef(-beta * omega)], [r, p_ext[:n_loc], v], p_ext[:n_loc], n_loc)
        D.gspmv(comm, p_ext, v)
        rv = reduce([(rh, v)])[0]
        with np.errstate(divide="ignore", invalid="ignore"):
            al = rho / rv
        brk = active & ((rv == 0.0) | ~np.isfinite(al))
        status[brk] = BREAKDOWN
        active &= ~brk
        alpha = np.where(active, al, 0.0)
        # s = r - alpha v, t = A s; ||s||^2 (half-step test), (t, s), (t, t) in ONE allreduce of 3 m
        # scalars. t is also formed for columns that stop at the half step; they do not use it.
        ops.lincomb([None, coef(-alpha)], [r, v], s_ext[:n_loc], n_loc)
        D.gspmv(comm, s_ext, t)
        red3 = reduce([(s_ext[:n_loc], s_ext[:n_loc]), (t, s_ext[:n_loc]), (t, t)])
        ss, ts, tt = red3[0], red3[1], red3[2]
        half = active & (ss <= thr2)
        if half.any():  # x += alpha p for the columns converged at the half step
            ops.lincomb([None, coef(np.where(half, alpha, 0.0))], [x_ext[:n_loc], p_ext[:n_loc]], x_ext[:n_loc], n_loc)
            status[half] = CONVERGED
            active &= ~half
        if not active.any():
            break
        with np.errstate(divide="ignore", invalid="ignore"):
            om = ts / tt
        brk = active & ((tt == 0.0) | ~np.isfinite(om))
        status[brk] = BREAKDOWN
        active &= ~brk
        omega = np.where(active, om, 0.0)
        a_x, o_x = np.where(active, alpha, 0.0), omega
        ops.lincomb([None, coef(a_x), coef(o_x)], [x_ext[:n_loc], p_ext[:n_loc], s_ext[:n_loc]], x_ext[:n_loc], n_loc)
        ops.lincomb([None, coef(-omega)], [s_ext[:n_loc], t], r, n_loc)
        rr = reduce([(r, r), (rh, r)])
        rn2, rhor = rr[0], rr[1]
        nf = active & ~np.isfinite(rn2)
        status[nf] = NONFINITE
        active &= ~nf
        conv = active & (rn2 <= thr2)
        status[conv] = CONVERGED
        active &= ~conv
        om0 = active & (omega == 0.0)
        status[om0] = BREAKDOWN
        active &= ~om0
        rho_old = np.where(active, rho, rho_old)
        if it < max_iter:  # the next iteration's rho and its breakdown test
            nf = active & ~np.isfinite(rhor)
            status[nf] = NONFINITE
            iters[nf] = it + 1
            active &= ~nf
            tiny = active & (np.abs(rhor) <= 1e-300 * np.sqrt(rh2) * np.sqrt(rn2))
            status[tiny] = BREAKDOWN
            iters[tiny] = it + 1
            active &= ~tiny
            rho = np.where(active, rhor, rho)
    status[active] = MAXITER
    x_loc = x_ext[:n_loc]
    if zero_b.any():
        ops.lincomb([coef(np.where(zero_b, 0.0, 1.0))], [x_loc], x_loc, n_loc)
    if singular:  # zero-mean solution (columns that iterated)
        mean = reduce([(x_loc, ones)])[0] / float(rb.n_global)
        ops.lincomb([None, coef(np.where(early, 0.0, -mean))], [x_loc, ones], x_loc, n_loc)
    # true residual ||b - A x|| / ||b||
    D.gspmv(comm, x_ext, r)
    ops.lincomb([None, coef(-np.ones(m))], [b, r], r, n_loc)
    tr = reduce([(r, r)])[0]
    with np.errstate(divide="ignore", invalid="ignore"):
        relres = np.where(zero_b, 0.0, np.where(early & ~zero_b, np.nan, np.sqrt(tr / bn2)))
    return DistResult(X_loc=x_loc, iters=iters, relres=relres, status=status, allreduces=nred[0])
