"""Python binding of the ensemble-solve C ABI: argument marshalling only.

Tensors are PyTorch CUDA tensors (device memory and streams come from PyTorch); every step of
the computation runs in libensemble_solve.so. Blocks are (n, m) C-contiguous tensors, i.e. the
row-interleaved layout of Section 2.3 (element (k, l) at k*m + l).
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import _native as N
from ._native import EnsError  # noqa: F401


def _stream_handle(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(t):
    import torch

    if t.dtype == torch.float64:
        return N.ENS_F64
    if t.dtype == torch.float32:
        return N.ENS_F32
    raise TypeError(f"unsupported dtype {t.dtype}; expected float64 or float32")


def _np_dtype_code(a: np.ndarray):
    if a.dtype == np.float64:
        return N.ENS_F64
    if a.dtype == np.float32:
        return N.ENS_F32
    raise TypeError(f"unsupported dtype {a.dtype}")


class Matrix:
    """A device-resident CSR matrix owned by the library (ens_create_matrix)."""

    def __init__(self, row_ptr, col_idx, val, singular: bool = False, stream=None):
        L = N.lib()
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float64)
        n = row_ptr.shape[0] - 1
        h = ctypes.c_void_p()
        st = L.ens_create_matrix(
            n,
            col_idx.shape[0],
            row_ptr.ctypes.data_as(ctypes.c_void_p),
            col_idx.ctypes.data_as(ctypes.c_void_p),
            val.ctypes.data_as(ctypes.c_void_p),
            N.ENS_MATRIX_SINGULAR if singular else 0,
            _stream_handle(stream),
            ctypes.byref(h),
        )
        N.check(st)
        self._h = h
        self.singular = bool(singular)
        n_, nnz_, mr = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        N.check(L.ens_matrix_info(self._h, ctypes.byref(n_), ctypes.byref(nnz_), ctypes.byref(mr)))
        self.n, self.nnz, self.max_row_len = n_.value, nnz_.value, mr.value

    @classmethod
    def from_operator(cls, op, stream=None):
        return cls(op.row_ptr, op.col_idx, op.val, singular=op.singular, stream=stream)

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("matrix has been destroyed")
        return self._h

    def set_f64_mode(self, mode: str):
        code = {"auto": N.ENS_F64_AUTO, "native": N.ENS_F64_NATIVE, "split": N.ENS_F64_SPLIT, "hybrid": N.ENS_F64_HYBRID}[mode]
        N.check(N.lib().ens_set_f64_mode(self.handle, code))

    def set_native_share(self, share: int):
        """Split-float FP64: 32nds of row sweeps on native DFMA (-1: library table/autotuner)."""
        N.check(N.lib().ens_set_native_share(self.handle, int(share)))

    def set_untiled(self, mode: int):
        """GSpMV row traversal: -1 autotuner's choice, 0 shared-memory tiles, 1 untiled rows."""
        N.check(N.lib().ens_set_untiled(self.handle, int(mode)))

    def autotune(self, m: int, dtype: str = "f64", stream=None) -> dict:
        """Time the GSpMV candidates for width m and keep the fastest (ens_autotune)."""
        lanes, share, us = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        code = {"f64": N.ENS_F64, "f32": N.ENS_F32}[dtype]
        N.check(
            N.lib().ens_autotune(self.handle, int(m), code, _stream_handle(stream), ctypes.byref(lanes), ctypes.byref(share), ctypes.byref(us))
        )
        ul = ctypes.c_int32()
        N.check(N.lib().ens_tuned_variant(self.handle, int(m), code, None, None, ctypes.byref(ul)))
        return {"m": int(m), "dtype": dtype, "lanes": lanes.value, "share": share.value, "untiled": bool(ul.value == 1),
                "best_us": us.value}

    def amg_setup(self, stream=None, **opts):
        """Build the aggregation multigrid hierarchy (ens_amg_setup); keyword overrides of
        ens_amg_opts: theta, max_levels, coarse_size, smooth_steps, coarse_steps, cheb_lo, cheb_hi."""
        o = N.AmgOpts()
        N.lib().ens_default_amg_opts(ctypes.byref(o))
        known = {f[0] for f in N.AmgOpts._fields_}
        for k, v in opts.items():
            if k not in known:
                raise TypeError(f"unknown AMG option {k!r}; expected one of {sorted(known)}")
            setattr(o, k, v)
        N.check(N.lib().ens_amg_setup(self.handle, ctypes.byref(o), _stream_handle(stream)))
        return self.amg_info()

    def amg_info(self) -> list:
        """[(rows, nnz)] per level of the hierarchy ([] without one)."""
        nl = ctypes.c_int32()
        N.check(N.lib().ens_amg_info(self.handle, ctypes.byref(nl), None, None))
        rows = np.zeros(max(nl.value, 1), dtype=np.int64)
        nnz = np.zeros(max(nl.value, 1), dtype=np.int64)
        N.check(N.lib().ens_amg_info(self.handle, ctypes.byref(nl), rows.ctypes.data_as(ctypes.c_void_p), nnz.ctypes.data_as(ctypes.c_void_p)))
        return [(int(rows[l]), int(nnz[l])) for l in range(nl.value)]

    def amg_level(self, level: int):
        """(row_ptr, col_idx, val, agg) of one hierarchy level (agg None on the coarsest)."""
        info = self.amg_info()
        nl, nz = info[level]
        row = np.zeros(nl + 1, dtype=np.int32)
        col = np.zeros(max(nz, 1), dtype=np.int32)
        val = np.zeros(max(nz, 1))
        agg = np.zeros(nl, dtype=np.int32) if level < len(info) - 1 else None
        vp = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        N.check(N.lib().ens_amg_level(self.handle, int(level), vp(row), vp(col), vp(val), vp(agg)))
        return row, col[:nz], val[:nz], agg

    def close(self):
        if getattr(self, "_h", None) is not None:
            N.check(N.lib().ens_destroy_matrix(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _check_block(A: Matrix, t, name):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dim() != 2 or t.shape[0] != A.n or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous ({A.n}, m) tensor, got {tuple(t.shape)}")


def gspmv(A: Matrix, X, Y=None, stream=None):
    """Y = A X (ens_gspmv); X, Y are (n, m) float64 or float32 CUDA tensors."""
    import torch

    _check_block(A, X, "X")
    if Y is None:
        Y = torch.empty_like(X)
    _check_block(A, Y, "Y")
    if Y.dtype != X.dtype or Y.shape != X.shape:
        raise ValueError("X and Y must have the same shape and dtype")
    N.check(
        N.lib().ens_gspmv(
            A.handle, X.shape[1], _dtype_code(X), ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()), _stream_handle(stream)
        )
    )
    return Y


def gspmv_host(A: Matrix, X: np.ndarray, Y: np.ndarray | None = None, stream=None) -> np.ndarray:
    """Y = A X with host arrays (ens_gspmv_host; copies inside, synchronous)."""
    if X.ndim != 2 or X.shape[0] != A.n or not X.flags.c_contiguous:
        raise ValueError(f"X must be a C-contiguous ({A.n}, m) array")
    if Y is None:
        Y = np.empty_like(X)
    if Y.shape != X.shape or Y.dtype != X.dtype or not Y.flags.c_contiguous:
        raise ValueError("Y must match X")
    N.check(
        N.lib().ens_gspmv_host(
            A.handle,
            X.shape[1],
            _np_dtype_code(X),
            X.ctypes.data_as(ctypes.c_void_p),
            Y.ctypes.data_as(ctypes.c_void_p),
            _stream_handle(stream),
        )
    )
    return Y


COL_STATUS = {0: "converged", 1: "maxiter", 2: "breakdown", 3: "nonfinite", 4: "incompatible"}


def amg_apply(A: Matrix, R, Z=None, stream=None):
    """Z = V(R): one V-cycle of A's hierarchy on an (n, m) float64/float32 CUDA block (ens_amg_apply)."""
    import torch

    _check_block(A, R, "R")
    if Z is None:
        Z = torch.empty_like(R)
    _check_block(A, Z, "Z")
    N.check(
        N.lib().ens_amg_apply(A.handle, R.shape[1], _dtype_code(R), ctypes.c_void_p(R.data_ptr()), ctypes.c_void_p(Z.data_ptr()), _stream_handle(stream))
    )
    return Z


def solve_opts(**kw) -> N.SolveOpts:
    """ens_solve_opts with the library defaults, overridden by keyword (precond / precision may be
    given by name: 'none' | 'chebyshev' | 'amg', 'f64' | 'mixed')."""
    o = N.SolveOpts()
    N.lib().ens_default_solve_opts(ctypes.byref(o))
    known = {f[0] for f in N.SolveOpts._fields_}
    for k, v in kw.items():
        if k not in known:
            raise TypeError(f"unknown solve option {k!r}; expected one of {sorted(known)}")
        if v is None:
            continue
        if k == "precond":
            v = {"none": N.ENS_PRECOND_NONE, "chebyshev": N.ENS_PRECOND_CHEBYSHEV, "amg": N.ENS_PRECOND_AMG}.get(v, v)
        if k == "precision":
            v = {"f64": N.ENS_PREC_F64, "mixed": N.ENS_PREC_MIXED}.get(v, v)
        if k == "x0_zero":
            v = int(bool(v))
        setattr(o, k, v)
    return o


def solve_block(A: Matrix, B, X=None, tol=1e-8, stream=None, **opts):
    """Solve A X = B for all m columns (ens_solve_block). B: (n, m) float64 CUDA tensor; X (same
    shape) holds the initial guess unless omitted (then x0 = 0) and receives the solution.

    Returns (X, stats) with stats = dict(iters, relres, status, outer) as numpy arrays.
    """
    import torch

    _check_block(A, B, "B")
    if B.dtype != torch.float64:
        raise TypeError("B must be float64")
    m = B.shape[1]
    if X is None:
        X = torch.zeros_like(B)
        opts.setdefault("x0_zero", True)
    _check_block(A, X, "X")
    if X.dtype != torch.float64 or X.shape != B.shape:
        raise ValueError("X must be a float64 tensor shaped like B")
    tolv = np.ascontiguousarray(np.broadcast_to(np.asarray(tol, dtype=np.float64), (m,)))
    iters = np.zeros(m, dtype=np.int32)
    relres = np.zeros(m, dtype=np.float64)
    status = np.zeros(m, dtype=np.int32)
    outer = np.zeros(m, dtype=np.int32)
    st = N.SolveStats(
        iters.ctypes.data_as(ctypes.c_void_p),
        relres.ctypes.data_as(ctypes.c_void_p),
        status.ctypes.data_as(ctypes.c_void_p),
        outer.ctypes.data_as(ctypes.c_void_p),
    )
    o = solve_opts(**opts)
    N.check(
        N.lib().ens_solve_block(
            A.handle,
            m,
            ctypes.c_void_p(B.data_ptr()),
            ctypes.c_void_p(X.data_ptr()),
            tolv.ctypes.data_as(ctypes.c_void_p),
            ctypes.byref(o),
            ctypes.byref(st),
            _stream_handle(stream),
        )
    )
    return X, {"iters": iters, "relres": relres, "status": status, "outer": outer}


def solve_block_coupled(A: Matrix, B, X=None, tol=1e-8, stream=None, **opts):
    """Coupled block BiCGStab on all m columns (ens_solve_block_coupled): one Krylov space, m x m
    step matrices. Arguments and result as solve_block; float64 only."""
    import torch

    _check_block(A, B, "B")
    if B.dtype != torch.float64:
        raise TypeError("B must be float64")
    m = B.shape[1]
    if X is None:
        X = torch.zeros_like(B)
        opts.setdefault("x0_zero", True)
    _check_block(A, X, "X")
    tolv = np.ascontiguousarray(np.broadcast_to(np.asarray(tol, dtype=np.float64), (m,)))
    st, d = _stats_arrays(m)
    o = solve_opts(**opts)
    N.check(
        N.lib().ens_solve_block_coupled(A.handle, m, ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                                        tolv.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o), ctypes.byref(st), _stream_handle(stream))
    )
    return X, d


def _stats_arrays(m):
    iters = np.zeros(m, dtype=np.int32)
    relres = np.zeros(m, dtype=np.float64)
    status = np.zeros(m, dtype=np.int32)
    outer = np.zeros(m, dtype=np.int32)
    st = N.SolveStats(
        iters.ctypes.data_as(ctypes.c_void_p),
        relres.ctypes.data_as(ctypes.c_void_p),
        status.ctypes.data_as(ctypes.c_void_p),
        outer.ctypes.data_as(ctypes.c_void_p),
    )
    return st, {"iters": iters, "relres": relres, "status": status, "outer": outer}


def solve_batch(systems, stream=None, **opts):
    """Solve several systems at once (ens_solve_batch: one CUDA graph launch).

    systems: list of (Matrix, B, X or None, tol). B: (n, m) float64 CUDA tensor; X (same shape) is the
    initial guess and receives the solution (None: a zero initial guess in a new tensor).
    Returns a list of (X, stats) in the order given.
    """
    import torch

    items = (N.BatchItem * len(systems))()
    keep = []
    out = []
    for i, (A, B, X, tol) in enumerate(systems):
        _check_block(A, B, "B")
        if B.dtype != torch.float64:
            raise TypeError("B must be float64")
        m = B.shape[1]
        if X is None:
            X = torch.zeros_like(B)
        _check_block(A, X, "X")
        if X.dtype != torch.float64 or X.shape != B.shape:
            raise ValueError("X must be a float64 tensor shaped like B")
        tolv = np.ascontiguousarray(np.broadcast_to(np.asarray(tol, dtype=np.float64), (m,)))
        st, d = _stats_arrays(m)
        keep += [tolv, st]
        items[i].A = A.handle
        items[i].m = m
        items[i].B = B.data_ptr()
        items[i].X = X.data_ptr()
        items[i].tol = tolv.ctypes.data
        items[i].stats = ctypes.pointer(st)
        out.append((X, d))
    o = solve_opts(**opts)
    N.check(N.lib().ens_solve_batch(len(systems), items, ctypes.byref(o), _stream_handle(stream)))
    return out


class RectMatrix(Matrix):
    """A row block of a distributed matrix (ens_create_matrix_rect): n_rows rows whose columns index an
    extended local vector of n_cols rows. Works with gspmv_rect."""

    def __init__(self, row_ptr, col_idx, val, n_cols: int, stream=None):
        L = N.lib()
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float64)
        h = ctypes.c_void_p()
        N.check(
            L.ens_create_matrix_rect(
                row_ptr.shape[0] - 1,
                int(n_cols),
                col_idx.shape[0],
                row_ptr.ctypes.data_as(ctypes.c_void_p),
                col_idx.ctypes.data_as(ctypes.c_void_p),
                val.ctypes.data_as(ctypes.c_void_p),
                _stream_handle(stream),
                ctypes.byref(h),
            )
        )
        self._h = h
        self.singular = False
        r, c = ctypes.c_int64(), ctypes.c_int64()
        N.check(L.ens_matrix_shape(self._h, ctypes.byref(r), ctypes.byref(c)))
        self.n, self.n_cols = r.value, c.value
        n_, nnz_, mr = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        N.check(L.ens_matrix_info(self._h, ctypes.byref(n_), ctypes.byref(nnz_), ctypes.byref(mr)))
        self.nnz, self.max_row_len = nnz_.value, mr.value


def gspmv_rect(A: RectMatrix, X, Y, stream=None):
    """Y (n_rows x m) = A X (n_cols x m) for a row block (ens_gspmv); float64 or float32 CUDA tensors."""
    if not (X.is_cuda and Y.is_cuda and X.is_contiguous() and Y.is_contiguous()):
        raise ValueError("X and Y must be contiguous CUDA tensors")
    if X.shape[0] != A.n_cols or Y.shape[0] != A.n or X.shape[1] != Y.shape[1] or X.dtype != Y.dtype:
        raise ValueError(f"shapes: X must be ({A.n_cols}, m) and Y ({A.n}, m) of one dtype")
    N.check(
        N.lib().ens_gspmv(A.handle, X.shape[1], _dtype_code(X), ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()), _stream_handle(stream))
    )
    return Y


def _ptr_array(ts):
    arr = (ctypes.c_void_p * len(ts))()
    for k, t in enumerate(ts):
        arr[k] = None if t is None else t.data_ptr()
    return arr


def _block_check(t, rows, m):
    import torch

    if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.dim() != 2 or t.shape[0] < rows or t.shape[1] != m:
        raise ValueError(f"blocks must be contiguous float64 CUDA tensors with >= {rows} rows and {m} columns")


def block_dots(pairs, rows: int, out=None, stream=None):
    """Per-column partial dots of the first `rows` rows of each pair (ens_block_dots):
    out[k*m + l] = sum_i X_k[i, l] Y_k[i, l]; pairs = [(X_0, Y_0), ...] (at most 4)."""
    import torch

    m = pairs[0][0].shape[1]
    for x, y in pairs:
        _block_check(x, rows, m)
        _block_check(y, rows, m)
    if out is None:
        out = torch.empty(len(pairs) * m, dtype=torch.float64, device=pairs[0][0].device)
    xs, ys = _ptr_array([p[0] for p in pairs]), _ptr_array([p[1] for p in pairs])
    N.check(N.lib().ens_block_dots(int(rows), m, len(pairs), xs, ys, ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
    return out


def block_lincomb(coefs, vecs, out, rows: int, stream=None):
    """out[:rows] = sum_k diag(c_k) V_k[:rows] (ens_block_lincomb); c_k: float64 CUDA tensors of m
    values or None (= 1). out may be one of the V_k."""
    m = out.shape[1]
    _block_check(out, rows, m)
    for v in vecs:
        _block_check(v, rows, m)
    for c in coefs:
        if c is not None and (c.numel() != m or not c.is_cuda or not c.is_contiguous()):
            raise ValueError("coefficients must be contiguous CUDA tensors of m values")
    N.check(
        N.lib().ens_block_lincomb(int(rows), m, len(vecs), _ptr_array(coefs), _ptr_array(vecs), ctypes.c_void_p(out.data_ptr()), _stream_handle(stream))
    )
    return out


def gather_rows(idx, X, out, stream=None):
    """out[k] = X[idx[k]] row by row (ens_gather_rows); idx an int32 CUDA tensor."""
    import torch

    if idx.dtype != torch.int32 or not idx.is_cuda:
        raise ValueError("idx must be an int32 CUDA tensor")
    m = X.shape[1]
    _block_check(X, 0, m)
    _block_check(out, idx.numel(), m)
    N.check(N.lib().ens_gather_rows(idx.numel(), m, ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
    return out


def version() -> str:
    return N.lib().ens_version().decode()


class Grid:
    """A device copy of a staggered grid for the projection step (ens_create_grid): node
    coordinates, boundary types per direction and an optional solid-cell mask."""

    BC = {"neumann": 0, "wall": 0, "periodic": 1, "dirichlet": 2}

    def __init__(self, shape, nodes, bcs, solid=None, stream=None):
        nx, ny, nz = (int(v) for v in shape)
        xn, yn, zn = (np.ascontiguousarray(a, dtype=np.float64) for a in nodes)
        bc = np.array([self.BC[b] if isinstance(b, str) else int(b) for b in bcs], dtype=np.int32)
        sp = None if solid is None else np.ascontiguousarray(np.asarray(solid, dtype=bool).reshape(-1), dtype=np.uint8)
        for a, want in ((xn, nx + 1), (yn, ny + 1), (zn, nz + 1)):
            if a.shape != (want,):
                raise ValueError("node arrays must have N + 1 entries per direction")
        if sp is not None and sp.shape != (nx * ny * nz,):
            raise ValueError("solid mask must have nx * ny * nz entries")
        h = ctypes.c_void_p()
        vp = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        N.check(
            N.lib().ens_create_grid(nx, ny, nz, vp(xn), vp(yn), vp(zn), vp(bc), vp(sp), _stream_handle(stream), ctypes.byref(h))
        )
        self._h = h
        rows, faces = ctypes.c_int64(), (ctypes.c_int64 * 3)()
        N.check(N.lib().ens_grid_info(self._h, ctypes.byref(rows), faces))
        self.n = rows.value
        self.nfaces = tuple(int(f) for f in faces)

    @classmethod
    def from_grid(cls, g, stream=None):
        """From a gen.Grid (the grid a gen operator was assembled on)."""
        return cls(g.shape, g.nodes, g.bcs, g.solid, stream=stream)

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("grid has been destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            N.check(N.lib().ens_destroy_grid(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _check_faces(G: Grid, comps, m=None):
    for d, t in enumerate(comps):
        if not t.is_cuda or t.dtype.itemsize != 8 or not t.is_floating_point() or not t.is_contiguous() or t.dim() != 2:
            raise ValueError("velocity components must be contiguous (faces, m) float64 CUDA tensors")
        if t.shape[0] != G.nfaces[d] or (m is not None and t.shape[1] != m):
            raise ValueError(f"component {d} must have shape ({G.nfaces[d]}, m)")


def divergence(G: Grid, U, V, W, scale: float = 1.0, D=None, stream=None):
    """D = scale * div(u) per fluid-cell row (ens_divergence); U, V, W are (faces_d, m) tensors."""
    import torch

    m = U.shape[1]
    _check_faces(G, (U, V, W), m)
    if D is None:
        D = torch.empty(G.n, m, dtype=torch.float64, device=U.device)
    if D.shape != (G.n, m) or D.dtype != torch.float64 or not D.is_contiguous():
        raise ValueError("D must be a contiguous (n, m) float64 tensor")
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    N.check(N.lib().ens_divergence(G.handle, m, float(scale), ptr(U), ptr(V), ptr(W), ptr(D), _stream_handle(stream)))
    return D


def grad_correct(G: Grid, P, U, V, W, tau: float, stream=None):
    """U, V, W -= tau * grad(P) on the open faces, in place (ens_grad_correct)."""
    import torch

    m = P.shape[1]
    _check_faces(G, (U, V, W), m)
    if P.shape != (G.n, m) or P.dtype != torch.float64 or not P.is_contiguous() or not P.is_cuda:
        raise ValueError("P must be a contiguous (n, m) float64 CUDA tensor")
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    N.check(N.lib().ens_grad_correct(G.handle, m, float(tau), ptr(P), ptr(U), ptr(V), ptr(W), _stream_handle(stream)))
    return U, V, W
