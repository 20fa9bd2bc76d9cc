"""CPU FP64 oracle for the multi-RHS pressure-Poisson hot path (arXiv 1711.10622).

TEST INFRASTRUCTURE. This package is the plain, slow, obviously correct reference the CUDA
path is checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it. It shares no code with the CUDA library: the arithmetic lives in
``oracle.c`` (compiled with gcc, FP64, no FMA contraction) and in ``estimates.py`` (the paper's
closed-form performance model, Section 2.3).

Parity pins (see tests/test_oracle_pins.py): closed-form eigenpairs of the 7-point operator,
dense products on tiny grids, a textbook LU solve, Krylov termination on k-mode right-hand
sides, the Chebyshev scalar polynomial on Fourier modes, and the printed estimate columns of
Tables 4 and 5.
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build
from . import estimates  # noqa: F401  (re-exported)

CONVERGED, MAXITER, BREAKDOWN, NONFINITE, INCOMPATIBLE = 0, 1, 2, 3, 4

_lib = None
_lib_omp = None

_i64 = ctypes.c_int64
_vp = ctypes.c_void_p


class _Opts(ctypes.Structure):
    _fields_ = [
        ("max_iter", ctypes.c_int),
        ("precond", ctypes.c_int),
        ("cheb_steps", ctypes.c_int),
        ("cheb_lo", ctypes.c_double),
        ("cheb_hi", ctypes.c_double),
        ("singular", ctypes.c_int),
        ("amg", ctypes.c_void_p),
    ]


def _declare(L):
    L.oracle_spmv.argtypes = [_i64, _vp, _vp, _vp, _vp, _i64, _vp, _i64]
    L.oracle_gspmv.argtypes = [_i64, _vp, _vp, _vp, ctypes.c_int, _vp, _vp]
    L.oracle_chebyshev.argtypes = [_i64, _vp, _vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    L.oracle_bicgstab.argtypes = [_i64, _vp, _vp, _vp, _vp, _vp, ctypes.c_double, ctypes.POINTER(_Opts), _vp, _vp]
    L.oracle_bicgstab.restype = ctypes.c_int
    L.oracle_solve_block.argtypes = [_i64, _vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp, ctypes.POINTER(_Opts), _vp, _vp, _vp]
    L.oracle_lu_solve.argtypes = [ctypes.c_int, _vp, _vp]
    L.oracle_lu_solve.restype = ctypes.c_int
    L.oracle_amg_setup.argtypes = [_i64, _vp, _vp, _vp, ctypes.c_double, ctypes.c_int, _i64, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int]
    L.oracle_amg_setup.restype = _vp
    L.oracle_amg_free.argtypes = [_vp]
    L.oracle_amg_levels.argtypes = [_vp, _vp, _vp]
    L.oracle_amg_levels.restype = ctypes.c_int
    L.oracle_amg_level.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp, _vp]
    L.oracle_amg_vcycle.argtypes = [_vp, _vp, _vp]
    grid_args = [_i64, _i64, _i64, _vp, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_double]
    L.oracle_divergence.argtypes = grid_args + [_vp, _vp, _vp, _vp]
    L.oracle_grad_correct.argtypes = grid_args + [_vp, _vp, _vp, _vp]
    L.oracle_gspmv_rowwise.argtypes = [_i64, _vp, _vp, _vp, ctypes.c_int, _vp, _vp]
    L.oracle_threads.restype = ctypes.c_int
    L.oracle_block_bicgstab.argtypes = [_i64, _vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp, ctypes.POINTER(_Opts), _vp, _vp, _vp]
    L.oracle_block_bicgstab.restype = ctypes.c_int
    return L


def lib():
    """The serial oracle (the test oracle)."""
    global _lib
    if _lib is None:
        _lib = _declare(ctypes.CDLL(_build.build()))
    return _lib


def lib_omp():
    """The same sources built with OpenMP (all host cores; same results bit for bit), for the CPU
    baseline; None if the compiler lacks OpenMP."""
    global _lib_omp
    if _lib_omp is None:
        path = _build.build_omp()
        if path is None:
            return None
        _lib_omp = _declare(ctypes.CDLL(path))
    return _lib_omp


def _pick(parallel):
    if not parallel:
        return lib()
    L = lib_omp()
    if L is None:
        raise RuntimeError("the OpenMP build of the oracle is unavailable (gcc without -fopenmp)")
    return L


def threads(parallel: bool = True) -> int:
    """Threads the (OpenMP) oracle uses: omp_get_max_threads(), 1 for the serial build."""
    return int(_pick(parallel).oracle_threads())


def _p(a: np.ndarray):
    return a.ctypes.data_as(_vp)


def _csr(A):
    row = np.ascontiguousarray(A.row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(A.col_idx, dtype=np.int32)
    val = np.ascontiguousarray(A.val, dtype=np.float64)
    return row, col, val


def spmv(A, x: np.ndarray) -> np.ndarray:
    """y = A x for one vector (Section 2.3, Fig. GSpMV with m = 1)."""
    row, col, val = _csr(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(A.n, dtype=np.float64)
    lib().oracle_spmv(A.n, _p(row), _p(col), _p(val), _p(x), 1, _p(y), 1)
    return y


def gspmv(A, X: np.ndarray, parallel: bool = False) -> np.ndarray:
    """Y = A X for an n x m row-interleaved block, column by column (Section 2.3). parallel: the
    OpenMP build (rows split over the host cores; same bits)."""
    row, col, val = _csr(A)
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    m = X.shape[1]
    Y = np.empty_like(X)
    _pick(parallel).oracle_gspmv(A.n, _p(row), _p(col), _p(val), m, _p(X), _p(Y))
    return Y


def gspmv_rowwise(A, X: np.ndarray, parallel: bool = False) -> np.ndarray:
    """Y = A X with the m columns of each row together (the loop order of Fig. GSpMV); the same
    bits as gspmv()."""
    row, col, val = _csr(A)
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    m = X.shape[1]
    Y = np.empty_like(X)
    _pick(parallel).oracle_gspmv_rowwise(A.n, _p(row), _p(col), _p(val), m, _p(X), _p(Y))
    return Y


DEFAULT_CHEB_HI = 2.0
DEFAULT_CHEB_LO = 2.0 / 30.0
DEFAULT_CHEB_STEPS = 4


def chebyshev(A, r: np.ndarray, lo=DEFAULT_CHEB_LO, hi=DEFAULT_CHEB_HI, steps=DEFAULT_CHEB_STEPS):
    """z = p(D^-1 A) D^-1 r, Chebyshev iteration from zero (Saad 2003, Alg. 12.1)."""
    row, col, val = _csr(A)
    r = np.ascontiguousarray(r, dtype=np.float64)
    z = np.empty(A.n, dtype=np.float64)
    lib().oracle_chebyshev(A.n, _p(row), _p(col), _p(val), _p(r), _p(z), lo, hi, steps)
    return z


def _opts(max_iter, precond, singular, cheb_lo, cheb_hi, cheb_steps, amg=None):
    code = {"none": 0, "chebyshev": 1, "amg": 2}[precond]
    if code == 2 and amg is None:
        raise ValueError("precond='amg' needs the hierarchy (amg=oracle.AMG(...))")
    return _Opts(
        max_iter=max_iter,
        precond=code,
        cheb_steps=cheb_steps,
        cheb_lo=cheb_lo,
        cheb_hi=cheb_hi,
        singular=int(bool(singular)),
        amg=None if amg is None else amg.handle,
    )


AMG_DEFAULTS = dict(theta=0.08, max_levels=8, coarse_size=512, smooth=2, coarse=16)


class AMG:
    """Aggregation multigrid hierarchy of the oracle (amg.c): plain aggregation, Galerkin coarse
    operators P^T A P, Chebyshev smoothing; vcycle() applies one V-cycle per column."""

    def __init__(self, A, theta=0.08, max_levels=8, coarse_size=512, lo=DEFAULT_CHEB_LO, hi=DEFAULT_CHEB_HI, smooth=2, coarse=16):
        row, col, val = _csr(A)
        self._keep = (row, col, val)
        self.handle = lib().oracle_amg_setup(row.shape[0] - 1, _p(row), _p(col), _p(val), float(theta), int(max_levels),
                                             int(coarse_size), float(lo), float(hi), int(smooth), int(coarse))
        n = np.zeros(16, dtype=np.int64)
        nnz = np.zeros(16, dtype=np.int64)
        self.nlev = lib().oracle_amg_levels(self.handle, _p(n), _p(nnz))
        self.sizes = [(int(n[l]), int(nnz[l])) for l in range(self.nlev)]

    def level(self, l):
        """(row_ptr, col_idx, val, agg) of level l; agg is None on the coarsest level."""
        nl, nz = self.sizes[l]
        row = np.zeros(nl + 1, dtype=np.int32)
        col = np.zeros(max(nz, 1), dtype=np.int32)
        val = np.zeros(max(nz, 1))
        agg = np.full(nl, -1, dtype=np.int32) if l < self.nlev - 1 else None
        lib().oracle_amg_level(self.handle, l, _p(row), _p(col), _p(val), None if agg is None else _p(agg))
        return row, col[:nz], val[:nz], agg

    def vcycle(self, R: np.ndarray) -> np.ndarray:
        R = np.ascontiguousarray(R, dtype=np.float64)
        one = R.ndim == 1
        R2 = R[:, None] if one else R
        Z = np.zeros_like(R2)
        for l in range(R2.shape[1]):
            r = np.ascontiguousarray(R2[:, l])
            z = np.zeros_like(r)
            lib().oracle_amg_vcycle(self.handle, _p(r), _p(z))
            Z[:, l] = z
        return Z[:, 0] if one else Z

    def close(self):
        if getattr(self, "handle", None):
            lib().oracle_amg_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_block(
    A,
    B: np.ndarray,
    tol,
    X0: np.ndarray | None = None,
    max_iter: int = 10000,
    precond: str = "none",
    singular: bool | None = None,
    cheb_lo=DEFAULT_CHEB_LO,
    cheb_hi=DEFAULT_CHEB_HI,
    cheb_steps=DEFAULT_CHEB_STEPS,
    amg=None,
    parallel: bool = False,
):
    """m independent BiCGStab solves A x_l = b_l (Section 2.2 / 4.1); precond 'none', 'chebyshev'
    or 'amg' (with amg = an oracle.AMG hierarchy of A). parallel: the OpenMP build (columns solved
    on separate host cores; same bits).

    Returns (X, iters[m], relres[m], status[m]); relres is the true residual at exit.
    """
    row, col, val = _csr(A)
    B = np.ascontiguousarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    n, m = B.shape
    X = np.zeros_like(B) if X0 is None else np.array(X0, dtype=np.float64, order="C", copy=True)
    tolv = np.broadcast_to(np.asarray(tol, dtype=np.float64), (m,)).copy()
    iters = np.zeros(m, dtype=np.int32)
    relres = np.zeros(m, dtype=np.float64)
    status = np.zeros(m, dtype=np.int32)
    sing = A.singular if singular is None else singular
    o = _opts(max_iter, precond, sing, cheb_lo, cheb_hi, cheb_steps, amg)
    L = _pick(parallel)
    L.oracle_solve_block(
        n, _p(row), _p(col), _p(val), m, _p(B), _p(X), _p(tolv), ctypes.byref(o), _p(iters), _p(relres), _p(status)
    )
    return X, iters, relres, status


def block_solve(
    A,
    B: np.ndarray,
    tol,
    X0: np.ndarray | None = None,
    max_iter: int = 10000,
    precond: str = "none",
    singular: bool | None = None,
    cheb_lo=DEFAULT_CHEB_LO,
    cheb_hi=DEFAULT_CHEB_HI,
    cheb_steps=DEFAULT_CHEB_STEPS,
    amg=None,
):
    """Coupled block BiCGStab on all m columns at once (block_krylov.c): one Krylov space, m x m step
    matrices. Returns (X, iters[m], relres[m], status[m]) like solve_block."""
    row, col, val = _csr(A)
    B = np.ascontiguousarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    n, m = B.shape
    X = np.zeros_like(B) if X0 is None else np.array(X0, dtype=np.float64, order="C", copy=True)
    tolv = np.broadcast_to(np.asarray(tol, dtype=np.float64), (m,)).copy()
    iters = np.zeros(m, dtype=np.int32)
    relres = np.zeros(m, dtype=np.float64)
    status = np.zeros(m, dtype=np.int32)
    sing = A.singular if singular is None else singular
    o = _opts(max_iter, precond, sing, cheb_lo, cheb_hi, cheb_steps, amg)
    lib().oracle_block_bicgstab(
        n, _p(row), _p(col), _p(val), m, _p(B), _p(X), _p(tolv), ctypes.byref(o), _p(iters), _p(relres), _p(status)
    )
    return X, iters, relres, status


def lu_solve(Adense: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Dense LU with partial pivoting (textbook) on a copy of Adense."""
    a = np.array(Adense, dtype=np.float64, order="C", copy=True)
    x = np.array(b, dtype=np.float64, copy=True)
    if lib().oracle_lu_solve(a.shape[0], _p(a), _p(x)) != 0:
        raise np.linalg.LinAlgError("zero pivot")
    return x


def _grid_args(grid):
    nx, ny, nz = grid.shape
    xn, yn, zn = (np.ascontiguousarray(a, dtype=np.float64) for a in grid.nodes)
    bc = np.ascontiguousarray(grid.bc_codes, dtype=np.int32)
    rows = np.ascontiguousarray(grid.row_of_cell, dtype=np.int64)
    keep = (xn, yn, zn, bc, rows)
    return keep, [nx, ny, nz, _p(xn), _p(yn), _p(zn), _p(bc), _p(rows)]


def divergence(grid, U, V, W, scale: float = 1.0) -> np.ndarray:
    """scale * (D u) per fluid-cell row, (n, m): the outward face-flux sum of the staggered field
    (U, V, W) (projection.c; Section 2.2, Eq. eq3's right-hand side with scale = 1/tau up to the
    sign convention A = -L)."""
    comps = [np.ascontiguousarray(c, dtype=np.float64) for c in (U, V, W)]
    m = comps[0].shape[1]
    out = np.zeros((grid.n, m))
    keep, args = _grid_args(grid)
    lib().oracle_divergence(*args, m, float(scale), *(_p(c) for c in comps), _p(out))
    return out


def grad_correct(grid, P, U, V, W, tau: float):
    """(U, V, W) - tau * G p on the open faces (Section 2.2, Eq. eq2); returns new arrays."""
    comps = [np.array(c, dtype=np.float64, order="C", copy=True) for c in (U, V, W)]
    P = np.ascontiguousarray(P, dtype=np.float64)
    m = P.shape[1]
    keep, args = _grid_args(grid)
    lib().oracle_grad_correct(*args, m, float(tau), _p(P), *(_p(c) for c in comps))
    return tuple(comps)


def relerr_rows(Y: np.ndarray, Yref: np.ndarray, A, X: np.ndarray) -> float:
    """max_l ||Y_l - Yref_l||_inf / || |A| |X_l| ||_inf: the GSpMV error scale per column."""
    absA = A.to_scipy().copy()
    absA.data = np.abs(absA.data)
    scale = np.abs(absA @ np.abs(np.asarray(X).reshape(A.n, -1))).max(axis=0)
    err = np.abs(np.asarray(Y).reshape(A.n, -1) - np.asarray(Yref).reshape(A.n, -1)).max(axis=0)
    scale = np.where(scale == 0, 1.0, scale)
    return float((err / scale).max()) if err.size else 0.0


def rows_view(A, rows):
    """CSR arrays (row_ptr, col_idx, val) of the rows ``rows`` of A, columns unchanged."""
    rows = np.asarray(rows, dtype=np.int64)
    rp = np.asarray(A.row_ptr, dtype=np.int64)
    starts, ends = rp[rows], rp[rows + 1]
    lens = ends - starts
    sub_rp = np.zeros(rows.shape[0] + 1, dtype=np.int64)
    np.cumsum(lens, out=sub_rp[1:])
    total = int(sub_rp[-1])
    idx = np.arange(total, dtype=np.int64) - np.repeat(sub_rp[:-1], lens) + np.repeat(starts, lens)
    return (
        sub_rp.astype(np.int32),
        np.ascontiguousarray(A.col_idx[idx], dtype=np.int32),
        np.ascontiguousarray(A.val[idx], dtype=np.float64),
    )


def gspmv_csr(view, X: np.ndarray) -> np.ndarray:
    """Y = A_sub X for a row subset (from rows_view) of a matrix whose columns index X's rows."""
    sub_rp, sub_col, sub_val = view
    X = np.ascontiguousarray(X, dtype=np.float64)
    m = X.shape[1]
    nrows = sub_rp.shape[0] - 1
    Y = np.empty((nrows, m), dtype=np.float64)
    lib().oracle_gspmv(nrows, _p(sub_rp), _p(sub_col), _p(sub_val), m, _p(X), _p(Y))
    return Y


def gspmv_rows(A, rows, X: np.ndarray) -> np.ndarray:
    """Rows ``rows`` of Y = A X by the definition of Section 2.3, for sampled checks at full size."""
    return gspmv_csr(rows_view(A, rows), X)
