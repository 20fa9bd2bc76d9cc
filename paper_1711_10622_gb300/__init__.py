"""GB300 (sm_103a) hot path of the multiple-ensemble method of arXiv 1711.10622.

m pressure-Poisson solves that share one sparse matrix: the generalised SpMV Y = A X on an
n x m row-interleaved block, inside a multi-RHS BiCGStab with block vector updates, per-column
dot products and a Chebyshev polynomial preconditioner, plus the projection step around the
solve (divergence right-hand sides, pressure-gradient correction). The computation lives in the C-ABI
library libensemble_solve.so (include/ensemble_solve.h); this package is its Python binding.
"""

from .api import COL_STATUS, EnsError, Grid, Matrix, amg_apply, divergence, grad_correct, gspmv, gspmv_host, solve_batch, solve_block, solve_block_coupled, solve_opts, version  # noqa: F401

__all__ = [
    "Matrix",
    "Grid",
    "EnsError",
    "gspmv",
    "gspmv_host",
    "solve_block",
    "solve_batch",
    "solve_block_coupled",
    "solve_opts",
    "divergence",
    "amg_apply",
    "grad_correct",
    "COL_STATUS",
    "version",
]
