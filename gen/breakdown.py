"""Inputs on which BiCGStab breaks down in its first iteration, in exact arithmetic.

Input data only: a block-diagonal CSR matrix of 2 x 2 integer blocks and right-hand sides whose
entries are small integers. Every quantity of the first BiCGStab iteration is then a dyadic
rational with few bits, so floating point computes it exactly, in any summation order, on the
CPU and on the GPU alike, and the breakdown tests see exact zeros on both sides.

The matrix has two regions:
  rows [0, n1)        blocks M1 = [[-2, -2], [-2, 0]]   (invertible, det -4, indefinite)
  rows [n1, n1 + n2)  blocks M2 = [[-2, -2], [ 1, 1]]   (singular, det 0)
Columns of the block B (each zero outside its region):
  0  region 1, per 8 rows (2,-1) (2,-1) (2,-1) (0,1): b^T M1 b = 0 blockwise, so (rhat, v) = 0
  1  region 1, per 4 rows (-2,-1) (-1,1): alpha = -1/2 and (t, s) = 0, so omega = 0
  2  region 2, per 2 rows (1,1): alpha = -1, s = (-3, 3) per block and t = M2 s = 0, so (t, t) = 0
  3  region 1, seeded integers in [-3, 3]: an ordinary column (converges)
With ``patterns`` a power of 4, ||b_0|| and ||b_2|| are powers of 2, so b / ||b|| is exact too
(the mixed-precision inner solve starts from it).
"""

from __future__ import annotations

import numpy as np

from .operators import Operator

M1 = ((-2.0, -2.0), (-2.0, 0.0))
M2 = ((-2.0, -2.0), (1.0, 1.0))


def _blocks(nblocks: int, M, row0: int):
    rows, cols, vals = [], [], []
    for k in range(nblocks):
        r = row0 + 2 * k
        for i in range(2):
            for j in range(2):
                if M[i][j] != 0.0:
                    rows.append(r + i)
                    cols.append(r + j)
                    vals.append(M[i][j])
    return rows, cols, vals


def breakdown_system(patterns: int = 1024, seed: int = 17):
    """(Operator, B) with n = 12 * patterns rows and the four columns described above."""
    n1, n2 = 8 * patterns, 4 * patterns
    r1, c1, v1 = _blocks(n1 // 2, M1, 0)
    r2, c2, v2 = _blocks(n2 // 2, M2, n1)
    rows = np.array(r1 + r2, dtype=np.int64)
    cols = np.array(c1 + c2, dtype=np.int32)
    vals = np.array(v1 + v2, dtype=np.float64)
    n = n1 + n2
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    op = Operator(
        name=f"breakdown2x2_{patterns}",
        shape=(n, 1, 1),
        bcs=("none", "none", "none"),
        row_ptr=row_ptr,
        col_idx=cols,
        val=vals,
        singular=False,
        meta={"n1": n1, "n2": n2},
    )
    B = np.zeros((n, 4))
    B[:n1, 0] = np.tile([2.0, -1.0, 2.0, -1.0, 2.0, -1.0, 0.0, 1.0], patterns)
    B[:n1, 1] = np.tile([-2.0, -1.0, -1.0, 1.0], 2 * patterns)
    B[n1:, 2] = 1.0
    B[:n1, 3] = np.random.default_rng(seed).integers(-3, 4, size=n1).astype(np.float64)
    return op, B
