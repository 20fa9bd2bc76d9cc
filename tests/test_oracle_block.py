"""Pins of the oracle's coupled block BiCGStab (block_krylov.c; Guennouni, Jbilou and Sadok 2003,
standing in for the multiple right-hand-side extension that Section 3 names without describing).

* m = 1 is scalar BiCGStab: the block recurrences reduce to the scalar ones in exact arithmetic
  (beta = -(r~, t)/(r~, v) = (rho_new/rho)(alpha/omega)), so the first iterates agree with the
  pinned scalar oracle to rounding, with and without the Chebyshev preconditioner.
* Converged block solutions agree with a dense LU solve on 8^3 (config-1 boundary types).
* Permuting the right-hand sides permutes the iterates (R~ = R_0 moves with them).
* A = c I: the first half step is exact, x = b / c after one iteration.
* Two identical right-hand sides make R~^T V singular: BREAKDOWN at the first iteration, x = x0.
* A singular channel with zero-mean right-hand sides converges to zero-mean solutions.
"""

import numpy as np
import pytest

import gen
import oracle
from gen.operators import Operator


def _dense(op):
    return op.to_scipy().toarray()


@pytest.mark.parametrize("precond", ["none", "chebyshev"])
def test_one_column_is_scalar_bicgstab(precond):
    op = gen.dirichlet_box(8)
    b = gen.rhs_uniform(op.n, 1, 5)
    for k in range(1, 7):
        Xs, its, _, sts = oracle.solve_block(op, b, 1e-30, max_iter=k, precond=precond)
        Xb, itb, _, stb = oracle.block_solve(op, b, 1e-30, max_iter=k, precond=precond)
        assert its[0] == itb[0] == k and sts[0] == stb[0] == oracle.MAXITER
        assert np.linalg.norm(Xb - Xs) <= 1e-11 * np.linalg.norm(Xs), k
    Xs, its, _, _ = oracle.solve_block(op, b, 1e-10, precond=precond)
    Xb, itb, rr, stb = oracle.block_solve(op, b, 1e-10, precond=precond)
    assert stb[0] == 0 and rr[0] <= 1e-10 and abs(int(itb[0]) - int(its[0])) <= 1


def test_block_solution_matches_dense_lu():
    op = gen.dirichlet_box(8)
    B = gen.rhs_uniform(op.n, 4, 6)
    X, it, rr, st = oracle.block_solve(op, B, 1e-12)
    assert (st == 0).all() and np.all(rr <= 1e-12) and len(set(it.tolist())) == 1
    Ad = _dense(op)
    for l in range(4):
        xl = oracle.lu_solve(Ad, B[:, l])
        assert np.linalg.norm(X[:, l] - xl) <= 1e-8 * np.linalg.norm(xl)


def test_permuting_the_right_hand_sides_permutes_the_iterates():
    op = gen.dirichlet_box(8)
    B = gen.rhs_uniform(op.n, 3, 7)
    perm = [2, 0, 1]
    for k in (1, 3):
        X, *_ = oracle.block_solve(op, B, 1e-30, max_iter=k)
        Xp, *_ = oracle.block_solve(op, B[:, perm], 1e-30, max_iter=k)
        assert np.linalg.norm(Xp - X[:, perm]) <= 1e-12 * np.linalg.norm(X)


def _scaled_identity(n, c):
    return Operator(name="cI", shape=(n, 1, 1), bcs=("none",) * 3, row_ptr=np.arange(n + 1, dtype=np.int32),
                    col_idx=np.arange(n, dtype=np.int32), val=np.full(n, c), singular=False)


def test_scaled_identity_converges_in_one_step():
    op = _scaled_identity(100, 2.0)
    B = gen.rhs_normal(100, 3, 8)
    X, it, rr, st = oracle.block_solve(op, B, 1e-12)
    assert (st == 0).all() and (it == 1).all()
    np.testing.assert_allclose(X, B / 2.0, rtol=1e-14, atol=0)


def test_identical_columns_break_down():
    op = gen.dirichlet_box(6)
    b = gen.rhs_uniform(op.n, 1, 9)
    B = np.ascontiguousarray(np.hstack([b, b]))
    X, it, rr, st = oracle.block_solve(op, B, 1e-10)
    assert (st == oracle.BREAKDOWN).all() and (it == 1).all()
    np.testing.assert_array_equal(X, 0.0)


def test_singular_channel_zero_mean():
    op = gen.channel(16, 12, 8)
    B = gen.rhs_normal(op.n, 4, 10, zero_mean=True)
    X, it, rr, st = oracle.block_solve(op, B, 1e-10)
    assert (st == 0).all() and np.all(rr <= 1e-10)
    np.testing.assert_allclose(X.sum(axis=0), 0.0, atol=1e-9 * np.abs(X).max() * op.n)
    Xs, *_ = oracle.solve_block(op, B, 1e-12)
    assert np.all(np.linalg.norm(X - Xs, axis=0) <= 1e-6 * np.linalg.norm(Xs, axis=0))
