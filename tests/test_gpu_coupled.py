"""Coupled block BiCGStab through the C ABI (ens_solve_block_coupled) against the oracle's block
solver (oracle/block_krylov.c) and the definitions it reduces to.

Bars: statuses equal the oracle's; the block iteration count within 25 % + 2 of the oracle's (the
GPU's products and Gram sums round differently, and the coupled recurrences amplify that more than
independent ones do); every converged column's true residual (oracle SpMV) <= tol and its solution
within 1e-6 of the oracle's block solution; exact breakdown inputs give the oracle's breakdown and
iterate; m = 1 reduces to the scalar BiCGStab of ens_solve_block.
"""

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ens():
    from paper_1711_10622_gb300 import build

    build.build()
    import paper_1711_10622_gb300 as ens

    return ens


def _true_relres(op, B, X):
    return np.linalg.norm(B - oracle.gspmv(op, X), axis=0) / np.linalg.norm(B, axis=0)


def _check(op, B, X, st, ref, tol):
    Xo, it_o, rr_o, st_o = ref
    np.testing.assert_array_equal(st["status"], st_o)
    assert np.all(np.abs(st["iters"] - it_o) <= 0.25 * it_o + 2), (st["iters"], it_o)
    conv = st_o == 0
    assert np.all(_true_relres(op, B, X)[conv] <= 1.05 * tol)
    for l in np.nonzero(conv)[0]:
        assert np.linalg.norm(X[:, l] - Xo[:, l]) <= 1e-6 * np.linalg.norm(Xo[:, l]), l


@pytest.mark.parametrize("m", [1, 3, 4, 8])
def test_coupled_unpreconditioned_matches_oracle(ens, m):
    op = gen.dirichlet_box(16)
    B = gen.rhs_uniform(op.n, m, 20 + m)
    tol = 1e-9
    ref = oracle.block_solve(op, B, tol)
    with ens.Matrix.from_operator(op) as A:
        X, st = ens.solve_block_coupled(A, torch.from_numpy(B).cuda(), tol=tol)
    _check(op, B, X.cpu().numpy(), st, ref, tol)


@pytest.mark.parametrize("precond", ["chebyshev", "amg"])
def test_coupled_preconditioned_matches_oracle(ens, precond):
    op = gen.cubes(48, 32, 24, size=4)
    B = gen.rhs_normal(op.n, 6, 31, zero_mean=True)
    tol = 1e-9
    H = oracle.AMG(op) if precond == "amg" else None
    ref = oracle.block_solve(op, B, tol, precond=precond, amg=H)
    with ens.Matrix.from_operator(op) as A:
        if precond == "amg":
            A.amg_setup()
        X, st = ens.solve_block_coupled(A, torch.from_numpy(B).cuda(), tol=tol, precond=precond)
    X = X.cpu().numpy()
    _check(op, B, X, st, ref, tol)
    np.testing.assert_allclose(X.sum(axis=0), 0.0, atol=1e-9 * np.abs(X).max() * op.n)


def test_coupled_one_column_is_scalar_bicgstab(ens):
    op = gen.dirichlet_box(24)
    B = torch.from_numpy(gen.rhs_uniform(op.n, 1, 40)).cuda()
    with ens.Matrix.from_operator(op) as A:
        Xc, stc = ens.solve_block_coupled(A, B, tol=1e-10)
        Xs, sts = ens.solve_block(A, B, tol=1e-10)
    # the same recurrences in exact arithmetic; over ~100 iterations the two roundings drift apart
    assert abs(int(stc["iters"][0]) - int(sts["iters"][0])) <= 0.05 * int(sts["iters"][0]) + 1
    assert torch.linalg.vector_norm(Xc - Xs) <= 1e-8 * torch.linalg.vector_norm(Xs)


def test_coupled_identical_columns_break_down(ens):
    op = gen.dirichlet_box(12)
    b = gen.rhs_uniform(op.n, 1, 41)
    B = np.ascontiguousarray(np.hstack([b, b, gen.rhs_uniform(op.n, 1, 42)]))
    Xo, it_o, _, st_o = oracle.block_solve(op, B, 1e-10)
    assert (st_o == oracle.BREAKDOWN).all() and (it_o == 1).all()
    with ens.Matrix.from_operator(op) as A:
        X, st = ens.solve_block_coupled(A, torch.from_numpy(B).cuda(), tol=1e-10)
    np.testing.assert_array_equal(st["status"], st_o)
    np.testing.assert_array_equal(st["iters"], it_o)
    np.testing.assert_array_equal(X.cpu().numpy(), 0.0)


def test_coupled_edge_columns_and_wide_block(ens):
    """b = 0 and non-finite columns leave before the first iteration; m = 32 converges."""
    op = gen.cubes(48, 32, 24, size=4)
    B = gen.rhs_normal(op.n, 32, 43, zero_mean=True)
    B[:, 5] = 0.0
    B[7, 9] = np.nan
    with ens.Matrix.from_operator(op) as A:
        X, st = ens.solve_block_coupled(A, torch.from_numpy(B).cuda(), tol=1e-8, precond="chebyshev")
    X = X.cpu().numpy()
    assert st["status"][5] == 0 and st["relres"][5] == 0 and np.all(X[:, 5] == 0)
    assert st["status"][9] == oracle.NONFINITE
    ok = [l for l in range(32) if l not in (5, 9)]
    assert np.all(st["status"][ok] == 0) and np.all(_true_relres(op, B[:, ok], X[:, ok]) <= 1.05e-8)


@pytest.mark.parametrize("mode", ["native", "split"])
def test_coupled_arithmetic_modes_match_oracle(ens, mode):
    """The Gram products and block updates run as native DFMA or as split-float products (the
    matrix's float64 mode); both meet the oracle's bars on a preconditioned solve with odd k."""
    op = gen.cubes(48, 32, 24, size=4)
    B = gen.rhs_normal(op.n, 5, 44, zero_mean=True)
    tol = 1e-9
    ref = oracle.block_solve(op, B, tol, precond="chebyshev")
    with ens.Matrix.from_operator(op) as A:
        A.set_f64_mode(mode)
        X, st = ens.solve_block_coupled(A, torch.from_numpy(B).cuda(), tol=tol, precond="chebyshev")
    _check(op, B, X.cpu().numpy(), st, ref, tol)


@pytest.mark.parametrize("scale", [2.0**60, 2.0**-60])
def test_coupled_values_outside_split_window(ens, scale):
    """Right-hand sides scaled far outside the split window [2^-40, 2^44) send every row of the
    updates and every Gram tile to native DFMA; the solve still meets the oracle's bars (the
    oracle solves the scaled system)."""
    op = gen.dirichlet_box(16)
    B = gen.rhs_uniform(op.n, 4, 45) * scale
    tol = 1e-9
    ref = oracle.block_solve(op, B, tol)
    with ens.Matrix.from_operator(op) as A:
        A.set_f64_mode("split")
        X, st = ens.solve_block_coupled(A, torch.from_numpy(B).cuda(), tol=tol)
    _check(op, B, X.cpu().numpy(), st, ref, tol)


def test_coupled_mixed_scales_across_columns(ens):
    """Columns of very different magnitude: some rows fall back, others stay split, and the
    fallback decision is per row group, so both paths meet within one update."""
    op = gen.dirichlet_box(16)
    B = gen.rhs_uniform(op.n, 4, 46)
    B[:, 1] *= 2.0**50
    B[: op.n // 2, 3] *= 2.0**-45
    tol = 1e-9
    ref = oracle.block_solve(op, B, tol)
    with ens.Matrix.from_operator(op) as A:
        A.set_f64_mode("split")
        X, st = ens.solve_block_coupled(A, torch.from_numpy(B).cuda(), tol=tol)
    _check(op, B, X.cpu().numpy(), st, ref, tol)
