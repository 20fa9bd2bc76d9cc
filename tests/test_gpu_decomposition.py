"""Multi-GPU decomposition through the library's device work (include/ensemble_dist.h) on one GPU.

The building blocks against plain definitions: row-block GSpMV (Fig. GSpMV on a rectangular block;
1e-12 of |A||X| against the oracle), per-column block dots (1e-13 relative to sum |x y|), block
linear combinations, row gather (exact). Then the row split and the ensemble split driven with the
CUDA blocks, G ranks emulated as host threads on this one GPU (tests/dist_thread_comm.py): the halo
product against the oracle's global product, the distributed BiCGStab against the oracle's solves
(statuses, iterations within 25 % + 2, solutions within 1e-6; the exact breakdown inputs give the
oracle's breakdowns and iterates exactly), the ensemble split against one block solve.
"""

import os
import sys

import numpy as np
import pytest

import gen
import oracle
from gen.breakdown import breakdown_system

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ens():
    from paper_1711_10622_gb300 import build

    build.build()
    import paper_1711_10622_gb300 as ens

    return ens


def _scale(csr, n_cols, X):
    import scipy.sparse as sp

    rp, ci, v = csr
    S = sp.csr_matrix((np.abs(v), ci, rp), shape=(len(rp) - 1, n_cols))
    return S @ np.abs(X)


@pytest.mark.parametrize("m", [1, 3, 8, 32])
def test_row_block_gspmv(ens, m):
    from paper_1711_10622_gb300 import api
    from paper_1711_10622_gb300 import decomposition as dc

    op = gen.cubes(48, 32, 24, size=4)
    bounds = dc.slab_bounds(op.n, 3, plane=48 * 32)
    rb = dc.row_block(op.row_ptr, op.col_idx, op.val, bounds, 1)
    X = gen.rhs_normal(rb.n_ext, m, 300 + m)
    for csr in (rb.A_int, rb.A_bnd):
        A = api.RectMatrix(*csr, n_cols=rb.n_ext)
        Y = api.gspmv_rect(A, torch.from_numpy(X).cuda(), torch.empty(A.n, m, dtype=torch.float64, device="cuda"))
        ref = oracle.gspmv_csr(csr, X)
        assert np.all(np.abs(Y.cpu().numpy() - ref) <= 1e-12 * _scale(csr, rb.n_ext, X))
        A.close()


def test_rect_matrix_is_rejected_where_a_square_one_is_needed(ens):
    from paper_1711_10622_gb300 import api

    A = api.RectMatrix(np.array([0, 1, 2], np.int32), np.array([0, 3], np.int32), np.array([1.0, 2.0]), n_cols=5)
    assert (A.n, A.n_cols) == (2, 5)
    B = torch.zeros(2, 1, dtype=torch.float64, device="cuda")
    with pytest.raises(ens.EnsError, match="square"):
        ens.solve_block(A, B, tol=1e-8)
    with pytest.raises(ens.EnsError, match="square"):
        A.amg_setup()
    A.close()


@pytest.mark.parametrize("n,m,npairs", [(0, 4, 1), (1, 1, 1), (1000, 3, 2), (70001, 16, 3), (262144, 64, 4), (5000, 256, 1)])
def test_block_dots_and_lincomb(ens, n, m, npairs):
    from paper_1711_10622_gb300 import api

    rng = np.random.default_rng(n + m)
    Xs = [rng.standard_normal((n, m)) for _ in range(npairs)]
    Ys = [rng.standard_normal((n, m)) for _ in range(npairs)]
    dX, dY = [torch.from_numpy(a).cuda() for a in Xs], [torch.from_numpy(a).cuda() for a in Ys]
    d = api.block_dots(list(zip(dX, dY)), n).cpu().numpy().reshape(npairs, m)
    d2 = api.block_dots(list(zip(dX, dY)), n).cpu().numpy().reshape(npairs, m)
    np.testing.assert_array_equal(d, d2)  # fixed summation order
    for k in range(npairs):
        ref = (Xs[k] * Ys[k]).sum(axis=0)
        bound = 1e-13 * np.abs(Xs[k] * Ys[k]).sum(axis=0) + 1e-300
        assert np.all(np.abs(d[k] - ref) <= bound)
    if n == 0:
        return
    cs = [rng.standard_normal(m) for _ in range(npairs)]
    dc_ = [torch.from_numpy(c).cuda() for c in cs]
    out = torch.empty(n, m, dtype=torch.float64, device="cuda")
    api.block_lincomb([None] + dc_[1:], dX, out, n)
    ref = Xs[0] + sum(cs[k] * Xs[k] for k in range(1, npairs))
    scale = np.abs(Xs[0]) + sum(np.abs(cs[k] * Xs[k]) for k in range(1, npairs))
    assert np.all(np.abs(out.cpu().numpy() - ref) <= 4e-16 * npairs * scale)
    api.block_lincomb(dc_[:1], dX[:1], dX[0], n)  # in place
    np.testing.assert_array_equal(dX[0].cpu().numpy(), cs[0] * Xs[0])
    idx = torch.from_numpy(rng.integers(0, n, size=777).astype(np.int32)).cuda()
    g = api.gather_rows(idx, dY[0], torch.empty(777, m, dtype=torch.float64, device="cuda"))
    np.testing.assert_array_equal(g.cpu().numpy(), Ys[0][idx.cpu().numpy()])


def _case(name):
    if name == "dirichlet":
        op = gen.dirichlet_box(24)
        return op, gen.rhs_uniform(op.n, 4, 81), 1e-9, 24 * 24
    if name == "cubes":
        op = gen.cubes(48, 32, 24, size=4)
        return op, gen.rhs_normal(op.n, 3, 82, zero_mean=True), 1e-9, 48 * 32
    op, B = breakdown_system(patterns=512)
    return op, B, 1e-10, None


@pytest.mark.parametrize("case,size", [("dirichlet", 2), ("cubes", 3), ("breakdown", 2)])
def test_row_split_on_emulated_ranks(ens, case, size):
    from dist_thread_comm import run_ranks

    from paper_1711_10622_gb300 import decomposition as dc

    op, B, tol, plane = _case(case)
    n, m = B.shape
    bounds = dc.slab_bounds(n, size, plane=plane)
    X = gen.rhs_normal(n, m, 91)

    def rank_fn(comm):
        ops = dc.CudaOps()
        rb = dc.row_block(op.row_ptr, op.col_idx, op.val, bounds, comm.rank)
        D = dc.DistMatrix(rb, ops, m)
        Xe = ops.zeros(rb.n_ext, m)
        Xe[: rb.n_loc] = torch.from_numpy(X[rb.glob]).cuda()
        Y = ops.zeros(rb.n_loc, m)
        D.gspmv(comm, Xe, Y)
        res = dc.dist_bicgstab(comm, ops, rb, torch.from_numpy(np.ascontiguousarray(B[rb.glob])).cuda(), tol,
                               singular=op.singular)
        torch.cuda.synchronize()
        return rb.glob, Y.cpu().numpy(), res.X_loc.cpu().numpy(), res.status, res.iters, res.relres

    out = run_ranks(size, rank_fn)
    Y = np.zeros((n, m))
    Xd = np.zeros((n, m))
    for glob, Yr, Xr, *_ in out:
        Y[glob] = Yr
        Xd[glob] = Xr
    S = op.to_scipy().copy()
    S.data = np.abs(S.data)
    assert np.all(np.abs(Y - oracle.gspmv(op, X)) <= 1e-12 * (S @ np.abs(X)))
    st, it, rr = out[0][3], out[0][4], out[0][5]
    Xo, it_o, rr_o, st_o = oracle.solve_block(op, B, tol)
    np.testing.assert_array_equal(st, st_o)
    assert np.all(np.abs(it - it_o) <= 0.25 * it_o + 2), (it, it_o)
    if case == "breakdown":
        np.testing.assert_array_equal(it[:3], it_o[:3])
        np.testing.assert_array_equal(Xd[:, :3], Xo[:, :3])
    for l in np.nonzero(st_o == 0)[0]:
        assert rr[l] <= tol * 1.05
        assert np.linalg.norm(Xd[:, l] - Xo[:, l]) <= 1e-6 * np.linalg.norm(Xo[:, l])


def test_ensemble_split_on_emulated_ranks(ens):
    from dist_thread_comm import run_ranks

    from paper_1711_10622_gb300 import decomposition as dc

    op = gen.cubes(48, 32, 24, size=4)
    B = torch.from_numpy(gen.rhs_normal(op.n, 5, 93, zero_mean=True)).cuda()
    with ens.Matrix.from_operator(op) as A:
        Xfull, st_full = ens.solve_block(A, B, tol=1e-9, precond="chebyshev")

        def rank_fn(comm):
            X, st, share = dc.solve_ensemble_split(
                comm, B, lambda Bs: ens.solve_block(A, Bs.contiguous(), tol=1e-9, precond="chebyshev"))
            torch.cuda.synchronize()
            return X.cpu().numpy(), share

        out = run_ranks(2, rank_fn)
    # every rank holds the whole solution; each column is solved to the tolerance by an independent
    # recurrence (its rounding depends on the block width it ran in), so it matches the one-block
    # solve to the solution-error bar, and the oracle confirms its residual
    Xf = Xfull.cpu().numpy()
    Bh = B.cpu().numpy()
    for X, share in out:
        err = np.linalg.norm(X - Xf, axis=0) / np.linalg.norm(Xf, axis=0)
        assert err.max() <= 1e-6, err
        R = Bh - oracle.gspmv(op, X)
        assert np.all(np.linalg.norm(R, axis=0) <= 1.05e-9 * np.linalg.norm(Bh, axis=0))
    np.testing.assert_array_equal(out[0][0], out[1][0])
