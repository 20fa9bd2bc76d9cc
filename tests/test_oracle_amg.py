"""Pins of the aggregation-multigrid oracle (oracle/amg.c) against what the mathematics fixes.

The hierarchy (plain aggregation, Galerkin coarse operators, Chebyshev-smoothed V-cycle) stands
in for the paper's BiCGStab + AMG solver (Section 4.1). Checked here:
  * aggregates of a 1D chain derived by hand from the three phases;
  * every row lies in exactly one aggregate and every aggregate is connected by strong edges;
  * A_c = P^T A P against a sparse triple product computed independently with scipy;
  * coarse operators stay symmetric, weakly diagonally dominant (so the Chebyshev interval
    [2/30, 2] remains valid on every level) and keep the constants in the null space when A does;
  * the V-cycle is a linear, symmetric operator (pre- and post-smoothing with the same polynomial)
    whose stationary iteration converges on the SPD Poisson operator;
  * BiCGStab + V-cycle solves to the dense LU solution on 8^3 and needs fewer iterations than
    BiCGStab + Chebyshev on the channel and cube operators.
"""

import numpy as np
import pytest
import scipy.sparse as sp

import gen
import oracle


def _chain(n):
    """1D Dirichlet Poisson chain (tridiagonal 2, -1) as a gen.Operator-like object."""
    A = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")
    A.sort_indices()
    return gen.Operator("chain", (n, 1, 1), ("dirichlet",) * 3, A.indptr.astype(np.int32), A.indices.astype(np.int32),
                        A.data.astype(np.float64), False)


def _P(agg, nc):
    return sp.csr_matrix((np.ones(agg.size), (np.arange(agg.size), agg)), shape=(agg.size, nc))


def test_chain_aggregates_by_hand():
    # 9-node chain, every off-diagonal strong. Phase 1: node 0 (neighbour 1 free) -> {0,1}; node 2
    # has aggregated neighbour 1 -> skipped; node 3 -> {2,3,4}; node 5 skipped; node 6 -> {5,6,7};
    # node 8 (neighbour 7 aggregated) skipped. Phase 2: node 8 joins the aggregate of 7.
    H = oracle.AMG(_chain(9), coarse_size=1, max_levels=2)
    _, _, _, agg = H.level(0)
    assert agg.tolist() == [0, 0, 1, 1, 1, 2, 2, 2, 2]
    # coarse operator by hand: (A_c)_II = sum of the aggregate's block (2k - 2(k-1) = 2 for k
    # nodes in a row of the chain), (A_c)_IJ = -1 across each cut edge
    row, col, val, _ = H.level(1)
    Ac = sp.csr_matrix((val, col, row), shape=(3, 3)).toarray()
    assert np.array_equal(Ac, np.array([[2.0, -1.0, 0.0], [-1.0, 2.0, -1.0], [0.0, -1.0, 2.0]]))


def _graph(n, edges, extra_diag):
    """Symmetric M-matrix with -w on each edge (i, j, w) and diagonal = incident weights + extra."""
    A = np.zeros((n, n))
    for i, j, w in edges:
        A[i, j] = A[j, i] = -w
        A[i, i] += w
        A[j, j] += w
    A += np.diag(extra_diag)
    S = sp.csr_matrix(A)
    S.sort_indices()
    return gen.Operator("graph", (n, 1, 1), ("dirichlet",) * 3, S.indptr.astype(np.int32), S.indices.astype(np.int32),
                        S.data.astype(np.float64), False)


@pytest.mark.parametrize("w43,expected", [(2.0, [0, 0, 1, 1, 1, 2]), (1.0, [0, 0, 1, 1, 0, 2])])
def test_phase2_joins_strongest_neighbour(w43, expected):
    # Edges 0-1, 2-3, 1-4 (weight 1), 3-4 (weight w43); node 5 isolated. Phase 1: node 0 -> {0,1},
    # node 2 -> {2,3}; node 4 has aggregated neighbours 1 and 3 -> skipped; node 5 -> {5}. Phase 2:
    # node 4 joins the aggregate of its strongest neighbour (3 when w43 = 2), on a tie the smaller
    # index (1 when w43 = 1).
    op = _graph(6, [(0, 1, 1.0), (2, 3, 1.0), (1, 4, 1.0), (3, 4, w43)], [1.0, 1.0, 1.0, 1.0, 1.0, 1.0])
    H = oracle.AMG(op, coarse_size=1, max_levels=2)
    _, _, _, agg = H.level(0)
    assert agg.tolist() == expected


def _ops():
    return {
        "dirichlet12": gen.dirichlet_box(12),
        "channel32x24x16": gen.channel(32, 24, 16),
        "cubes48x32x24": gen.cubes(48, 32, 24, size=4),
    }


@pytest.mark.parametrize("name", ["dirichlet12", "channel32x24x16", "cubes48x32x24"])
def test_hierarchy_structure(name):
    op = _ops()[name]
    H = oracle.AMG(op, coarse_size=64)
    assert H.nlev >= 3
    for l in range(H.nlev - 1):
        row, col, val, agg = H.level(l)
        A = sp.csr_matrix((val, col, row), shape=(row.size - 1,) * 2)
        nc = H.sizes[l + 1][0]
        # partition: every row in exactly one aggregate, every aggregate used
        assert agg.min() == 0 and agg.max() == nc - 1 and np.unique(agg).size == nc
        # connected aggregates in the strength graph (theta = 0.08)
        d = np.abs(A.diagonal())
        C = A.tocoo()
        strong = (C.row != C.col) & (np.abs(C.data) >= 0.08 * np.sqrt(d[C.row] * d[C.col]))
        S = sp.csr_matrix((np.ones(strong.sum()), (C.row[strong], C.col[strong])), shape=A.shape)
        same = agg[S.tocoo().row] == agg[S.tocoo().col]
        W = sp.csr_matrix((np.ones(same.sum()), (S.tocoo().row[same], S.tocoo().col[same])), shape=A.shape)
        ncomp, lab = sp.csgraph.connected_components(W, directed=False)
        comp_per_agg = np.array([np.unique(lab[agg == I]).size for I in range(nc)])
        assert np.all(comp_per_agg == 1)
        # Galerkin operator against an independent sparse triple product
        r2, c2, v2, _ = H.level(l + 1)
        Ac = sp.csr_matrix((v2, c2, r2), shape=(nc, nc))
        ref = (_P(agg, nc).T @ A @ _P(agg, nc)).tocsr()
        assert abs(Ac - ref).max() <= 1e-13 * abs(A).max()
        # symmetric, weakly diagonally dominant, constants preserved
        assert abs(Ac - Ac.T).max() <= 1e-13 * abs(Ac).max()
        off = np.asarray(abs(Ac).sum(axis=1)).ravel() - np.abs(Ac.diagonal())
        assert np.all(Ac.diagonal() >= off * (1 - 1e-12))
        if op.singular:
            assert np.abs(Ac @ np.ones(nc)).max() <= 1e-12 * abs(Ac).max()


@pytest.mark.parametrize("name", ["dirichlet12", "cubes48x32x24"])
def test_vcycle_linear_and_symmetric(name):
    op = _ops()[name]
    H = oracle.AMG(op, coarse_size=64)
    rng = np.random.default_rng(4)
    r1, r2 = rng.standard_normal((2, op.n))
    z1, z2 = H.vcycle(r1), H.vcycle(r2)
    z12 = H.vcycle(2.0 * r1 - 3.0 * r2)
    assert np.abs(z12 - (2.0 * z1 - 3.0 * z2)).max() <= 1e-12 * np.abs(z12).max()
    assert abs(r2 @ z1 - r1 @ z2) <= 1e-12 * abs(r2 @ z1)


def test_stationary_vcycle_iteration_converges():
    op = gen.dirichlet_box(16)
    H = oracle.AMG(op, coarse_size=64)
    A = op.to_scipy()
    rng = np.random.default_rng(5)
    x_true = rng.standard_normal(op.n)
    b = A @ x_true
    x = np.zeros(op.n)
    errs = []
    for _ in range(12):
        x = x + H.vcycle(b - A @ x)
        errs.append(np.linalg.norm(x - x_true))
    assert errs[-1] <= 0.05 * errs[0]
    assert all(e1 < e0 for e0, e1 in zip(errs, errs[1:]))


def test_amg_bicgstab_matches_lu():
    op = gen.dirichlet_box(8)
    H = oracle.AMG(op, coarse_size=16)
    B = gen.rhs_uniform(op.n, 3, 6)
    X, it, rr, st = oracle.solve_block(op, B, 1e-12, precond="amg", amg=H)
    assert np.all(st == oracle.CONVERGED)
    ref = np.stack([oracle.lu_solve(op.to_scipy().toarray(), B[:, l]) for l in range(3)], axis=1)
    assert np.abs(X - ref).max() <= 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("name", ["channel32x24x16", "cubes48x32x24"])
def test_amg_fewer_iterations_than_chebyshev(name):
    op = _ops()[name]
    H = oracle.AMG(op)
    B = gen.rhs_normal(op.n, 2, 7, zero_mean=op.singular)
    _, it_c, _, st_c = oracle.solve_block(op, B, 1e-8, precond="chebyshev")
    _, it_a, rr, st_a = oracle.solve_block(op, B, 1e-8, precond="amg", amg=H)
    assert np.all(st_a == 0) and np.all(st_c == 0) and np.all(rr <= 1e-8)
    assert np.all(it_a < it_c)
