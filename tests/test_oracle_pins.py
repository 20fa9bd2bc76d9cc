"""Pins of the CPU oracle against what the mathematics and the paper fix (no GPU).

Each test checks the oracle against something other than itself: closed-form eigenpairs of the
7-point operator, dense library products on tiny grids, a library dense solve, Krylov
termination on right-hand sides with k eigencomponents, the scalar Chebyshev polynomial on
Fourier modes, and the values the paper prints for its performance model.
"""

import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

import gen
import oracle
from gen.operators import DIRICHLET, NEUMANN, PERIODIC, fv_poisson, uniform_nodes, tanh_nodes
from oracle import estimates as est

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_estimates.json")


# ----------------------------------------------------------------------------- eigenpairs
def _mode_1d(bc, N, q):
    """1D eigenvector of the cell-centred second difference and its angle."""
    i = np.arange(N) + 0.5
    if bc == DIRICHLET:  # p = q+1 in 1..N
        th = (q + 1) * np.pi / N
        return np.sin(th * i), th
    if bc == NEUMANN:  # q in 0..N-1
        th = q * np.pi / N
        return np.cos(th * i), th
    th = 2 * np.pi * q / N  # periodic
    return np.cos(th * np.arange(N)), th


def _eig_case(bcs, dims, spacing, modes):
    hx, hy, hz = spacing
    nx, ny, nz = dims
    A = fv_poisson(uniform_nodes(nx, nx * hx), uniform_nodes(ny, ny * hy), uniform_nodes(nz, nz * hz), bcs=bcs)
    w = (hy * hz / hx, hx * hz / hy, hx * hy / hz)  # face weight area/dist per direction
    out = []
    for qx, qy, qz in modes:
        vx, tx = _mode_1d(bcs[0], nx, qx)
        vy, ty = _mode_1d(bcs[1], ny, qy)
        vz, tz = _mode_1d(bcs[2], nz, qz)
        v = (vz[:, None, None] * vy[None, :, None] * vx[None, None, :]).reshape(-1)
        lam = w[0] * (2 - 2 * np.cos(tx)) + w[1] * (2 - 2 * np.cos(ty)) + w[2] * (2 - 2 * np.cos(tz))
        out.append((v, lam))
    return A, out


@pytest.mark.parametrize(
    "bcs,dims,spacing",
    [
        ((DIRICHLET, NEUMANN, DIRICHLET), (7, 6, 5), (0.3, 0.5, 0.7)),
        ((PERIODIC, NEUMANN, PERIODIC), (8, 5, 6), (0.25, 1.0, 0.5)),
        ((NEUMANN, DIRICHLET, PERIODIC), (5, 7, 9), (1.0, 0.2, 0.4)),
    ],
)
def test_spmv_closed_form_eigenpairs(bcs, dims, spacing):
    modes = [(0, 0, 0), (1, 2, 3), (2, 1, 0), (3, 4, 1), (4, 0, 2)]
    A, pairs = _eig_case(bcs, dims, spacing, modes)
    for v, lam in pairs:
        y = oracle.spmv(A, v)
        scale = max(lam, 1e-300) * np.abs(v).max()
        lam_max = 12 * max(spacing) ** 2 / min(spacing)
        assert np.abs(y - lam * v).max() <= 1e-13 * max(scale, lam_max * np.abs(v).max())


def test_gspmv_layout_against_dense_product():
    # Stretched, periodic, with a removed cell: exercises variable coefficients and wrap-around.
    solid = np.zeros((4, 5, 6), dtype=bool)
    solid[1, 0, 2] = True
    A = fv_poisson(uniform_nodes(6, 2.0), tanh_nodes(5, 2.0), uniform_nodes(4, 1.0), solid=solid)
    rng = np.random.default_rng(0)
    for m in (1, 2, 3, 5, 8):
        X = rng.standard_normal((A.n, m))
        Y = oracle.gspmv(A, X)
        Yd = A.to_scipy().toarray() @ X  # library dense product
        assert Y.shape == (A.n, m)
        np.testing.assert_allclose(Y, Yd, rtol=0, atol=1e-13 * np.abs(Yd).max())
        # column l of the block equals a single SpMV of column l
        for l in range(m):
            np.testing.assert_array_equal(Y[:, l], oracle.spmv(A, X[:, l].copy()))


def test_relerr_metric_detects_errors():
    A = gen.dirichlet_box(4)
    X = np.random.default_rng(1).standard_normal((A.n, 3))
    Y = oracle.gspmv(A, X)
    assert oracle.relerr_rows(Y, Y, A, X) == 0.0
    Yb = Y.copy()
    Yb[5, 1] += 1e-6
    assert oracle.relerr_rows(Yb, Y, A, X) > 1e-8


# ----------------------------------------------------------------------------- operators
def test_operator_symmetry_and_null_space():
    A = gen.channel(8, 12, 6)
    S = A.to_scipy()
    assert abs(S - S.T).max() == 0.0
    rowsum = S @ np.ones(A.n)
    assert np.abs(rowsum).max() <= 1e-14 * np.abs(A.val).max()
    assert A.singular
    B = gen.dirichlet_box(6)
    assert not B.singular
    assert (B.to_scipy() @ np.ones(B.n)).min() >= -1e-14 * np.abs(B.val).max()


def test_config1_sizes_closed_form():
    A = gen.dirichlet_box(32)
    N = 32
    # row length 7 minus the number of boundary faces of the cell
    hist = {4: 8, 5: 12 * (N - 2), 6: 6 * (N - 2) ** 2, 7: (N - 2) ** 3}
    assert A.n == N**3
    assert A.row_length_histogram() == hist
    assert A.nnz == sum(k * v for k, v in hist.items())


def test_cubes_sizes_closed_form():
    A = gen.cubes()
    n_expected = 192 * 128 * 96 - 16 * 16**3
    assert A.n == n_expected
    # blocked faces: bottom wall outside the cube footprints, top wall, 5 exposed faces per cube
    one_face = (192 * 96 - 16 * 256) + 192 * 96 + 16 * 5 * 256
    two_faces = 16 * 4 * 16  # bottom-wall cells beside a cube side
    hist = A.row_length_histogram()
    assert hist[5] == two_faces
    assert hist[6] == one_face - 2 * two_faces
    assert hist[7] == n_expected - hist[5] - hist[6]
    assert A.singular


# ----------------------------------------------------------------------------- LU
def test_lu_matches_library_solve():
    rng = np.random.default_rng(2)
    M = rng.standard_normal((60, 60)) + 5 * np.eye(60)
    b = rng.standard_normal(60)
    x = oracle.lu_solve(M, b)
    xr = np.linalg.solve(M, b)
    np.testing.assert_allclose(x, xr, rtol=1e-12, atol=1e-12)
    # pivoting is needed: zero leading entry
    P = np.array([[0.0, 1.0], [2.0, 3.0]])
    np.testing.assert_allclose(oracle.lu_solve(P, np.array([1.0, 5.0])), [1.0, 1.0], rtol=1e-15)


# ----------------------------------------------------------------------------- Chebyshev
def _cheb_closed(mu, lo, hi, steps):
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    Ts = npcheb.Chebyshev.basis(steps)
    return (1.0 - Ts((theta - mu) / delta) / Ts(theta / delta)) / mu


@pytest.mark.parametrize("steps", [1, 2, 4, 6])
def test_chebyshev_scalar_polynomial_on_fourier_modes(steps):
    N = 8
    A = fv_poisson(uniform_nodes(N, N), uniform_nodes(N, N), uniform_nodes(N, N), bcs=(PERIODIC,) * 3)
    d = 6.0  # constant diagonal of the periodic unit-spacing operator
    lo, hi = oracle.DEFAULT_CHEB_LO, oracle.DEFAULT_CHEB_HI
    i = np.arange(N)
    for kx, ky, kz in [(1, 0, 0), (1, 2, 3), (4, 4, 4), (2, 3, 0), (0, 0, 1)]:
        v = (
            np.cos(2 * np.pi * kz * i / N)[:, None, None]
            * np.cos(2 * np.pi * ky * i / N)[None, :, None]
            * np.cos(2 * np.pi * kx * i / N)[None, None, :]
        ).reshape(-1)
        lam = sum(2 - 2 * np.cos(2 * np.pi * k / N) for k in (kx, ky, kz))
        mu = lam / d
        z = oracle.chebyshev(A, v, lo, hi, steps)
        expect = _cheb_closed(mu, lo, hi, steps) / d * v
        np.testing.assert_allclose(z, expect, rtol=0, atol=1e-13 * np.abs(expect).max())


def test_chebyshev_is_linear():
    A = gen.cubes(24, 20, 24, size=4)
    rng = np.random.default_rng(3)
    r1, r2 = rng.standard_normal(A.n), rng.standard_normal(A.n)
    z = oracle.chebyshev(A, 2.0 * r1 - 0.5 * r2)
    z12 = 2.0 * oracle.chebyshev(A, r1) - 0.5 * oracle.chebyshev(A, r2)
    np.testing.assert_allclose(z, z12, rtol=0, atol=1e-13 * np.abs(z).max())


# ----------------------------------------------------------------------------- BiCGStab
def test_bicgstab_matches_dense_solve_8cubed():
    A = gen.dirichlet_box(8)
    B = gen.rhs_uniform(A.n, 3, 99)
    X, iters, relres, status = oracle.solve_block(A, B, 1e-10)
    assert (status == oracle.CONVERGED).all()
    assert (relres <= 1e-10 * 1.01).all()
    Ad = A.to_scipy().toarray()
    for l in range(3):
        xl = np.linalg.solve(Ad, B[:, l])
        xo = oracle.lu_solve(Ad, B[:, l])
        assert np.linalg.norm(X[:, l] - xl) <= 1e-8 * np.linalg.norm(xl)
        assert np.linalg.norm(xo - xl) <= 1e-12 * np.linalg.norm(xl)


@pytest.mark.parametrize("N", [2, 3])
def test_bicgstab_tiny_brute_force_inverse(N):
    A = gen.dirichlet_box(N)
    B = gen.rhs_uniform(A.n, 2, 5)
    X, iters, relres, status = oracle.solve_block(A, B, 1e-13)
    Xinv = np.linalg.inv(A.to_scipy().toarray()) @ B
    np.testing.assert_allclose(X, Xinv, rtol=0, atol=1e-11 * np.abs(Xinv).max())


def test_bicgstab_terminates_in_k_steps_on_k_modes():
    # With rhat = r0 on a symmetric matrix, BiCG is CG; BiCGStab's residual carries the BiCG
    # polynomial, so a right-hand side with k eigencomponents (distinct eigenvalues) is solved
    # after at most k iterations.
    bcs = (DIRICHLET, NEUMANN, DIRICHLET)
    dims = (7, 6, 5)
    A, pairs = _eig_case(bcs, dims, (1.0, 1.0, 1.0), [(0, 0, 0), (1, 2, 3), (3, 4, 1), (2, 1, 0)])
    vs = [p[0] for p in pairs]
    lams = [p[1] for p in pairs]
    assert len(set(np.round(lams, 12))) == 4
    # one mode: x = v / lambda after one iteration
    X, iters, relres, status = oracle.solve_block(A, vs[1], 1e-12)
    assert iters[0] == 1 and status[0] == oracle.CONVERGED
    np.testing.assert_allclose(X[:, 0], vs[1] / lams[1], rtol=0, atol=1e-13 * np.abs(vs[1]).max() / lams[1])
    for k in (2, 3, 4):
        b = sum(vs[:k])
        X, iters, relres, status = oracle.solve_block(A, b, 1e-11)
        assert status[0] == oracle.CONVERGED
        assert iters[0] <= k
        xs = sum(v / lam for v, lam in zip(vs[:k], lams[:k]))
        assert np.linalg.norm(X[:, 0] - xs) <= 1e-9 * np.linalg.norm(xs)


@pytest.mark.parametrize("precond", ["none", "chebyshev"])
def test_bicgstab_manufactured_singular_channel(precond):
    A = gen.channel(16, 12, 8)
    rng = np.random.default_rng(7)
    xs = rng.standard_normal((A.n, 2))
    xs -= xs.mean(axis=0)
    B = oracle.gspmv(A, xs)
    X, iters, relres, status = oracle.solve_block(A, B, 1e-11, precond=precond)
    assert (status == oracle.CONVERGED).all()
    np.testing.assert_allclose(X.sum(axis=0), 0.0, atol=1e-10 * np.abs(X).max() * A.n)
    for l in range(2):
        assert np.linalg.norm(X[:, l] - xs[:, l]) <= 1e-6 * np.linalg.norm(xs[:, l])


def test_chebyshev_reduces_iterations_same_solution():
    A = gen.cubes(48, 32, 24, size=4)
    B = gen.rhs_normal(A.n, 2, 11, zero_mean=True)
    X0, it0, rr0, st0 = oracle.solve_block(A, B, 1e-9)
    X1, it1, rr1, st1 = oracle.solve_block(A, B, 1e-9, precond="chebyshev")
    assert (st0 == 0).all() and (st1 == 0).all()
    assert (it1 < it0).all()
    for l in range(2):
        assert np.linalg.norm(X1[:, l] - X0[:, l]) <= 1e-6 * np.linalg.norm(X0[:, l])


def test_bicgstab_statuses():
    A = gen.channel(8, 6, 6)
    n = A.n
    # zero right-hand side: x = 0, converged in 0 iterations
    X, it, rr, st = oracle.solve_block(A, np.zeros((n, 1)), 1e-8, X0=np.ones((n, 1)))
    assert st[0] == oracle.CONVERGED and it[0] == 0 and (X == 0).all()
    # incompatible right-hand side for a singular operator
    b = np.ones((n, 1))
    X, it, rr, st = oracle.solve_block(A, b, 1e-8)
    assert st[0] == oracle.INCOMPATIBLE
    # non-finite right-hand side
    b = gen.rhs_normal(n, 1, 1, zero_mean=True)
    b[3, 0] = np.nan
    X, it, rr, st = oracle.solve_block(A, b, 1e-8)
    assert st[0] == oracle.NONFINITE
    # iteration cap
    b = gen.rhs_normal(n, 1, 1, zero_mean=True)
    X, it, rr, st = oracle.solve_block(A, b, 1e-14, max_iter=2)
    assert st[0] == oracle.MAXITER and it[0] == 2


def test_true_residual_reported():
    A = gen.dirichlet_box(6)
    B = gen.rhs_uniform(A.n, 2, 4)
    X, it, rr, st = oracle.solve_block(A, B, 1e-9)
    R = B - A.to_scipy() @ X
    np.testing.assert_allclose(rr, np.linalg.norm(R, axis=0) / np.linalg.norm(B, axis=0), rtol=1e-10)


# ----------------------------------------------------------------------------- Section 2.3 model
def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def test_traffic_formula_matches_gain_formula():
    for C in (4.0, 6.98, 7.0, 20.0):
        n = 1000
        nnz = C * n
        for m in (1, 2, 4, 8, 16, 32):
            g = m * est.traffic_bytes(n, nnz, 1) / est.traffic_bytes(n, nnz, m)
            assert math.isclose(g, est.gain_full(m, C), rel_tol=1e-14)
        assert math.isclose(est.gain_full(16, 1e12), est.gain_compact(16), rel_tol=1e-9)


@pytest.mark.parametrize("table", ["table4_estimate", "table5_estimate"])
def test_printed_step_estimates(table):
    g = _golden()[table]
    for m, v in zip(g["m"], g["value"]):
        got = est.step_speedup(g["theta"], est.gain_compact(m))
        assert abs(got - v) <= 0.005 + 1e-12, (m, got, v)


def test_printed_optimal_ensembles():
    g = _golden()["optimal_m_theta085"]
    for beta, best in zip(g["beta"], g["best_m"]):
        vals = {m: est.overall_speedup_closed(m, beta, g["theta"]) for m in g["m_candidates"]}
        assert max(vals, key=vals.get) == best


def test_printed_speedup_range():
    g = _golden()["speedup_range_theta085"]
    for beta, m, pct in zip(g["beta"], g["best_m"], g["percent"]):
        p = est.overall_speedup_closed(m, beta, g["theta"])
        assert abs(100 * (p - 1) - pct) <= 0.5


def test_printed_channel_fullscale_estimate():
    g = _golden()["channel_fullscale"]
    p = est.overall_speedup(g["m"], g["beta"], g["step_gain"])
    assert abs(p - g["expected"]) <= 0.005


def test_optimal_m_is_the_maximiser():
    from scipy.optimize import minimize_scalar

    for beta in (2.0, 5.0, 20.0, 40.0):
        for theta in (0.75, 0.85, 0.95):
            res = minimize_scalar(lambda m: -est.overall_speedup_closed(m, beta, theta), bounds=(1.0, 100.0), method="bounded", options={"xatol": 1e-10})
            assert abs(res.x - est.optimal_m(beta, theta)) <= 1e-4 * res.x
    # est3 is est2 with est2_1 and the compact gain substituted
    for m in (1, 2, 4, 8):
        a = est.overall_speedup(m, 7.0, est.step_speedup(0.85, est.gain_compact(m)))
        assert math.isclose(a, est.overall_speedup_closed(m, 7.0, 0.85), rel_tol=1e-14)
