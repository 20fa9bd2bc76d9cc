"""Pins of the oracle's BiCGStab breakdown branches and of the AMG V-cycle's composition.

Breakdown (Section 4.1 names BiCGStab; van der Vorst 1992 as cited in Section 1). The paper does
not say what happens when a step length cannot be formed; the reading used on both sides is: status
BREAKDOWN, no restart, x keeps its last finite iterate. The inputs (gen.breakdown) make every
quantity of the first iteration an exact dyadic number, so the expected results below follow by
hand from the recurrences with x0 = 0, r0 = rhat = b, p1 = r0:
  column 0: (rhat, v) = b^T A b = 0, so alpha cannot be formed: BREAKDOWN after 1 iteration, x = 0
  column 1: alpha = (b, b) / (b, A b) = -1/2, s = b + A b / 2 and (t, s) = s^T A s = 0, so omega = 0:
            x = alpha b = -b / 2 is kept, r = s, BREAKDOWN after 1 iteration
  column 2: alpha = -1, s = b + A b = (-3, 3) per block and t = A s = 0, so (t, t) = 0: BREAKDOWN
            after 1 iteration before x is updated, x = 0
  column 3: an ordinary right-hand side on the invertible region converges to x = A^-1 b (the 2 x 2
            block inverse written out by hand)
A planted mistake in any branch (no omega test, x not kept, x updated before the (t, t) test, ...)
changes a status, an iteration count or an x below.

V-cycle (Section 4.1's AMG, restated as aggregation multigrid): the two-level cycle
z = S r; z += P C P^T (r - A z); z += S (r - A z) is a fixed linear operator. It is built here as a
dense matrix from the closed form of the Chebyshev iteration (after k updates from zero the error
is R_k(D^-1 A) applied to the initial error, R_k(l) = T_k((theta - l) / delta) / T_k(theta / delta),
T_k the Chebyshev polynomial; so S = (I - R_k(D^-1 A)) A^-1) and compared with the oracle's cycle
column by column. A wrong sign or a missing term in the coarse correction fails it.
"""

import numpy as np
import pytest

import gen
import oracle
from gen.breakdown import breakdown_system

BREAKDOWN = oracle.BREAKDOWN


@pytest.fixture(scope="module")
def system():
    return breakdown_system(patterns=256)


def _region1_solution(b1):
    # M1 = [[-2, -2], [-2, 0]], det = -4, M1^-1 = [[0, -1/2], [-1/2, 1/2]]
    u, w = b1[0::2], b1[1::2]
    x = np.empty_like(b1)
    x[0::2] = -0.5 * w
    x[1::2] = -0.5 * u + 0.5 * w
    return x


def test_breakdown_inputs_are_what_the_pins_assume(system):
    op, B = system
    A = op.to_scipy().toarray() if op.n <= 4096 else None
    S = op.to_scipy()
    b0, b1, b2 = B[:, 0], B[:, 1], B[:, 2]
    assert b0 @ (S @ b0) == 0.0
    Ab1 = S @ b1
    assert (b1 @ b1) / (b1 @ Ab1) == -0.5
    s1 = b1 + 0.5 * Ab1
    assert s1 @ (S @ s1) == 0.0 and np.any(S @ s1 != 0)
    Ab2 = S @ b2
    assert (b2 @ b2) / (b2 @ Ab2) == -1.0
    assert np.all(S @ (b2 + Ab2) == 0) and np.any(b2 + Ab2 != 0)
    # the exact solution of column 3 solves the system
    n1 = op.meta["n1"]
    x3 = np.zeros(op.n)
    x3[:n1] = _region1_solution(B[:n1, 3])
    np.testing.assert_array_equal(S @ x3, B[:, 3])
    del A


def test_oracle_breakdown_statuses_iterations_and_iterates(system):
    op, B = system
    tol = 1e-10
    X, it, rr, st = oracle.solve_block(op, B, tol)
    assert list(st) == [BREAKDOWN, BREAKDOWN, BREAKDOWN, oracle.CONVERGED], st
    assert list(it[:3]) == [1, 1, 1], it
    np.testing.assert_array_equal(X[:, 0], 0.0)
    np.testing.assert_array_equal(X[:, 1], -0.5 * B[:, 1])
    np.testing.assert_array_equal(X[:, 2], 0.0)
    # true residuals at exit: x = 0 gives 1; column 1 keeps r = s = b + A b / 2
    S = op.to_scipy()
    s1 = B[:, 1] + 0.5 * (S @ B[:, 1])
    assert rr[0] == 1.0 and rr[2] == 1.0
    assert abs(rr[1] - np.linalg.norm(s1) / np.linalg.norm(B[:, 1])) <= 1e-15
    n1 = op.meta["n1"]
    x3 = np.zeros(op.n)
    x3[:n1] = _region1_solution(B[:n1, 3])
    assert rr[3] <= tol
    assert np.linalg.norm(X[:, 3] - x3) <= 1e-9 * np.linalg.norm(x3)


def test_oracle_breakdown_keeps_a_given_initial_guess(system):
    """With x0 = 0 on the breakdown columns the iterate stays 0; a nonzero x0 whose residual is the
    same b (x0 in the null space of the singular region) is kept exactly by the (t, t) breakdown."""
    op, B = system
    n1 = op.meta["n1"]
    X0 = np.zeros_like(B)
    X0[n1:, 2] = np.tile([1.0, -1.0], op.meta["n2"] // 2)  # M2 (1, -1) = 0
    X, it, rr, st = oracle.solve_block(op, B, 1e-10, X0=X0)
    assert st[2] == BREAKDOWN and it[2] == 1
    np.testing.assert_array_equal(X[:, 2], X0[:, 2])


def _cheb_residual_poly(Bmat, k, lo, hi):
    """R_k(Bmat) = T_k((theta I - Bmat) / delta) / T_k(theta / delta), by the three-term recurrence."""
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    n = Bmat.shape[0]
    Y = (theta * np.eye(n) - Bmat) / delta
    T0, T1 = np.eye(n), Y.copy()
    t0, t1 = 1.0, theta / delta
    if k == 0:
        return T0
    for _ in range(k - 1):
        T0, T1 = T1, 2.0 * Y @ T1 - T0
        t0, t1 = t1, 2.0 * (theta / delta) * t1 - t0
    return T1 / t1


def _cheb_operator(Ad, k, lo, hi):
    D = np.diag(Ad)
    R = _cheb_residual_poly(Ad / D[:, None], k, lo, hi)
    return (np.eye(Ad.shape[0]) - R) @ np.linalg.inv(Ad)


def test_chebyshev_closed_form_matches_the_oracle_iteration():
    """The closed form used below for the smoother agrees with the oracle's Chebyshev iteration."""
    op = gen.dirichlet_box(6)
    Ad = op.to_scipy().toarray()
    lo, hi = oracle.DEFAULT_CHEB_LO, oracle.DEFAULT_CHEB_HI
    for k in (1, 2, 4, 7):
        S = _cheb_operator(Ad, k, lo, hi)
        r = gen.rhs_normal(op.n, 1, 40 + k)[:, 0]
        z = oracle.chebyshev(op, r, lo, hi, k)
        assert np.linalg.norm(z - S @ r) <= 1e-12 * np.linalg.norm(S @ r), k


@pytest.mark.parametrize("smooth,coarse", [(2, 16), (3, 5)])
def test_two_level_vcycle_matches_its_dense_composition(smooth, coarse):
    op = gen.dirichlet_box(8)  # 8^3 = 512 rows, config-1 boundary types
    lo, hi = oracle.DEFAULT_CHEB_LO, oracle.DEFAULT_CHEB_HI
    H = oracle.AMG(op, max_levels=2, coarse_size=64, smooth=smooth, coarse=coarse)
    assert H.nlev == 2
    agg = H.level(0)[3]
    nc = H.sizes[1][0]
    n = op.n
    P = np.zeros((n, nc))
    P[np.arange(n), agg] = 1.0
    Ad = op.to_scipy().toarray()
    Ac = P.T @ Ad @ P
    S = _cheb_operator(Ad, smooth, lo, hi)
    C = _cheb_operator(Ac, coarse, lo, hi)
    I = np.eye(n)
    V1 = S                                  # pre-smoothing
    V2 = V1 + P @ C @ P.T @ (I - Ad @ V1)   # coarse correction
    V = V2 + S @ (I - Ad @ V2)              # post-smoothing
    R = gen.rhs_normal(n, 6, 99)
    Z = H.vcycle(R)
    ref = V @ R
    err = np.linalg.norm(Z - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert err.max() <= 1e-11, err
    # the same check rejects a reversed coarse correction
    bad = (V1 - P @ C @ P.T @ (I - Ad @ V1))
    bad = bad + S @ (I - Ad @ bad)
    assert (np.linalg.norm(Z - bad @ R, axis=0) / np.linalg.norm(ref, axis=0)).min() > 1e-3
    H.close()
