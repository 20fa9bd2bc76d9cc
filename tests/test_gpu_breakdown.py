"""BiCGStab breakdown through the C ABI (ens_solve_block, ens_solve_batch) against the oracle.

The inputs (gen.breakdown) make the first iteration exact in floating point on both sides, so the
GPU must reproduce the oracle's statuses, iteration counts and iterates exactly:
  column 0  (rhat, v) = 0     -> BREAKDOWN after 1 iteration, x = x0 = 0
  column 1  omega = 0         -> BREAKDOWN after 1 iteration, x = alpha b = -b/2 (kept)
  column 2  (t, t) = 0        -> BREAKDOWN after 1 iteration, x = 0
  column 3  ordinary          -> CONVERGED, solution within 1e-9 of the oracle's
Every FP64 arithmetic mode, the device-driven (graph) and host-driven loops, and the batched launch
are covered. Mixed precision has no oracle of its own: an inner solve that breaks down before its
first update gives d = 0 and the refinement step would repeat it, so the column ends with
BREAKDOWN and x = x0 (columns 0 and 2); column 1's inner solve does update x, and refinement
restarts from the new residual, so only its reported residual is checked there.
"""

import numpy as np
import pytest

import oracle
from gen.breakdown import breakdown_system

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-10


@pytest.fixture(scope="module")
def ens():
    from paper_1711_10622_gb300 import build

    build.build()
    import paper_1711_10622_gb300 as ens

    return ens


@pytest.fixture(scope="module")
def system():
    op, B = breakdown_system(patterns=1024)  # n = 12,288: 48 row tiles
    Xo, it_o, rr_o, st_o = oracle.solve_block(op, B, TOL)
    assert list(st_o) == [2, 2, 2, 0]
    return op, B, (Xo, it_o, rr_o, st_o)


def _true_relres(op, B, X):
    R = B - oracle.gspmv(op, X)
    return np.linalg.norm(R, axis=0) / np.linalg.norm(B, axis=0)


def _check_f64(op, B, X, st, ref):
    Xo, it_o, rr_o, st_o = ref
    np.testing.assert_array_equal(st["status"], st_o)
    np.testing.assert_array_equal(st["iters"][:3], it_o[:3])
    np.testing.assert_array_equal(X[:, :3], Xo[:, :3])
    assert np.all(np.abs(st["relres"][:3] - rr_o[:3]) <= 1e-12 * rr_o[:3])
    assert st["relres"][3] <= TOL * 1.05
    assert np.linalg.norm(X[:, 3] - Xo[:, 3]) <= 1e-9 * np.linalg.norm(Xo[:, 3])
    assert abs(int(st["iters"][3]) - int(it_o[3])) <= 0.25 * it_o[3] + 2


@pytest.mark.parametrize("mode", ["auto", "native", "split", "hybrid"])
@pytest.mark.parametrize("graph", [True, False])
def test_f64_breakdown_matches_oracle(ens, system, mode, graph):
    op, B, ref = system
    with ens.Matrix.from_operator(op) as A:
        A.set_f64_mode(mode)
        X, st = ens.solve_block(A, torch.from_numpy(B).cuda(), tol=TOL, use_graph=int(graph))
        X = X.cpu().numpy()
    _check_f64(op, B, X, st, ref)


@pytest.mark.parametrize("graph", [True, False])
def test_mixed_breakdown_before_first_update(ens, system, graph):
    op, B, ref = system
    Xo = ref[0]
    with ens.Matrix.from_operator(op) as A:
        X, st = ens.solve_block(A, torch.from_numpy(B).cuda(), tol=TOL, precision="mixed", use_graph=int(graph))
        X = X.cpu().numpy()
    assert st["status"][0] == 2 and st["status"][2] == 2, st["status"]
    assert st["iters"][0] == 1 and st["iters"][2] == 1, st["iters"]
    assert st["outer"][0] == 1 and st["outer"][2] == 1, st["outer"]
    np.testing.assert_array_equal(X[:, 0], 0.0)
    np.testing.assert_array_equal(X[:, 2], 0.0)
    assert st["status"][3] == 0 and st["relres"][3] <= TOL * 1.05
    assert np.linalg.norm(X[:, 3] - Xo[:, 3]) <= 1e-9 * np.linalg.norm(Xo[:, 3])
    assert st["status"][1] in (0, 1, 2)
    true = _true_relres(op, B, X)
    assert np.all(np.abs(st["relres"] - true) <= 1e-10 * np.maximum(true, 1e-300) + 1e-14), (st["relres"], true)


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_batch_breakdown_matches_single_solves(ens, system, precision):
    """The batched launch gives each system exactly its single-solve result, breakdowns included."""
    import gen

    op, B, ref = system
    box = gen.dirichlet_box(16)
    B2 = gen.rhs_uniform(box.n, 2, 5)
    with ens.Matrix.from_operator(op) as A, ens.Matrix.from_operator(box) as A2:
        Bd, B2d = torch.from_numpy(B).cuda(), torch.from_numpy(B2).cuda()
        (X, st), (X2, st2) = ens.solve_batch([(A, Bd, None, TOL), (A2, B2d, None, TOL)], precision=precision)
        Xs, sts = ens.solve_block(A, Bd, tol=TOL, precision=precision)
        X, Xs = X.cpu().numpy(), Xs.cpu().numpy()
    np.testing.assert_array_equal(st["status"], sts["status"])
    np.testing.assert_array_equal(st["iters"], sts["iters"])
    np.testing.assert_array_equal(X, Xs)
    if precision == "f64":
        _check_f64(op, B, X, st, ref)
    assert np.all(st2["status"] == 0) and np.all(st2["relres"] <= TOL * 1.05)
