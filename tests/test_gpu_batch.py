"""Batched solves (ens_solve_batch): several systems of uneven n and m in one CUDA graph launch.

Each system runs the ens_solve_block algorithm with the same kernels and block width, so its
solution and statistics must equal those of solving it alone, bit for bit; the mixed-precision
batch must also meet the FP64 oracle (residual and solution error).
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


def _systems():
    return [
        (gen.cubes(48, 32, 24, size=4), 4, 11),
        (gen.channel(32, 24, 16), 3, 12),
        (gen.dirichlet_box(12), 8, 13),
        (gen.channel(20, 14, 10), 1, 14),
    ]


@pytest.mark.parametrize("precision,precond", [("f64", "chebyshev"), ("f64", "none"), ("mixed", "chebyshev")])
def test_batch_equals_individual_solves(ens, precision, precond):
    tol = 1e-9
    mats, Bs = [], []
    for op, m, seed in _systems():
        mats.append((op, ens.Matrix.from_operator(op)))
        Bs.append(torch.from_numpy(gen.rhs_normal(op.n, m, seed, zero_mean=op.singular)).cuda())
    try:
        res = ens.solve_batch([(A, B, None, tol) for (op, A), B in zip(mats, Bs)], precond=precond, precision=precision)
        for ((op, A), B), (Xb, sb) in zip(zip(mats, Bs), res):
            Xs, ss = ens.solve_block(A, B, tol=tol, precond=precond, precision=precision)
            assert torch.equal(Xb, Xs)
            for k in ("iters", "status", "outer"):
                assert np.array_equal(sb[k], ss[k]), k
            assert np.array_equal(sb["relres"], ss["relres"])
            assert (sb["status"] == 0).all() and np.all(sb["relres"] <= tol * 1.05)
            Bn, Xn = B.cpu().numpy(), Xb.cpu().numpy()
            R = Bn - oracle.gspmv(op, Xn)
            assert np.all(np.linalg.norm(R, axis=0) <= tol * 1.05 * np.linalg.norm(Bn, axis=0))
    finally:
        for _, A in mats:
            A.close()


def test_mixed_batch_matches_fp64_oracle(ens):
    tol = 1e-10
    systems = _systems()[:3]
    mats = [(op, ens.Matrix.from_operator(op)) for op, m, s in systems]
    Bs = [gen.rhs_normal(op.n, m, s, zero_mean=op.singular) for op, m, s in systems]
    try:
        res = ens.solve_batch([(A, torch.from_numpy(B).cuda(), None, tol) for (op, A), B in zip(mats, Bs)], precond="chebyshev", precision="mixed")
        for (op, A), B, (X, st) in zip(mats, Bs, res):
            assert (st["status"] == 0).all() and np.all(st["relres"] <= 1.05 * tol)
            Xo, it, rr, so = oracle.solve_block(op, B, tol, precond="chebyshev")
            Xg = X.cpu().numpy()
            for l in range(B.shape[1]):
                assert np.linalg.norm(Xg[:, l] - Xo[:, l]) <= 1e-6 * np.linalg.norm(Xo[:, l])
    finally:
        for _, A in mats:
            A.close()


def test_batch_reports_the_bad_item(ens):
    op = gen.dirichlet_box(6)
    with ens.Matrix.from_operator(op) as A:
        B = torch.ones(op.n, 2, dtype=torch.float64, device="cuda")
        with pytest.raises(ens.EnsError, match="item 1"):
            ens.solve_batch([(A, B, None, 1e-8), (A, B, None, [1e-8, -1.0])])


def test_config4_uneven_batch_full_size(ens):
    """The four systems of the batching workload (channel 256 x 192 x 192 m = 16, 64^3 m = 4,
    128^3 m = 8, 96 x 160 x 96 m = 32) in one launch, FP32 inner / FP64 refinement to 1e-10; true
    residuals recomputed by the oracle's SpMV."""
    specs = [((256, 192, 192), 16), ((64, 64, 64), 4), ((128, 128, 128), 8), ((96, 160, 96), 32)]
    mats, Bs = [], []
    for i, (dims, m) in enumerate(specs):
        op = gen.channel(*dims)
        mats.append((op, ens.Matrix.from_operator(op)))
        Bs.append(gen.rhs_normal(op.n, m, 10622 + 40 + i, zero_mean=True))
    try:
        res = ens.solve_batch([(A, torch.from_numpy(B).cuda(), None, 1e-10) for (op, A), B in zip(mats, Bs)], precond="chebyshev", precision="mixed")
        for (op, A), B, (X, st) in zip(mats, Bs, res):
            assert (st["status"] == 0).all(), st
            R = B - oracle.gspmv(op, X.cpu().numpy())
            assert np.all(np.linalg.norm(R, axis=0) <= 1.05e-10 * np.linalg.norm(B, axis=0))
    finally:
        for _, A in mats:
            A.close()
