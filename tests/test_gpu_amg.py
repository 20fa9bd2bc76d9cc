"""GPU parity of the aggregation multigrid preconditioner (ens_amg_setup / ens_amg_apply /
ENS_PRECOND_AMG) against the oracle (oracle/amg.c), through the C ABI.

The hierarchy is built on the host by the library's own code and must reproduce the oracle's
aggregates exactly (integer work: bit-exact) and its Galerkin operators (same summation order);
the V-cycle on the GPU must match the oracle's V-cycle column by column; BiCGStab + V-cycle must
converge to the oracle's solution in about the oracle's iteration count.
"""

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

OPS = {
    "dirichlet12": lambda: gen.dirichlet_box(12),
    "channel32x24x16": lambda: gen.channel(32, 24, 16),
    "cubes48x32x24": lambda: gen.cubes(48, 32, 24, size=4),
}
AMG = dict(theta=0.08, max_levels=8, coarse_size=64, smooth_steps=2, coarse_steps=16)


@pytest.fixture(scope="module")
def ens():
    import paper_1711_10622_gb300 as e
    from paper_1711_10622_gb300 import build

    build.build()
    return e


def _oracle_amg(op):
    return oracle.AMG(op, theta=AMG["theta"], max_levels=AMG["max_levels"], coarse_size=AMG["coarse_size"],
                      smooth=AMG["smooth_steps"], coarse=AMG["coarse_steps"])


@pytest.mark.parametrize("name", list(OPS))
def test_hierarchy_matches_oracle(ens, name):
    op = OPS[name]()
    H = _oracle_amg(op)
    with ens.Matrix.from_operator(op) as A:
        info = A.amg_setup(**AMG)
        assert info == H.sizes
        for l in range(H.nlev):
            row, col, val, agg = A.amg_level(l)
            r2, c2, v2, a2 = H.level(l)
            assert np.array_equal(row, r2) and np.array_equal(col, c2)
            assert np.array_equal(val, v2)  # same sums in the same order
            if a2 is not None:
                assert np.array_equal(agg, a2)


@pytest.mark.parametrize("name", list(OPS))
@pytest.mark.parametrize("m", [1, 3, 8])
def test_vcycle_parity(ens, name, m):
    op = OPS[name]()
    H = _oracle_amg(op)
    R = gen.rhs_normal(op.n, m, 40 + m)
    ref = H.vcycle(R)
    with ens.Matrix.from_operator(op) as A:
        A.amg_setup(**AMG)
        Z = ens.amg_apply(A, torch.from_numpy(R).cuda()).cpu().numpy()
        Z32 = ens.amg_apply(A, torch.from_numpy(R.astype(np.float32)).cuda()).cpu().numpy()
    scale = np.abs(ref).max(axis=0)
    assert np.all(np.abs(Z - ref).max(axis=0) <= 1e-11 * scale)
    assert np.all(np.abs(Z32 - ref).max(axis=0) <= 1e-4 * scale)


def test_vcycle_fp32_views(ens):
    """ens_amg_apply on float32 blocks that are 8- but not 16-byte aligned takes two columns per lane
    (16-byte aligned blocks take four): both match the oracle's V-cycle."""
    op = OPS["cubes48x32x24"]()
    H = _oracle_amg(op)
    m = 8
    R = gen.rhs_normal(op.n, m, 45)
    ref = H.vcycle(R.astype(np.float32).astype(np.float64))
    scale = np.abs(ref).max(axis=0)
    with ens.Matrix.from_operator(op) as A:
        A.amg_setup(**AMG)
        buf = torch.zeros(op.n * m + 2, dtype=torch.float32, device="cuda")
        Rv = buf[2:].view(op.n, m)  # 8-byte aligned, not 16
        Rv.copy_(torch.from_numpy(R.astype(np.float32)))
        zbuf = torch.zeros(op.n * m + 2, dtype=torch.float32, device="cuda")
        Zv = zbuf[2:].view(op.n, m)
        ens.amg_apply(A, Rv, Zv)
        Za = ens.amg_apply(A, torch.from_numpy(R.astype(np.float32)).cuda())
    for Z in (Zv.cpu().numpy(), Za.cpu().numpy()):
        assert np.all(np.abs(Z - ref).max(axis=0) <= 1e-4 * scale)


@pytest.mark.parametrize("name", list(OPS))
def test_solve_with_amg_matches_oracle(ens, name):
    op = OPS[name]()
    H = _oracle_amg(op)
    m, tol = 4, 1e-9
    B = gen.rhs_normal(op.n, m, 50, zero_mean=op.singular)
    Xo, it_o, rr_o, st_o = oracle.solve_block(op, B, tol, precond="amg", amg=H)
    with ens.Matrix.from_operator(op) as A:
        A.amg_setup(**AMG)
        for use_graph in (1, 0):
            X, st = ens.solve_block(A, torch.from_numpy(B).cuda(), tol=tol, precond="amg", use_graph=use_graph)
            Xn = X.cpu().numpy()
            assert np.all(st["status"] == 0) and np.all(st["relres"] <= tol * 1.05)
            assert np.all(np.abs(st["iters"] - it_o) <= 0.25 * it_o + 2)
            err = np.linalg.norm(Xn - Xo, axis=0) / np.linalg.norm(Xo, axis=0)
            assert np.all(err <= 1e-6)


def test_amg_needs_fewer_iterations_than_chebyshev(ens):
    op = gen.cubes(96, 64, 48, size=8)
    B = torch.from_numpy(gen.rhs_normal(op.n, 8, 51, zero_mean=True)).cuda()
    with ens.Matrix.from_operator(op) as A:
        A.amg_setup()
        _, sc = ens.solve_block(A, B, tol=1e-8, precond="chebyshev")
        _, sa = ens.solve_block(A, B, tol=1e-8, precond="amg")
    assert np.all(sa["status"] == 0) and np.all(sc["status"] == 0)
    assert np.all(sa["iters"] < sc["iters"])


def test_mixed_precision_with_amg(ens):
    op = gen.channel(48, 32, 24)
    m, tol = 4, 1e-10
    B = gen.rhs_normal(op.n, m, 52, zero_mean=True)
    Xo, _, _, _ = oracle.solve_block(op, B, 1e-12, precond="chebyshev")
    with ens.Matrix.from_operator(op) as A:
        A.amg_setup()
        X, st = ens.solve_block(A, torch.from_numpy(B).cuda(), tol=tol, precond="amg", precision="mixed")
    assert np.all(st["status"] == 0) and np.all(st["relres"] <= tol * 1.05)
    err = np.linalg.norm(X.cpu().numpy() - Xo, axis=0) / np.linalg.norm(Xo, axis=0)
    assert np.all(err <= 1e-6)


def test_batch_with_amg_equals_individual(ens):
    systems = [(gen.cubes(48, 32, 24, size=4), 4, 61), (gen.channel(32, 24, 16), 2, 62)]
    mats, Bs = [], []
    try:
        for op, m, seed in systems:
            A = ens.Matrix.from_operator(op)
            A.amg_setup()
            mats.append(A)
            Bs.append(torch.from_numpy(gen.rhs_normal(op.n, m, seed, zero_mean=op.singular)).cuda())
        res = ens.solve_batch([(A, B, None, 1e-9) for A, B in zip(mats, Bs)], precond="amg")
        for A, B, (Xb, sb) in zip(mats, Bs, res):
            Xs, ss = ens.solve_block(A, B, tol=1e-9, precond="amg")
            assert torch.equal(Xb, Xs)
            assert np.array_equal(sb["iters"], ss["iters"]) and np.all(sb["status"] == 0)
    finally:
        for A in mats:
            A.close()


def test_amg_errors(ens):
    op = gen.dirichlet_box(8)
    with ens.Matrix.from_operator(op) as A:
        B = torch.zeros(op.n, 2, dtype=torch.float64, device="cuda")
        with pytest.raises(ens.EnsError):
            ens.solve_block(A, B, precond="amg")  # no hierarchy yet
        with pytest.raises(ens.EnsError):
            ens.amg_apply(A, B)
        with pytest.raises(ens.EnsError):
            A.amg_setup(theta=1.5)
        assert A.amg_info() == []
        A.amg_setup()
        assert len(A.amg_info()) >= 1


@pytest.mark.parametrize("workload", ["cubes192x128x96_m8", "channel256x128x128"])
def test_full_size_hierarchy_matches_oracle(ens, workload):
    """The hierarchies of the full-size workloads: every level's aggregates and coarse operator
    equal the oracle's (integer maps bit for bit, Galerkin sums in the same order), and one V-cycle
    on sampled columns matches the oracle's on every row."""
    op = gen.WORKLOADS[workload]["op"]()
    H = oracle.AMG(op)
    with ens.Matrix.from_operator(op) as A:
        assert A.amg_setup() == H.sizes
        for l in range(H.nlev):
            row, col, val, agg = A.amg_level(l)
            r2, c2, v2, a2 = H.level(l)
            assert np.array_equal(row, r2) and np.array_equal(col, c2) and np.array_equal(val, v2)
            if a2 is not None:
                assert np.array_equal(agg, a2)
        R = gen.rhs_normal(op.n, 2, 77, zero_mean=op.singular)
        Z = ens.amg_apply(A, torch.from_numpy(R).cuda()).cpu().numpy()
    ref = H.vcycle(R)
    assert np.all(np.abs(Z - ref).max(axis=0) <= 1e-11 * np.abs(ref).max(axis=0))
