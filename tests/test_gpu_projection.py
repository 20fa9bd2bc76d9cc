"""GPU parity of the projection step (Section 2.2, Eqs. eq2/eq3) against the oracle.

ens_divergence and ens_grad_correct run through the C ABI on seeded predictor fields (the
channel initial condition of Section 4.3.1 plus perturbations) and are compared element by element
with oracle.divergence / oracle.grad_correct. A full projection (divergence -> multi-RHS solve ->
correction) must leave a divergence equal to -tau times the solver's residual, face by face
consistent with the oracle.
"""

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GRIDS = {
    "dirichlet10x8x6": lambda: gen.dirichlet_box(10, nz=6, ny=8),
    "channel20x14x10": lambda: gen.channel(20, 14, 10),
    "cubes48x24x32": lambda: gen.cubes(48, 24, 32, size=4),
}


@pytest.fixture(scope="module")
def ens():
    import paper_1711_10622_gb300 as e
    from paper_1711_10622_gb300 import build

    build.build()
    return e


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _max_area(g):
    w = [np.diff(a) for a in g.nodes]
    return max(w[0].max() * w[1].max(), w[0].max() * w[2].max(), w[1].max() * w[2].max())


def _walls(g):
    from gen.fields import _wall_faces

    return [_wall_faces(g, d).reshape(-1) for d in range(3)]


@pytest.mark.parametrize("name", list(GRIDS))
@pytest.mark.parametrize("m", [1, 2, 3, 8])
def test_divergence_parity(ens, name, m):
    op = GRIDS[name]()
    g = gen.grid_of(op)
    U, V, W = gen.predictor_velocity(g, m, 100 + m, noise=0.3)
    with ens.Grid.from_grid(g) as G:
        assert G.n == op.n and G.nfaces == tuple(g.nfaces(d) for d in range(3))
        D = ens.divergence(G, _dev(U), _dev(V), _dev(W), scale=-2.5).cpu().numpy()
    ref = oracle.divergence(g, U, V, W, scale=-2.5)
    bound = 2.5 * 6 * _max_area(g) * max(np.abs(c).max() for c in (U, V, W))
    assert np.all(np.abs(D - ref) <= 1e-14 * bound)


@pytest.mark.parametrize("name", list(GRIDS))
def test_divergence_ignores_wall_faces(ens, name):
    op = GRIDS[name]()
    g = gen.grid_of(op)
    U, V, W = gen.predictor_velocity(g, 2, 55)
    ref = oracle.divergence(g, U, V, W)
    for c, wall in zip((U, V, W), _walls(g)):
        c[wall] = 1e6  # garbage on walls: no flux passes a wall
    with ens.Grid.from_grid(g) as G:
        D = ens.divergence(G, _dev(U), _dev(V), _dev(W)).cpu().numpy()
    assert np.allclose(D, ref, rtol=0, atol=1e-13 * 6 * _max_area(g) * 3)


@pytest.mark.parametrize("name", list(GRIDS))
@pytest.mark.parametrize("m", [1, 2, 5, 8])
def test_grad_correct_parity(ens, name, m):
    op = GRIDS[name]()
    g = gen.grid_of(op)
    U, V, W = gen.predictor_velocity(g, m, 200 + m, noise=0.3)
    P = np.random.default_rng(7 + m).standard_normal((op.n, m))
    tau = 0.013
    for c, wall in zip((U, V, W), _walls(g)):
        c[wall] = 7.0  # walls are never written: the sentinel must survive
    with ens.Grid.from_grid(g) as G:
        Ud, Vd, Wd = _dev(U), _dev(V), _dev(W)
        ens.grad_correct(G, _dev(P), Ud, Vd, Wd, tau)
        got = [t.cpu().numpy() for t in (Ud, Vd, Wd)]
    ref = oracle.grad_correct(g, P, U, V, W, tau)
    corr = oracle.grad_correct(g, P, *(np.zeros_like(c) for c in (U, V, W)), tau)  # -tau G p alone
    for d, (c, wall) in enumerate(zip((U, V, W), _walls(g))):
        scale = np.abs(ref[d]) + np.abs(c) + np.abs(corr[d])
        assert np.all(np.abs(got[d] - ref[d]) <= 1e-14 * scale), d
        assert np.all(got[d][wall] == 7.0)


@pytest.mark.parametrize("name", ["channel20x14x10", "cubes48x24x32", "dirichlet10x8x6"])
def test_projection_leaves_residual_divergence(ens, name):
    """div u~ = -tau * (b - A p): the divergence after the correction is the solver's residual."""
    op = GRIDS[name]()
    g = gen.grid_of(op)
    m, tau = 4, 0.05
    U, V, W = gen.predictor_velocity(g, m, 300, noise=0.5)
    with ens.Grid.from_grid(g) as G, ens.Matrix.from_operator(op) as A:
        Ud, Vd, Wd = _dev(U), _dev(V), _dev(W)
        B = ens.divergence(G, Ud, Vd, Wd, scale=-1.0 / tau)
        P, st = ens.solve_block(A, B, tol=1e-11, precond="chebyshev")
        assert np.all(st["status"] == 0)
        R = B - ens.gspmv(A, P)
        ens.grad_correct(G, P, Ud, Vd, Wd, tau)
        Dn = ens.divergence(G, Ud, Vd, Wd).cpu().numpy()
        Rn = R.cpu().numpy()
        Pn = P.cpu().numpy()
    assert np.all(np.abs(Dn + tau * Rn) <= 1e-9 * np.abs(tau * B.cpu().numpy()).max())
    d_star = oracle.divergence(g, U, V, W)
    # |D u~| = tau |r| <= tau * tol * ||B||_2 = tol * ||D u*||_2 per column (tol 1e-11, 2x slack)
    assert np.all(np.abs(Dn).max(axis=0) <= 2e-11 * np.linalg.norm(d_star, axis=0))
    # the corrected field is the oracle's correction with the GPU pressure
    ref = oracle.grad_correct(g, Pn, U, V, W, tau)
    for d, t in enumerate((Ud, Vd, Wd)):
        assert np.allclose(t.cpu().numpy(), ref[d], rtol=0, atol=1e-12 * np.abs(ref[d]).max())


def test_full_size_channel(ens):
    """The 256 x 128 x 128 channel at m = 8: whole-array parity with the oracle."""
    op = gen.channel(256, 128, 128)
    g = gen.grid_of(op)
    m = 8
    U, V, W = gen.predictor_velocity(g, m, 400, noise=0.1)
    P = np.random.default_rng(9).standard_normal((op.n, m))
    with ens.Grid.from_grid(g) as G:
        Ud, Vd, Wd = _dev(U), _dev(V), _dev(W)
        D = ens.divergence(G, Ud, Vd, Wd, scale=1.0).cpu().numpy()
        ens.grad_correct(G, _dev(P), Ud, Vd, Wd, 0.01)
        got = [t.cpu().numpy() for t in (Ud, Vd, Wd)]
    ref = oracle.divergence(g, U, V, W)
    big = max(np.abs(c).max() for c in (U, V, W)) * 8.0  # |area| <= 0.2 here, 6 faces
    assert np.abs(D - ref).max() <= 1e-13 * big
    refc = oracle.grad_correct(g, P, U, V, W, 0.01)
    for d in range(3):
        assert np.abs(got[d] - refc[d]).max() <= 1e-13 * (np.abs(refc[d]).max() + 1.0)


def test_invalid_arguments(ens):
    op = gen.channel(8, 6, 4)
    g = gen.grid_of(op)
    with pytest.raises(ens.EnsError):
        ens.Grid((8, 6, 2), g.nodes[:2] + (np.linspace(0, 1, 3),), ("periodic", "neumann", "periodic"))  # periodic < 3
    bad = (g.nodes[0][::-1].copy(), g.nodes[1], g.nodes[2])
    with pytest.raises(ens.EnsError):
        ens.Grid(g.shape, bad, g.bcs)
    with pytest.raises(ens.EnsError):
        ens.Grid(g.shape, g.nodes, g.bcs, solid=np.ones((4, 6, 8), dtype=bool))
    with ens.Grid.from_grid(g) as G:
        U = torch.zeros(G.nfaces[0], 2, dtype=torch.float64, device="cuda")
        V = torch.zeros(G.nfaces[1], 2, dtype=torch.float64, device="cuda")
        W = torch.zeros(G.nfaces[2], 2, dtype=torch.float64, device="cuda")
        with pytest.raises(ValueError):
            ens.divergence(G, U, V, W[:-1])
        with pytest.raises(ens.EnsError):
            ens.divergence(G, U, V, W, D=torch.zeros(G.n, 2, dtype=torch.float64, device="cuda").copy_(U[: G.n]), scale=float("nan"))


@pytest.mark.parametrize("m", [2, 8])
def test_divergence_split_fallback_states(ens, m):
    """Face values the split-float products cannot carry (exact zeros, 1e30, 1e-300) send their
    states to native DFMA; every state still matches the oracle."""
    op = GRIDS["cubes48x24x32"]()
    g = gen.grid_of(op)
    U, V, W = gen.predictor_velocity(g, m, 300 + m, noise=0.3)
    rng = np.random.default_rng(5)
    for c in (U, V, W):
        idx = rng.integers(0, c.shape[0], size=max(1, c.shape[0] // 50))
        c[idx, rng.integers(0, m, size=idx.shape[0])] = 0.0
    U[7, 0] = 1e30
    V[11, m - 1] = 1e-300
    with ens.Grid.from_grid(g) as G:
        D = ens.divergence(G, _dev(U), _dev(V), _dev(W), scale=-1.5).cpu().numpy()
    ref = oracle.divergence(g, U, V, W, scale=-1.5)
    # per-state bound: the largest face term of that state's cells
    big = np.abs(ref).max(axis=0) + 1.5 * 6 * _max_area(g) * np.array([max(np.abs(c[:, l]).max() for c in (U, V, W)) for l in range(m)])
    assert np.all(np.abs(D - ref) <= 1e-14 * big)
