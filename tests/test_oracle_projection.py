"""Pins of the projection-step oracle (Section 2.2, Eqs. eq2/eq3) against what the mathematics fixes.

oracle.divergence and oracle.grad_correct restate the staggered-grid divergence and pressure
gradient. They are checked here against facts that do not come from the oracle itself:
  * D G = -A for the independently assembled finite-volume operator (whose eigenpairs are pinned in
    test_oracle_pins.py), on uniform, stretched, Dirichlet and solid-cube grids;
  * the discrete divergence of a linear field equals the cell volume times its slope (Gauss);
  * the gradient of a linear pressure is its slope on uniform interior faces;
  * the channel initial condition of Section 4.3.1 is exactly divergence-free;
  * fluxes telescope: sum over cells of D u = 0 with walls and periodic directions;
  * after a projection with an exact (dense LU) pressure solve, D u~ = 0, and projecting twice
    changes nothing (the projection is idempotent).
"""

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _grids():
    return {
        "dirichlet6x5x4": gen.dirichlet_box(6, nz=4, ny=5),
        "channel12x10x8": gen.channel(12, 10, 8),
        "cubes24x12x16": gen.cubes(24, 12, 16, size=3),
    }


def _zeros(g, m):
    return [np.zeros((g.nfaces(d), m)) for d in range(3)]


@pytest.mark.parametrize("name", ["dirichlet6x5x4", "channel12x10x8", "cubes24x12x16"])
def test_div_grad_is_minus_operator(name):
    op = _grids()[name]
    g = gen.grid_of(op)
    p = np.random.default_rng(3).standard_normal((op.n, 3))
    G = oracle.grad_correct(g, p, *_zeros(g, 3), tau=-1.0)  # u = 0 - (-1) G p = G p
    D = oracle.divergence(g, *G)
    Ap = op.to_scipy() @ p
    assert np.max(np.abs(D + Ap)) <= 1e-13 * np.max(np.abs(op.to_scipy()) @ np.abs(p))


def test_divergence_of_linear_field_is_volume():
    # Dirichlet x: every x face is open, so u_f = x_f is linear across the whole grid.
    op = gen.dirichlet_box(5, nz=3, ny=4)
    g = gen.grid_of(op)
    xn, yn, zn = g.nodes
    U = np.zeros((g.nfaces(0), 1))
    Fx = g.face_counts()[0]
    U[:, 0] = np.tile(xn[:Fx], g.nfaces(0) // Fx) * 2.5  # slope 2.5
    D = oracle.divergence(g, U, *_zeros(g, 1)[1:])
    vol = np.einsum("k,j,i->kji", np.diff(zn), np.diff(yn), np.diff(xn)).reshape(-1)
    assert np.allclose(D[:, 0], 2.5 * vol, rtol=1e-14, atol=0)


def test_gradient_of_linear_pressure():
    op = gen.dirichlet_box(6, nz=4, ny=5)
    g = gen.grid_of(op)
    nx, ny, nz = g.shape
    xn, yn, zn = g.nodes
    xc = 0.5 * (xn[:-1] + xn[1:])
    yc = 0.5 * (yn[:-1] + yn[1:])
    p = (3.0 * xc[None, None, :] - 2.0 * yc[None, :, None] + 0 * zn[:nz, None, None]).reshape(-1, 1)
    U, V, W = oracle.grad_correct(g, p, *_zeros(g, 1), tau=-1.0)
    U = U.reshape(nz, ny, nx + 1)
    V = V.reshape(nz, ny + 1, nx)
    assert np.allclose(U[:, :, 1:nx], 3.0, rtol=1e-13)  # interior x faces
    assert np.allclose(V[:, 1:ny, :], -2.0, rtol=1e-13)  # interior y faces
    assert np.all(V[:, 0, :] == 0) and np.all(V[:, ny, :] == 0)  # Neumann walls untouched
    # Dirichlet boundary faces: p = 0 on the face, half a cell from the first centre
    h = xn[1] - xn[0]
    assert np.allclose(U[:, :, 0], (p.reshape(nz, ny, nx)[:, :, 0] - 0.0) / (h / 2), rtol=1e-13)


def test_initial_condition_is_divergence_free():
    op = gen.channel(16, 12, 10)
    g = gen.grid_of(op)
    U, V, W = gen.predictor_velocity(g, 4, 7, noise=0.0)
    assert np.any(U != 0) and np.any(W != 0)
    assert np.all(oracle.divergence(g, U, V, W) == 0.0)


@pytest.mark.parametrize("name", ["channel12x10x8", "cubes24x12x16"])
def test_fluxes_telescope(name):
    op = _grids()[name]
    g = gen.grid_of(op)
    U, V, W = gen.predictor_velocity(g, 3, 11)
    D = oracle.divergence(g, U, V, W)
    scale = sum(np.abs(c).sum(axis=0) for c in (U, V, W))
    assert np.all(np.abs(D.sum(axis=0)) <= 1e-13 * scale)


@pytest.mark.parametrize("name", ["dirichlet6x5x4", "channel12x10x8"])
def test_projection_with_exact_solve(name):
    op = _grids()[name]
    g = gen.grid_of(op)
    tau = 0.37
    U, V, W = gen.predictor_velocity(g, 2, 5, noise=0.2)
    b = oracle.divergence(g, U, V, W, scale=-1.0 / tau)  # A p = -(1/tau) D u*
    Ad = op.to_scipy().toarray()
    if op.singular:  # fix the constant: replace one equation by p_0 = 0 (b sums to zero)
        Ad[0, :] = 0.0
        Ad[0, 0] = 1.0
        b = b.copy()
        b[0] = 0.0
    P = np.stack([oracle.lu_solve(Ad, b[:, l]) for l in range(b.shape[1])], axis=1)
    Un, Vn, Wn = oracle.grad_correct(g, P, U, V, W, tau)
    d0 = np.abs(oracle.divergence(g, U, V, W)).max()
    d1 = np.abs(oracle.divergence(g, Un, Vn, Wn)).max()
    assert d0 > 1e-2 and d1 <= 1e-12 * d0
    # idempotent: the projected field needs no further correction
    b2 = oracle.divergence(g, Un, Vn, Wn, scale=-1.0 / tau)
    if op.singular:
        b2[0] = 0.0
    P2 = np.stack([oracle.lu_solve(Ad, b2[:, l]) for l in range(2)], axis=1)
    assert np.abs(P2).max() <= 1e-10 * np.abs(P).max()
