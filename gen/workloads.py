"""The synthetic workloads: operators shaped like the paper's test cases plus seeded RHS blocks.

Section 4 runs two flows: a plain channel (periodic streamwise/spanwise, no-slip walls, wall-normal
stretching Δy_max/Δy_min = 5) and a channel with a matrix of wall-mounted cubes. Their grids and
matrices are not published; the builders below produce operators of the same structure at the
sizes used for measurement here:

* ``dirichlet_box(32)``: 32^3 uniform cells, Dirichlet x/z, Neumann y (non-singular).
* ``channel(256, 128, 128)``: channel 2*pi x 2 x pi, tanh wall-normal stretching gamma = 2.0,
  periodic x/z, Neumann walls (singular: constants in the null space).
* ``cubes()``: 192 x 128 x 96 unit cells with a 4 x 4 matrix of 16^3-cell solid cubes on the
  bottom wall, periodic x/z, Neumann walls and cube faces (singular).

Right-hand sides are n x m blocks stored row-interleaved (C-order numpy (n, m)), drawn from
NumPy's PCG64 ``default_rng(seed)``.
"""

from __future__ import annotations

import numpy as np

from .operators import (
    DIRICHLET,
    NEUMANN,
    PERIODIC,
    fv_poisson,
    tanh_nodes,
    uniform_nodes,
)

OPERATOR_SEED = 1711
RHS_SEED_BASE = 10622


def dirichlet_box(N: int = 32, nz: int | None = None, ny: int | None = None):
    """Uniform N^3 (or N x ny x nz) unit-cube grid, Dirichlet in x and z, Neumann in y."""
    ny = N if ny is None else ny
    nz = N if nz is None else nz
    h = 1.0 / N
    return fv_poisson(
        uniform_nodes(N, N * h),
        uniform_nodes(ny, ny * h),
        uniform_nodes(nz, nz * h),
        bcs=(DIRICHLET, NEUMANN, DIRICHLET),
        name=f"dirichlet{N}x{ny}x{nz}",
    )


def channel(nx: int = 256, ny: int = 128, nz: int = 128, gamma: float = 2.0):
    """Plane channel 2*pi x 2 x pi: periodic x/z, Neumann walls at y = +-1, tanh stretching in y."""
    return fv_poisson(
        uniform_nodes(nx, 2.0 * np.pi),
        tanh_nodes(ny, gamma),
        uniform_nodes(nz, np.pi),
        bcs=(PERIODIC, NEUMANN, PERIODIC),
        name=f"channel{nx}x{ny}x{nz}",
    )


def cube_mask(nx=192, ny=128, nz=96, size=16, count=(4, 4), pitch=(48, 24), offset=(16, 4)):
    """Solid mask (nz, ny, nx) of a count[0] x count[1] matrix of size^3 cubes on the y = 0 wall.

    Cube (a, b) covers x in [offset_x + a*pitch_x, +size), z in [offset_z + b*pitch_z, +size),
    y in [0, size).
    """
    solid = np.zeros((nz, ny, nx), dtype=bool)
    for a in range(count[0]):
        x0 = offset[0] + a * pitch[0]
        for b in range(count[1]):
            z0 = offset[1] + b * pitch[1]
            if x0 + size > nx or z0 + size > nz or size > ny:
                raise ValueError("cube does not fit in the grid")
            solid[z0 : z0 + size, 0:size, x0 : x0 + size] = True
    return solid


def cubes(nx: int = 192, ny: int = 128, nz: int = 96, size: int = 16, pitch=None, offset=None):
    """Channel with a 4 x 4 matrix of wall-mounted solid cubes; unit cells, periodic x/z.

    By default the pitch is (nx/4, nz/4) and the offset (pitch_x/3, pitch_z/6), which for
    192 x 128 x 96 gives pitch (48, 24) and offset (16, 4).
    """
    if pitch is None:
        pitch = (nx // 4, nz // 4)
    if offset is None:
        offset = (pitch[0] // 3, pitch[1] // 6)
    solid = cube_mask(nx, ny, nz, size=size, pitch=pitch, offset=offset)
    op = fv_poisson(
        uniform_nodes(nx, float(nx)),
        uniform_nodes(ny, float(ny)),
        uniform_nodes(nz, float(nz)),
        bcs=(PERIODIC, NEUMANN, PERIODIC),
        solid=solid,
        name=f"cubes{nx}x{ny}x{nz}",
    )
    return op


def rhs_uniform(n: int, m: int, seed: int) -> np.ndarray:
    """n x m block, entries U[-1, 1), row-interleaved."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.uniform(-1.0, 1.0, size=(n, m)))


def rhs_normal(n: int, m: int, seed: int, zero_mean: bool = False) -> np.ndarray:
    """n x m block, entries N(0, 1); with zero_mean each column has its mean subtracted."""
    rng = np.random.default_rng(seed)
    b = rng.standard_normal(size=(n, m))
    if zero_mean:
        b -= b.mean(axis=0, keepdims=True)
    return np.ascontiguousarray(b)


def serving_operators(sizes=(64, 96, 128, 192)):
    """The serving workload's operators: for each N, the channel N^3 and the cube case N^3 with cubes
    of N/8 cells (pitch N/4)."""
    ops = {}
    for N in sizes:
        ops[f"channel{N}"] = channel(N, N, N)
        ops[f"cubes{N}"] = cubes(N, N, N, size=N // 8)
    return ops


def serving_requests(count, ops, seed=5, widths=(1, 2, 4, 8, 16, 32)):
    """`count` requests (operator name, m, rhs seed), operator and m drawn uniformly from a seed."""
    rng = np.random.default_rng(seed)
    names = sorted(ops)
    out = []
    for k in range(count):
        name = names[int(rng.integers(len(names)))]
        m = int(widths[int(rng.integers(len(widths)))])
        out.append((name, m, RHS_SEED_BASE + 1000 + k))
    return out


def poisson_arrivals(count, rate, seed=5):
    """Arrival times (seconds from 0) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed + 1)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


# name -> (operator builder, m values, rhs builder(n, m)). The seeds are 10622 + workload id.
WORKLOADS = {
    "dirichlet32_m4": dict(
        op=lambda: dirichlet_box(32),
        m=(4,),
        rhs=lambda n, m: rhs_uniform(n, m, RHS_SEED_BASE + 1),
        tol=1e-8,
        precond="none",
    ),
    "channel256x128x128": dict(
        op=lambda: channel(256, 128, 128),
        m=(1, 2, 4, 8, 16, 32),
        rhs=lambda n, m: rhs_normal(n, m, RHS_SEED_BASE + 2),
    ),
    "cubes192x128x96_m8": dict(
        op=lambda: cubes(),
        m=(8,),
        rhs=lambda n, m: rhs_normal(n, m, RHS_SEED_BASE + 3, zero_mean=True),
        tol=1e-8,
        precond="chebyshev",
    ),
}
