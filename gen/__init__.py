"""Seeded synthetic inputs shared by the CUDA path, the CPU oracle, the tests and the bench.

This package builds inputs only: finite-volume pressure-Poisson operators in CSR form and
seeded right-hand-side / ensemble blocks in the row-interleaved n x m layout (element (k, l)
of a block at flat index k*m + l, the layout of Section 2.3). It holds none of the method's
arithmetic (no SpMV, no Krylov step, no preconditioner); both the oracle and the GPU path
consume the arrays it returns.
"""

from .operators import Operator, fv_poisson, uniform_nodes, tanh_nodes
from .workloads import (
    dirichlet_box,
    channel,
    cubes,
    rhs_uniform,
    rhs_normal,
    WORKLOADS,
    serving_operators,
    serving_requests,
    poisson_arrivals,
)
from .fields import Grid, grid_of, predictor_velocity

__all__ = [
    "Operator",
    "fv_poisson",
    "uniform_nodes",
    "tanh_nodes",
    "dirichlet_box",
    "channel",
    "cubes",
    "rhs_uniform",
    "rhs_normal",
    "WORKLOADS",
    "serving_operators",
    "serving_requests",
    "poisson_arrivals",
    "Grid",
    "grid_of",
    "predictor_velocity",
]
