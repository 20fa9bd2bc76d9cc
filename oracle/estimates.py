"""The paper's closed-form performance model (Section 2.3), written out plainly in FP64.

TEST INFRASTRUCTURE: the reference the product's report module is compared against.

Symbols follow the paper: m ensembles (RHS vectors), n rows, nnz nonzeros, C = nnz/n,
beta = T_A / T_T (averaging over transition interval), theta = t_1^S / t_1 (solver share of a
time step).
"""

from __future__ import annotations

import math


def traffic_bytes(n: int, nnz: int, m: int) -> float:
    """Sigma_m = 4n(2m+1) + 12 nnz + 8 m nnz: bytes moved by CRS GSpMV, X re-read per nonzero
    (Section 2.3, the traffic count following Fig. GSpMV)."""
    return 4.0 * n * (2 * m + 1) + 12.0 * nnz + 8.0 * m * nnz


def gain_full(m: int, C: float) -> float:
    """m Sigma_1 / Sigma_m = m(5C+3) / (2m(C+1) + 3C + 1)  (Eq. mem_GSpMV_full)."""
    return m * (5.0 * C + 3.0) / (2.0 * m * (C + 1.0) + 3.0 * C + 1.0)


def gain_compact(m: int) -> float:
    """m Sigma_1 / Sigma_m ~ 5m / (2m + 3) for C >> 1  (Eq. mem_GSpMV_compact)."""
    return 5.0 * m / (2.0 * m + 3.0)


def step_speedup(theta: float, solver_gain: float) -> float:
    """m t_1 / t_m = 1 / (theta / (m t_1^S / t_m^S) + (1 - theta))  (Eq. est2_1)."""
    return 1.0 / (theta / solver_gain + (1.0 - theta))


def overall_speedup(m: int, beta: float, step_gain: float) -> float:
    """P_m = (1 + beta) / (m + beta) * (m t_1 / t_m)  (Eq. est2)."""
    return (1.0 + beta) / (m + beta) * step_gain


def overall_speedup_closed(m: int, beta: float, theta: float) -> float:
    """P_m = (1+beta)/(m+beta) * 5m / (5m - 3 theta (m-1))  (Eq. est3)."""
    return (1.0 + beta) / (m + beta) * 5.0 * m / (5.0 * m - 3.0 * theta * (m - 1))


def optimal_m(beta: float, theta: float) -> float:
    """m* = sqrt(3 beta theta / (5 - 3 theta)), the stationary point of Eq. est3 in m."""
    return math.sqrt(3.0 * beta * theta / (5.0 - 3.0 * theta))
