"""The product's report of the paper's model (a8) against the oracle's pinned formulas (no GPU)."""

import math

import pytest

from oracle import estimates as est
from paper_1711_10622_gb300 import report


@pytest.mark.parametrize("m", [1, 2, 4, 8, 16, 32])
def test_formulas_match_oracle(m):
    assert math.isclose(report.compact_gain(m), est.gain_compact(m), rel_tol=1e-15)
    for C in (6.5, 7.0, 20.0):
        assert math.isclose(report.full_gain(m, C), est.gain_full(m, C), rel_tol=1e-15)
    for theta in (0.75, 0.8, 0.85):
        g = est.gain_compact(m)
        assert math.isclose(report.step_gain(theta, g), est.step_speedup(theta, g), rel_tol=1e-15)
        for beta in (1.0, 5.0, 20.0, 40.0):
            s = est.step_speedup(theta, g)
            assert math.isclose(report.overall_speedup(m, beta, s), est.overall_speedup(m, beta, s), rel_tol=1e-15)


def test_table_on_model_times_reproduces_model():
    # times chosen so that the measured gain equals the compact model exactly
    n, nnz = 1000, 7000
    times = {m: m / est.gain_compact(m) for m in (1, 2, 4, 8, 16)}
    tab = report.estimate_table(times, n, nnz)
    for row in tab["rows"]:
        assert math.isclose(row["measured_gain"], est.gain_compact(row["m"]), rel_tol=1e-12)
        p = row["P_theta0.85_beta5"]
        assert math.isclose(p, est.overall_speedup_closed(row["m"], 5.0, 0.85), rel_tol=1e-12)
    # with theta = 0.85 the paper's optimum among powers of two is m = 2 for beta = 5, 4 for beta = 20
    assert tab["best_m"]["P_theta0.85_beta5"]["m"] == 2
    assert tab["best_m"]["P_theta0.85_beta20"]["m"] == 4


def test_table_needs_m1():
    with pytest.raises(ValueError):
        report.estimate_table({2: 1.0}, 10, 70)
