"""The OpenMP build of the oracle (the all-core CPU baseline) gives the serial oracle's bits.

It is the same C source compiled with -fopenmp: products split their rows over threads and block
solves their columns, and every value is still computed by the same serial code in the same order.
The row-wise product (the loop order of Fig. GSpMV, Section 2.3) sums every element in the same
order as the column-by-column definition, so it too must agree bit for bit.
"""

import numpy as np
import pytest

import gen
import oracle


@pytest.fixture(scope="module")
def omp():
    if oracle.lib_omp() is None:
        pytest.skip("gcc without OpenMP")
    return oracle


@pytest.mark.parametrize("m", [1, 3, 8])
def test_rowwise_and_parallel_products_match_the_definition_bitwise(omp, m):
    op = gen.cubes(48, 32, 24, size=4)
    X = gen.rhs_normal(op.n, m, 60 + m)
    ref = oracle.gspmv(op, X)
    np.testing.assert_array_equal(oracle.gspmv_rowwise(op, X), ref)
    np.testing.assert_array_equal(oracle.gspmv(op, X, parallel=True), ref)
    np.testing.assert_array_equal(oracle.gspmv_rowwise(op, X, parallel=True), ref)


@pytest.mark.parametrize("precond", ["none", "chebyshev", "amg"])
def test_parallel_block_solve_matches_serial_bitwise(omp, precond):
    op = gen.dirichlet_box(12)
    B = gen.rhs_uniform(op.n, 5, 61)
    H = oracle.AMG(op) if precond == "amg" else None
    a = oracle.solve_block(op, B, 1e-9, precond=precond, amg=H)
    b = oracle.solve_block(op, B, 1e-9, precond=precond, amg=H, parallel=True)
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
    assert oracle.threads(parallel=True) >= 1 and oracle.threads(parallel=False) == 1
