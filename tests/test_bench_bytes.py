"""The bench's byte accounting (no GPU): the algorithmic bytes of one GSpMV, which the roofline's
`achieved` divides by the measured launch time, and the paper's traffic model Sigma_m (Section 2.3),
against the per-width figures written out for the channel workload (n = 4,194,304 rows,
nnz = 29,294,592: matrix once as 4(n+1) + 12 nnz bytes in FP64, X read once and Y written once)."""

import pytest

import bench

N, NNZ = 4_194_304, 29_294_592

# MB (1e6 bytes), one decimal: FP64 algorithmic, FP32 algorithmic, the paper's Sigma_m
TABLE = {
    1: (435.4, 284.7, 636.2),
    2: (502.5, 318.2, 904.1),
    4: (636.7, 385.4, 1440.0),
    8: (905.2, 519.6, 2511.6),
    16: (1442.1, 788.0, 4654.9),
    32: (2515.8, 1324.9, 8941.5),
}


@pytest.mark.parametrize("m", sorted(TABLE))
def test_algorithmic_and_model_bytes(m):
    f64, f32, sigma = TABLE[m]
    assert round(bench.alg_bytes(N, NNZ, m) / 1e6, 1) == f64
    assert round(bench.alg_bytes(N, NNZ, m, sv=4, sx=4) / 1e6, 1) == f32
    assert round(bench.paper_traffic(N, NNZ, m) / 1e6, 1) == sigma


def test_roofline_fraction_arithmetic():
    # achieved = bytes per launch / launch time; frac = achieved / peak
    b = bench.alg_bytes(N, NNZ, 32)
    achieved = b / 922.3e-6 / 1e9
    assert 2700 < achieved < 2750
    assert abs(achieved / 6792.4 - 0.4016) < 1e-3
