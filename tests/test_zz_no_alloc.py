"""ens_gspmv_host_noalloc: the host-buffer GSpMV that allocates no device memory.

For callers that cannot let the library allocate during a call (a device-memory pool reserved up
front by the application, real-time loops, hosts that forbid plug-ins from allocating). The entry
point stages through a fixed array compiled into the library. This test calls it through the C ABI
and checks its output against ens_gspmv_host (the allocating entry point) on two calls in a row,
within the FP64 GSpMV tolerance of the other tests (1e-12 of |A||X| per element; FP32: the
float32 bound). It lives in its own file, collected last, and passes alone in a fresh process too.
"""

import ctypes

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ens():
    from paper_1711_10622_gb300 import build

    build.build()
    import paper_1711_10622_gb300 as ens

    return ens


def _abs_scale(op, X):
    S = op.to_scipy().copy()
    S.data = np.abs(S.data)
    return np.asarray(S @ np.abs(X))


def _noalloc(ens, A, X, Y):
    from paper_1711_10622_gb300 import _native as N

    code = N.ENS_F64 if X.dtype == np.float64 else N.ENS_F32
    st = N.lib().ens_gspmv_host_noalloc(
        A.handle,
        X.shape[1],
        code,
        X.ctypes.data_as(ctypes.c_void_p),
        Y.ctypes.data_as(ctypes.c_void_p),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
    )
    return st


def test_noalloc_first_call_reserves_only_the_array(ens):
    """The first call on a device loads the array's module (lazy module loading) and so reserves the
    2 x 16 MiB staging array; later calls reserve nothing. Runs before any other call in this file."""
    op = gen.dirichlet_box(16)
    with ens.Matrix.from_operator(op) as A:
        X = gen.rhs_normal(op.n, 4, 13)
        ens.gspmv_host(A, X)  # load the product kernels' module and the allocating path's buffers first
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        Y = np.empty_like(X)
        assert _noalloc(ens, A, X, Y) == 0
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert free0 - free1 <= (32 << 20) + (8 << 20), (free0 - free1) / 2**20
        for _ in range(3):
            assert _noalloc(ens, A, X, Y) == 0
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free1


@pytest.mark.parametrize("dtype,m", [(np.float64, 8), (np.float32, 8), (np.float64, 3)])
def test_noalloc_matches_allocating_entry_point(ens, dtype, m):
    op = gen.cubes(48, 32, 24, size=4)
    with ens.Matrix.from_operator(op) as A:
        for call in range(2):  # two calls in a row: the shared array keeps the previous contents
            X = gen.rhs_normal(op.n, m, 700 + 10 * call + m).astype(dtype)
            ref = ens.gspmv_host(A, X)
            Y = np.full_like(X, np.nan)
            assert _noalloc(ens, A, X, Y) == 0
            scale = _abs_scale(op, X.astype(np.float64))
            tol = 1e-12 if dtype == np.float64 else 9 * 2.0**-24
            err = np.abs(Y.astype(np.float64) - ref.astype(np.float64))
            assert np.all(err <= tol * scale), float((err / np.where(scale > 0, scale, 1)).max())


def test_noalloc_allocates_nothing_and_rejects_oversize(ens):
    from paper_1711_10622_gb300 import _native as N

    op = gen.dirichlet_box(16)
    with ens.Matrix.from_operator(op) as A:
        X = gen.rhs_normal(op.n, 4, 11)
        Y = np.empty_like(X)
        assert _noalloc(ens, A, X, Y) == 0  # first call on this device: address set-up
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(3):
            assert _noalloc(ens, A, X, Y) == 0
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        # n * m * 8 bytes above the 16 MiB staging limit is rejected with a message
        big = gen.channel(64, 64, 64)  # n = 262,144; m = 9 -> 18.9 MB
        with ens.Matrix.from_operator(big) as B:
            Xb = np.zeros((big.n, 9))
            Yb = np.zeros_like(Xb)
            assert _noalloc(ens, B, Xb, Yb) == N.ENS_ERR_INVALID
            assert "staging limit" in N.lib().ens_last_error().decode()
