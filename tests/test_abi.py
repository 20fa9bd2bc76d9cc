"""The C-ABI library builds, loads and exports every symbol its header declares (no GPU needed).

Argument validation happens on the host before any CUDA call, so invalid-argument paths are
exercised here too.
"""

import ctypes
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


@pytest.fixture(scope="module")
def native():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1711_10622_gb300 import build, _native

    build.build()
    return _native


def _declared_functions():
    names = set()
    for fn in os.listdir(HEADER_DIR):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(ens_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("ens_create_matrix", "ens_destroy_matrix", "ens_gspmv", "ens_gspmv_host", "ens_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(native):
    L = ctypes.CDLL(native.library_path())
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_version_and_empty_error(native):
    L = native.lib()
    assert b"sm_103a" in L.ens_version()
    assert L.ens_last_error() == b"" or isinstance(L.ens_last_error(), bytes)


def _create(native, row_ptr, col_idx, val, n=None, nnz=None, flags=0):
    L = native.lib()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    h = ctypes.c_void_p()
    st = L.ens_create_matrix(
        len(row_ptr) - 1 if n is None else n,
        len(col_idx) if nnz is None else nnz,
        row_ptr.ctypes.data_as(ctypes.c_void_p),
        col_idx.ctypes.data_as(ctypes.c_void_p),
        val.ctypes.data_as(ctypes.c_void_p),
        flags,
        None,
        ctypes.byref(h),
    )
    return st, L.ens_last_error().decode()


@pytest.mark.parametrize(
    "row_ptr,col_idx,kw,msg",
    [
        ([1, 2], [0], {}, "row_ptr[0]"),
        ([0, 2, 1], [0, 1], {}, "decreases"),
        ([0, 1, 2], [0, 2], {}, "col_idx"),
        ([0, 1, 2], [0, -1], {}, "col_idx"),
        ([0, 1, 3], [0, 1], {"nnz": 2}, "row_ptr[n]"),
        ([0], [], {"n": 0}, "n = 0"),
        ([0, 1], [0], {"flags": 0x10}, "flags"),
    ],
)
def test_create_matrix_rejects_bad_csr(native, row_ptr, col_idx, kw, msg):
    st, err = _create(native, row_ptr, col_idx, np.ones(len(col_idx)), **kw)
    assert st == native.ENS_ERR_INVALID
    assert msg in err


def test_null_arguments_rejected(native):
    L = native.lib()
    assert L.ens_gspmv(None, 4, 0, None, None, None) == native.ENS_ERR_INVALID
    assert "NULL" in L.ens_last_error().decode()
    assert L.ens_create_matrix(4, 4, None, None, None, 0, None, None) == native.ENS_ERR_INVALID
    assert L.ens_destroy_matrix(None) == native.ENS_OK
    assert L.ens_set_f64_mode(None, 0) == native.ENS_ERR_INVALID
    assert L.ens_matrix_info(None, None, None, None) == native.ENS_ERR_INVALID


def _create_grid(native, nx, ny, nz, nodes=None, bc=(1, 0, 1), solid=None, out=True):
    L = native.lib()
    if nodes is None:
        nodes = [np.linspace(0.0, 1.0, k + 1) for k in (nx, ny, nz)]
    nodes = [np.ascontiguousarray(a, dtype=np.float64) for a in nodes]
    bca = np.ascontiguousarray(bc, dtype=np.int32)
    sp = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8)
    h = ctypes.c_void_p()
    st = L.ens_create_grid(
        nx, ny, nz, *(a.ctypes.data_as(ctypes.c_void_p) for a in nodes), bca.ctypes.data_as(ctypes.c_void_p),
        None if sp is None else sp.ctypes.data_as(ctypes.c_void_p), None, ctypes.byref(h) if out else None,
    )
    return st, L.ens_last_error().decode()


@pytest.mark.parametrize(
    "args,msg",
    [
        (dict(nx=0, ny=4, nz=4), "dimensions"),
        (dict(nx=2, ny=4, nz=4), "periodic direction 0"),
        (dict(nx=4, ny=4, nz=4, bc=(1, 7, 1)), "unknown boundary code"),
        (dict(nx=4, ny=4, nz=4, nodes=[np.linspace(1, 0, 5), np.linspace(0, 1, 5), np.linspace(0, 1, 5)]), "increasing"),
        (dict(nx=4, ny=4, nz=4, nodes=[np.array([0, 1, np.nan, 3, 4.0]), np.linspace(0, 1, 5), np.linspace(0, 1, 5)]), "finite"),
        (dict(nx=4, ny=4, nz=4, solid=np.ones(64)), "solid"),
        (dict(nx=4, ny=4, nz=4, out=False), "out is NULL"),
    ],
)
def test_create_grid_rejects_bad_descriptions(native, args, msg):
    st, err = _create_grid(native, **args)
    assert st == native.ENS_ERR_INVALID
    assert msg in err


def test_projection_null_arguments_rejected(native):
    L = native.lib()
    assert L.ens_divergence(None, 2, 1.0, None, None, None, None, None) == native.ENS_ERR_INVALID
    assert L.ens_grad_correct(None, 2, 1.0, None, None, None, None, None) == native.ENS_ERR_INVALID
    assert L.ens_grid_info(None, None, None) == native.ENS_ERR_INVALID
    assert L.ens_destroy_grid(None) == native.ENS_OK
