"""GPU GSpMV (ens_gspmv through the C ABI) against the CPU oracle, element by element.

Tolerances (Section 2.3 definition, summation over j in CSR order):
* float64: |Y - Y_oracle| <= 1e-12 * (|A| |X|) per element (products and sums may be rounded
  differently from the oracle; both are far inside this bound).
* float32: the oracle evaluates the same product in float64 on the float32-rounded matrix and
  block; the float32 kernel's error is at most about (row length + 1) * 2^-24 of (|A| |X|).
"""

import numpy as np
import pytest

import gen
import oracle

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


def _random_csr(n, seed, max_len=12, empty_frac=0.1, long_rows=()):
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, max_len + 1, size=n)
    lens[rng.random(n) < empty_frac] = 0
    for r, L in long_rows:
        lens[r] = L
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    cols = np.concatenate([np.sort(rng.choice(n, size=L, replace=L > n)) for L in lens]) if rp[-1] else np.zeros(0)
    val = rng.standard_normal(int(rp[-1]))
    op = gen.Operator(
        name="random",
        shape=(n, 1, 1),
        bcs=("x", "x", "x"),
        row_ptr=rp.astype(np.int32),
        col_idx=cols.astype(np.int32),
        val=val,
        singular=False,
    )
    return op


OPS = {
    "dirichlet12": lambda: gen.dirichlet_box(12),
    "channel20x14x10": lambda: gen.channel(20, 14, 10),
    "cubes48x32x24": lambda: gen.cubes(48, 32, 24, size=4),
    "random777": lambda: _random_csr(777, 3, long_rows=[(5, 70), (100, 65)]),  # rows > 64: native only
    # split-eligible irregular rows: 0..12 nonzeros with empty rows, every tail-group size
    "random_split": lambda: _random_csr(1000, 5, max_len=12, empty_frac=0.1),
    # rows of up to 24 nonzeros: tile segments exceed the shared-memory tile (global-memory path)
    "random_wide": lambda: _random_csr(600, 6, max_len=24, empty_frac=0.05),
    "one_row": lambda: _random_csr(1, 4, max_len=1, empty_frac=0.0),
}
_cache = {}


def _op(name):
    if name not in _cache:
        _cache[name] = OPS[name]()
    return _cache[name]


def _check_f64(op, X, Y):
    ref = oracle.gspmv(op, X)
    scale = _abs_scale(op, X)
    err = np.abs(Y - ref)
    assert np.all(np.isfinite(Y))
    assert np.all(err <= 1e-12 * scale), float((err / np.where(scale > 0, scale, 1)).max())


def _check_f32(op, X32, Y32):
    op64 = gen.Operator(op.name, op.shape, op.bcs, op.row_ptr, op.col_idx, op.val.astype(np.float32).astype(np.float64), op.singular)
    X = X32.astype(np.float64)
    ref = oracle.gspmv(op64, X)
    scale = _abs_scale(op64, X)
    Lmax = int(np.diff(op.row_ptr).max())
    tol = (Lmax + 2) * 2.0**-24
    err = np.abs(Y32.astype(np.float64) - ref)
    assert np.all(err <= tol * scale + 1e-30), float((err / np.where(scale > 0, scale, 1)).max())


M_VALUES = [1, 2, 3, 4, 5, 7, 8, 16, 32, 33, 64]


@pytest.mark.parametrize("name", list(OPS))
@pytest.mark.parametrize("m", M_VALUES)
@pytest.mark.parametrize("mode", ["auto", "native", "split", "hybrid", "f32"])
def test_gspmv_parity(ens, name, m, mode):
    op = _op(name)
    X = gen.rhs_normal(op.n, m, 1000 + m)
    with ens.Matrix.from_operator(op) as A:
        if mode == "f32":
            X32 = X.astype(np.float32)
            Y = ens.gspmv(A, torch.from_numpy(X32).cuda()).cpu().numpy()
            _check_f32(op, X32, Y)
        else:
            A.set_f64_mode(mode)
            Y = ens.gspmv(A, torch.from_numpy(X).cuda()).cpu().numpy()
            _check_f64(op, X, Y)


@pytest.mark.parametrize("name", list(OPS))
@pytest.mark.parametrize("m", M_VALUES)
@pytest.mark.parametrize("mode", ["native", "split", "f32"])
def test_gspmv_parity_untiled(ens, name, m, mode):
    """The untiled row traversal (no shared-memory tile) on every operator shape, forced."""
    op = _op(name)
    X = gen.rhs_normal(op.n, m, 900 + m)
    with ens.Matrix.from_operator(op) as A:
        A.set_untiled(1)
        if mode == "f32":
            X32 = X.astype(np.float32)
            Y = ens.gspmv(A, torch.from_numpy(X32).cuda()).cpu().numpy()
            _check_f32(op, X32, Y)
            return
        A.set_f64_mode(mode)
        Y = ens.gspmv(A, torch.from_numpy(X).cuda()).cpu().numpy()
    _check_f64(op, X, Y)


@pytest.mark.parametrize("untiled", [0, 1])
def test_gspmv_host_pipelined_both_traversals(ens, untiled):
    op = gen.cubes(48, 32, 24, size=4)
    X = gen.rhs_normal(op.n, 8, 77)
    with ens.Matrix.from_operator(op) as A:
        A.set_untiled(untiled)
        Y = ens.gspmv_host(A, X)
    _check_f64(op, X, Y)


def test_gspmv_deterministic_and_on_side_stream(ens):
    op = _op("cubes48x32x24")
    X = torch.from_numpy(gen.rhs_normal(op.n, 8, 5)).cuda()
    s = torch.cuda.Stream()
    with ens.Matrix.from_operator(op) as A:
        Y1 = ens.gspmv(A, X)
        with torch.cuda.stream(s):
            Y2 = ens.gspmv(A, X, stream=s)
        s.synchronize()
        assert torch.equal(Y1, Y2)


def test_gspmv_misaligned_views(ens):
    op = _op("channel20x14x10")
    m = 4
    with ens.Matrix.from_operator(op) as A:
        for dt in (torch.float64, torch.float32):
            buf = torch.randn(op.n * m + 1, dtype=dt, device="cuda")
            X = buf[1:].view(op.n, m)  # 8-byte (f64) / 4-byte (f32) aligned, not 16-byte
            Yb = torch.zeros(op.n * m + 1, dtype=dt, device="cuda")
            Y = Yb[1:].view(op.n, m)
            ens.gspmv(A, X, Y)
            Xn = X.cpu().numpy()
            if dt == torch.float64:
                _check_f64(op, Xn, Y.cpu().numpy())
            else:
                _check_f32(op, Xn, Y.cpu().numpy())


def test_split_range_fallbacks(ens):
    op = _op("cubes48x32x24")
    m = 8
    X = gen.rhs_normal(op.n, m, 7)
    X[::97, 3] = 0.0  # exact zeros: native path for those row segments
    X[::89, 0] = 1e-20  # below the split range
    X[::83, 5] = 3e25  # above the split range
    with ens.Matrix.from_operator(op) as A:
        Y = ens.gspmv(A, torch.from_numpy(X).cuda()).cpu().numpy()
        _check_f64(op, X, Y)
    # products above the float range (|a| ~ 1e13, |x| ~ 3e25): the split accumulators overflow
    # and those row segments are recomputed natively
    big = gen.Operator(op.name, op.shape, op.bcs, op.row_ptr, op.col_idx, op.val * 1e15, op.singular)
    Xb = X.copy()
    Xb[::61, 6] = 3e25
    Xb[::67, 2] = 1e30  # above the split window
    with ens.Matrix.from_operator(big) as A:
        Y = ens.gspmv(A, torch.from_numpy(Xb).cuda()).cpu().numpy()
        assert np.all(np.isfinite(Y))
        _check_f64(big, Xb, Y)
    # matrix values outside the split range: the whole product is native
    scaled = gen.Operator(op.name, op.shape, op.bcs, op.row_ptr, op.col_idx, op.val * 1e-18, op.singular)
    with ens.Matrix.from_operator(scaled) as A:
        Y = ens.gspmv(A, torch.from_numpy(X).cuda()).cpu().numpy()
        _check_f64(scaled, X, Y)


def test_nonfinite_propagates(ens):
    op = _op("dirichlet12")
    X = gen.rhs_normal(op.n, 2, 8)
    X[10, 1] = np.nan
    with ens.Matrix.from_operator(op) as A:
        Y = ens.gspmv(A, torch.from_numpy(X).cuda()).cpu().numpy()
    ref = oracle.gspmv(op, X)
    assert np.array_equal(np.isnan(Y), np.isnan(ref))
    fin = ~np.isnan(ref)
    assert np.all(np.abs(Y[fin] - ref[fin]) <= 1e-12 * _abs_scale(op, np.nan_to_num(X))[fin])


def test_gspmv_host_buffers(ens):
    op = _op("channel20x14x10")
    for m, dt in ((8, np.float64), (3, np.float64), (8, np.float32)):
        X = gen.rhs_normal(op.n, m, 9).astype(dt)
        with ens.Matrix.from_operator(op) as A:
            Y = ens.gspmv_host(A, X)
        if dt == np.float64:
            _check_f64(op, X, Y)
        else:
            _check_f32(op, X, Y)


@pytest.mark.parametrize("m,dt", [(1, np.float64), (8, np.float64), (32, np.float64), (5, np.float64), (8, np.float32)])
def test_gspmv_host_pipelined(ens, m, dt):
    """ens_gspmv_host on an operator of 140 tiles: X arrives in row blocks, up to 16 row chunks run
    as the blocks they read land and their Y rows are copied out while later chunks compute; every
    row against the definition (FP64 bound 1e-12 of |A||X|, FP32 bound (L+2) 2^-24)."""
    op = _op("cubes48x32x24")
    X = gen.rhs_normal(op.n, m, 600 + m).astype(dt)
    with ens.Matrix.from_operator(op) as A:
        Y = ens.gspmv_host(A, X)
        Y2 = ens.gspmv_host(A, X)  # the pipeline's streams and events are reused
    assert np.array_equal(Y, Y2)
    if dt == np.float64:
        _check_f64(op, X, Y)
    else:
        _check_f32(op, X, Y)


@pytest.mark.parametrize("m", [1, 4, 16])
def test_gspmv_host_pipelined_periodic(ens, m):
    """A channel operator periodic in x and z: the first row chunk reads the last z-planes of X (the
    wrap-around coupling), so its X blocks are not a prefix; every row against the definition."""
    op = gen.channel(32, 16, 64)
    assert op.n // 256 >= 16  # at least 16 row chunks
    X = gen.rhs_normal(op.n, m, 700 + m)
    with ens.Matrix.from_operator(op) as A:
        Y = ens.gspmv_host(A, X)
    _check_f64(op, X, Y)


def test_gspmv_host_in_place(ens):
    """ens_gspmv_host with Y the same host array as X: the input is fully read before any output
    row is written back."""
    op = _op("cubes48x32x24")
    m = 8
    X = gen.rhs_normal(op.n, m, 610)
    buf = X.copy()
    with ens.Matrix.from_operator(op) as A:
        ens.gspmv_host(A, buf, buf)
    _check_f64(op, X, buf)


def test_invalid_arguments(ens):
    op = _op("dirichlet12")
    with ens.Matrix.from_operator(op) as A:
        X = torch.zeros(op.n, 4, dtype=torch.float64, device="cuda")
        with pytest.raises(ens.EnsError):
            ens.gspmv(A, X, X)  # overlapping X and Y
        with pytest.raises(ValueError):
            ens.gspmv(A, torch.zeros(op.n + 1, 4, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("m", [1, 8, 32])
def test_full_size_channel_sampled(ens, m):
    """The channel workload 256 x 128 x 128 at full size, in the launch configuration the bench
    times: sampled rows against the definition, plus 1^T A X = 0 (rows and columns of the
    symmetric singular operator sum to zero) over the whole output."""
    op = gen.WORKLOADS["channel256x128x128"]["op"]()
    X = gen.WORKLOADS["channel256x128x128"]["rhs"](op.n, m)
    rows = np.unique(np.concatenate([np.random.default_rng(m).integers(0, op.n, 3000), [0, op.n - 1]]))
    ref = oracle.gspmv_rows(op, rows, X)
    sub = gen.Operator("s", op.shape, op.bcs, op.row_ptr, op.col_idx, np.abs(op.val), op.singular)
    scale = oracle.gspmv_rows(sub, rows, np.abs(X))
    with ens.Matrix.from_operator(op) as A:
        Xd = torch.from_numpy(X).cuda()
        for mode in ("auto", "native", "hybrid", "split"):
            A.set_f64_mode(mode)
            Yd = ens.gspmv(A, Xd)
            Y = Yd[torch.from_numpy(rows).cuda()].cpu().numpy()
            assert np.all(np.abs(Y - ref) <= 1e-12 * scale)
            colsum = Yd.sum(dim=0).cpu().numpy()
            total = float(np.abs(op.val).max() * np.abs(X).sum(axis=0).max() * 7)
            assert np.all(np.abs(colsum) <= 1e-10 * total)
        Y32 = ens.gspmv(A, Xd.float())[torch.from_numpy(rows).cuda()].double().cpu().numpy()
        assert np.all(np.abs(Y32 - ref) <= 1e-5 * scale)


@pytest.mark.parametrize("share", [0, 8, 12, 16, 24, 32])
def test_hybrid_native_share_parity(ens, share):
    """Every split/native mix of the FP64 product stays within the FP64 bound."""
    op = _op("cubes48x32x24")
    for m in (2, 8, 32):
        X = gen.rhs_normal(op.n, m, 300 + m)
        with ens.Matrix.from_operator(op) as A:
            A.set_native_share(share)
            Y = ens.gspmv(A, torch.from_numpy(X).cuda()).cpu().numpy()
        _check_f64(op, X, Y)


def test_autotune_then_parity(ens):
    op = _op("channel20x14x10")
    with ens.Matrix.from_operator(op) as A:
        for m in (1, 4, 8, 32):
            for dt in ("f64", "f32"):
                r = A.autotune(m, dt)
                assert r["lanes"] >= 1 and r["best_us"] > 0
                assert r["share"] in (0, 8, 12, 16, 24, 32, 64) or dt == "f32"  # 64: column hybrid
                X = gen.rhs_normal(op.n, m, 500 + m)
                if dt == "f64":
                    Y = ens.gspmv(A, torch.from_numpy(X).cuda()).cpu().numpy()
                    _check_f64(op, X, Y)
                else:
                    X32 = X.astype(np.float32)
                    Y = ens.gspmv(A, torch.from_numpy(X32).cuda()).cpu().numpy()
                    _check_f32(op, X32, Y)
