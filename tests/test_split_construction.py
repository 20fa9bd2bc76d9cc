"""Host-side check of the split-float FP64 construction used by the GSpMV kernels.

The kernels cut a double x into floats hi + lo with integer bit operations (funnel shift, bit
select, masks) and one exact FP32 subtract and multiply. This test restates those bit operations
in numpy on the CPU and checks the mathematical claims the kernels rely on:
  * hi + lo reproduces x to better than 2^-46 |x| for every biased exponent in the window
    [983, 1110], and exactly for +-0;
  * lo is computed exactly (the subtract and the power-of-two scaling do not round);
  * the range word is below the window bound exactly for exponents inside the window.
"""

import numpy as np

E_LO = 983
WINDOW = np.uint32(128 << 21)
G_BITS = np.uint32(0x34000000)


def _words(x):
    b = np.asarray(x, dtype=np.float64).view(np.uint64)
    return (b >> np.uint64(32)).astype(np.uint32), (b & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def _split(x):
    hw, lw = _words(x)
    with np.errstate(over="ignore"):
        fb = (hw << np.uint32(3)) | (lw >> np.uint32(29))  # funnel shift (hw:lw) << 3, high word
        hb = (fb & np.uint32(0x3FFFFFFF)) | (hw & np.uint32(0xC0000000))
        g = ((lw >> np.uint32(6)) & np.uint32(0x007FFFFF)) | G_BITS
        p = hb & np.uint32(0xFF800000)
    hi = hb.view(np.float32)
    t = (g.view(np.float32) - G_BITS.view(np.float32)).astype(np.float32)
    lo = (t * p.view(np.float32)).astype(np.float32)
    exact_lo = t.astype(np.float64) * p.view(np.float32).astype(np.float64)
    return hi, lo, exact_lo


def _range_word(x):
    hw, _ = _words(x)
    with np.errstate(over="ignore"):
        return (hw * np.uint32(2) - np.uint32(E_LO << 21)).astype(np.uint32)


def test_split_error_bound_over_the_window():
    rng = np.random.default_rng(11)
    for E in range(E_LO, E_LO + 128):
        mant = rng.integers(0, 1 << 52, size=4000, dtype=np.uint64)
        sign = rng.integers(0, 2, size=4000, dtype=np.uint64) << np.uint64(63)
        bits = sign | (np.uint64(E) << np.uint64(52)) | mant
        x = bits.view(np.float64)
        hi, lo, exact_lo = _split(x)
        assert np.array_equal(lo.astype(np.float64), exact_lo), E  # no rounding in lo
        r = x - hi.astype(np.float64) - lo.astype(np.float64)  # exact in double (|r| < 2^-46 |x|)
        assert np.all(np.abs(r) < 2.0**-46 * np.abs(x)), E
        assert np.all(np.abs(r) <= 2.0 ** (E - 1023 - 46)), E  # only mantissa bits 5..0 dropped
        assert np.all(_range_word(x) < WINDOW), E


def test_split_zero_and_window_edges():
    hi, lo, _ = _split(np.array([0.0, -0.0]))
    assert np.all(hi == 0) and np.all(lo == 0)
    assert np.signbit(hi[1])
    inside = np.array([2.0**-40, -(2.0**-40), np.nextafter(2.0**88, 0), -np.nextafter(2.0**88, 0), 1.0, -3.5])
    outside = np.array([0.0, -0.0, np.nextafter(2.0**-40, 0), 2.0**88, -(2.0**88), 1e-310, np.inf, -np.inf, np.nan,
                        2.0**-1022, 1e300])
    assert np.all(_range_word(inside) < WINDOW)
    assert np.all(_range_word(outside) >= WINDOW)


def test_split_products_stay_normal_and_finite_in_range():
    # |a| in [2^-40, 2^60) and |x| in [2^-40, 2^88): the smallest product's low part is a normal
    # float; the largest products overflow only above 2^128, which the kernels detect as Inf/NaN.
    smallest_product = 2.0**-80
    assert smallest_product * 2.0**-24 > np.finfo(np.float32).tiny
    assert 2.0**60 * 2.0**88 > np.finfo(np.float32).max
