"""Pins of the oracle's double-precision input path.

The paper's kernels take FP32; double-precision datasets (Sec. II-B, Sec. V-A) are
read here as the same method with prequantization in double: step = 2 eb (1 - 2^-24),
k = nearest integer to x / step, x' = fl64(k * step).  Pinned by the error bound on
every element (decided exactly, with rationals, wherever the double difference is
near the bound), by adversarial values at the half points of both the exact and the
shrunk step, by Lorenzo residuals on planar fields, and by the guards.
"""
from fractions import Fraction

import numpy as np
import pytest


def _assert_bound_exact(x, y, eb):
    """|x - y| <= eb for every element, exactly."""
    d = np.abs(x - y)
    assert np.all(d <= eb * (1 + 1e-9))
    near = np.nonzero(d >= eb * (1 - 1e-9))[0]
    for i in near:
        assert abs(Fraction(float(x.flat[i])) - Fraction(float(y.flat[i]))) <= Fraction(eb), i


def _fields(rng):
    yield rng.standard_normal(7000).cumsum()
    yield rng.standard_normal((70, 131)).cumsum(0).cumsum(1) * 1e3
    yield rng.standard_normal((19, 23, 37)).cumsum(2) * 1e-3
    yield np.exp(rng.standard_normal((17, 17, 40)) * 3.0)


@pytest.mark.parametrize("eb", [1e-2, 1e-4, 1e-6])
@pytest.mark.parametrize("sel", [0, 2, 4])
def test_f64_error_bound_every_element(orc, eb, sel):
    rng = np.random.default_rng(int(1 / eb) + sel)
    for x in _fields(rng):
        st, ar = orc.compress_f64(x, orc.EB_REL, eb, select=sel)
        assert st == 0
        h = orc.parse_header(ar)
        assert h["flags"] & orc.FLAG_F64 and h["n_patch"] == 0
        assert h["eb_d"] == eb * (float(x.max()) - float(x.min()))
        st, y = orc.decompress_f64(ar, x.size)
        assert st == 0
        _assert_bound_exact(x.ravel(), y, h["eb_d"])


def test_f64_finer_than_fp32_can_hold(orc):
    """A bound FP32 cannot hold around these values: 1e-5 absolute on a field of
    magnitude ~1e3, where FP32's spacing is 6.1e-5 (x / step stays below the 2^27
    guard: 1000 / 2e-5 = 5e7)."""
    rng = np.random.default_rng(5)
    x = 1000.0 + rng.standard_normal(20000).cumsum() * 1e-3
    st, ar = orc.compress_f64(x, orc.EB_ABS, 1e-5)
    assert st == 0
    st, y = orc.decompress_f64(ar, x.size)
    _assert_bound_exact(x, y, 1e-5)
    assert np.abs(x.astype(np.float32).astype(np.float64) - x).max() > 1e-5  # FP32 alone would miss it


def test_f64_half_points(orc):
    """Values at and next to the half points of the exact step 2eb and of the shrunk
    step, across magnitudes up to the 2^27 guard: every one meets the bound exactly
    and none is refused (no verbatim patches exist for doubles)."""
    eb = 0.37
    st, eb_d, step, rstep = orc.eb_params_f64(orc.EB_ABS, eb)
    assert st == 0 and eb_d == eb
    assert step == (2 * eb) * (1 - 2.0 ** -24) and rstep == 1 / step
    vals = []
    for k in [0, 1, 2, 3, 1000, 12345, 2 ** 20 + 7, 2 ** 26 - 5, -1, -777, -(2 ** 26) + 3]:
        for base in (Fraction(2 * eb), Fraction(step)):
            c = float((Fraction(k) + Fraction(1, 2)) * base)
            for u in range(-3, 4):
                v = c
                for _ in range(abs(u)):
                    v = np.nextafter(v, np.inf if u > 0 else -np.inf)
                vals.append(float(v))
    for v in vals:
        st, k = orc.prequant_f64(v, eb_d, step, rstep)
        assert st == 0, v
        assert abs(Fraction(v) - Fraction(float(np.float64(k) * step))) <= Fraction(eb_d), v
    x = np.array(vals)
    st, ar = orc.compress_f64(x, orc.EB_ABS, eb)
    assert st == 0
    st, y = orc.decompress_f64(ar, x.size)
    _assert_bound_exact(x, y, eb)


def test_f64_planar_field_zero_residuals(orc):
    """A planar double field on the quantization lattice has k = a + b y + c x exactly,
    so the 2-D Lorenzo residual is zero away from the chunks' first row and column
    (Sec. IV-B2 predictor), as in the FP32 path."""
    eb = 0.01
    st, eb_d, step, rstep = orc.eb_params_f64(orc.EB_ABS, eb)
    yy, xx = np.mgrid[0:48, 0:80]
    k = 5 + 3 * yy - 2 * xx
    x = k.astype(np.float64) * step
    st, ar = orc.compress_f64(x, orc.EB_ABS, eb, select=orc.SEL_HUFF)
    assert st == 0
    nblk, _ = orc.geometry(x.shape)
    codes = np.zeros(nblk * 4096, np.uint16)
    assert orc.lib().orc_decode_codes(orc._p(ar, orc._u8p), ar.size, orc._p(codes, orc._u16p), codes.size) == 0
    # block (0, 0) is 48 rows x 64 columns, row-major inside the block
    blk = codes[:48 * 64].reshape(48, 64).astype(np.int64) - 512
    inner = np.ones((48, 64), bool)
    inner[::16, :] = False
    inner[:, ::16] = False
    assert np.all(blk[inner] == 0)
    assert np.all(blk[0, 1:16] == -2) and np.all(blk[1:16, 0] == 3)  # one-sided differences at chunk edges
    st, y = orc.decompress_f64(ar, x.size)
    assert np.array_equal(y.reshape(x.shape), x)


def test_f64_guards_and_type_checks(orc):
    st, _ = orc.compress_f64(np.array([1.0, np.nan, 2.0]), orc.EB_ABS, 0.1, raise_on_error=False)
    assert st == orc.E_NONFINITE
    st, _ = orc.compress_f64(np.array([0.0, 2.0 ** 27 * 0.2 * 1.01]), orc.EB_ABS, 0.1, raise_on_error=False)
    assert st == orc.E_RANGE
    st, _ = orc.compress_f64(np.full(100, 3.0), orc.EB_REL, 1e-3, raise_on_error=False)
    assert st == orc.E_ARG  # zero value range: no relative bound
    x = np.linspace(0, 1, 5000)
    st, ar64 = orc.compress_f64(x, orc.EB_ABS, 1e-4)
    st, ar32 = orc.compress(x.astype(np.float32), orc.EB_ABS, 1e-4)
    assert orc.decompress(ar64, x.size, raise_on_error=False)[0] == orc.E_ARG
    assert orc.decompress_f64(ar32, x.size, raise_on_error=False)[0] == orc.E_ARG
    # a double archive claiming a verbatim patch is corrupt
    bad = ar64.copy()
    bad[88] = 1
    bad[72] = (int(bad[72]) + 1) % 256
    assert orc.decompress_f64(bad, x.size, raise_on_error=False)[0] == orc.E_CORRUPT
