"""Edge cases and damaged archives for the CPU oracle (host-only fault tests)."""
import numpy as np
import pytest


def test_nonfinite_inputs(orc):
    x = np.ones((10, 10), np.float32)
    x[3, 4] = np.nan
    assert orc.compress(x, orc.EB_REL, 1e-3, raise_on_error=False)[0] == orc.E_NONFINITE
    assert orc.compress(x, orc.EB_ABS, 1e-3, raise_on_error=False)[0] == orc.E_NONFINITE
    x[3, 4] = np.inf
    assert orc.compress(x, orc.EB_ABS, 1e-3, raise_on_error=False)[0] == orc.E_NONFINITE


def test_degenerate_bounds(orc):
    x = np.full(100, 3.0, np.float32)
    assert orc.compress(x, orc.EB_REL, 1e-3, raise_on_error=False)[0] == orc.E_ARG  # zero range
    st, ar = orc.compress(x, orc.EB_ABS, 1e-3)
    assert orc.decompress(ar, x.size)[1].tolist() == pytest.approx(x.tolist(), abs=1e-3)
    for eb in (0.0, -1.0, float("nan"), float("inf")):
        assert orc.compress(x, orc.EB_ABS, eb, raise_on_error=False)[0] == orc.E_ARG
    assert orc.compress(x, orc.EB_ABS, 1e-3, radius=0, raise_on_error=False)[0] == orc.E_ARG
    assert orc.compress(x, orc.EB_ABS, 1e-3, radius=513, raise_on_error=False)[0] == orc.E_ARG
    assert orc.compress(x, orc.EB_ABS, 1e-3, select=9, raise_on_error=False)[0] == orc.E_ARG
    assert orc.compress(x, orc.EB_ABS, 1e-3, select=orc.SEL_LEARNED, raise_on_error=False)[0] == orc.E_ARG


def test_prequant_range_guard(orc):
    x = np.array([0.0, 1e7, 0.0], np.float32)
    assert orc.compress(x, orc.EB_ABS, 0.5, raise_on_error=False)[0] == orc.E_RANGE
    x = np.array([0.0, 8e6, 0.0], np.float32)
    assert orc.compress(x, orc.EB_ABS, 0.5, raise_on_error=False)[0] == orc.OK


def test_empty_and_oversized_shapes(orc):
    assert orc.geometry((4096,)) == (1, 4096)
    with pytest.raises(Exception):
        orc.geometry((0,))
    with pytest.raises(Exception):
        orc.geometry((1 << 31,))
    with pytest.raises(Exception):
        orc.geometry((2048, 1024, 1024))  # 2^19 blocks of 16^3: slots overflow 2^31
    assert orc.geometry((2048, 1024, 1008))[0] < (1 << 19)


@pytest.mark.parametrize("shape", [(1,), (2,), (1, 1), (1, 1, 1), (7,), (4097,), (65, 1), (1, 65),
                                   (17, 31, 5), (3, 129, 67), (64, 64), (16, 16, 16), (8191,)])
def test_tiny_and_ragged_shapes(orc, shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.standard_normal(shape).astype(np.float32).cumsum(axis=-1).astype(np.float32)
    for sel in range(5):
        st, ar = orc.compress(x, orc.EB_ABS, 1e-2, select=sel)
        st, y = orc.decompress(ar, x.size)
        assert np.abs(x.ravel().astype(np.float64) - y).max() <= orc.parse_header(ar)["eb_f"]


def test_decompress_capacity(orc):
    x = np.arange(100, dtype=np.float32)
    st, ar = orc.compress(x, orc.EB_ABS, 0.1)
    st, _ = orc.decompress(ar, 99, raise_on_error=False)
    assert st == orc.E_CAPACITY


def _archives(orc):
    rng = np.random.default_rng(8)
    x = rng.standard_normal((90, 140)).astype(np.float32).cumsum(1)
    x[20:60, :] = 0
    for sel in (0, 1, 2, 4):
        yield x, orc.compress(x, orc.EB_REL, 1e-2, radius=64, select=sel)[1]


def test_truncated_archives_rejected(orc):
    for x, ar in _archives(orc):
        for cut in (0, 10, 127, 128, ar.size // 2, ar.size - 1):
            st, _ = orc.decompress(ar[:cut], x.size, raise_on_error=False)
            assert st == orc.E_CORRUPT


def test_header_damage_rejected(orc):
    for x, ar in _archives(orc):
        for off, val in [(0, 0x00), (4, 9), (6, 4), (7, 5), (52, 0), (56, 7), (60, 16), (64, 3)]:
            bad = ar.copy()
            bad[off] = val
            st, _ = orc.decompress(bad, x.size, raise_on_error=False)
            assert st == orc.E_CORRUPT, off


def test_random_bit_flips_never_crash(orc):
    rng = np.random.default_rng(77)
    for x, ar in _archives(orc):
        for _ in range(150):
            bad = ar.copy()
            i = int(rng.integers(0, bad.size))
            bad[i] ^= np.uint8(1 << int(rng.integers(0, 8)))
            st, y = orc.decompress(bad, x.size, raise_on_error=False)
            assert st in (orc.OK, orc.E_CORRUPT)
