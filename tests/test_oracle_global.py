"""Pins of the oracle's global (unchunked) Lorenzo mode.

Sec. IV-B ("Partial-Sum Lorenzo Reconstruction") proves that the Lorenzo recurrence
equals the N-D partial sum of the fused codes; the proof does not need chunks, so
with one chunk spanning the field the reconstruction must equal the full-field
cumulative sum along every axis.  Pinned against numpy's cumsum over the whole field,
against polynomial fields whose residuals vanish away from the field's own faces
(not the chunk faces), by the error bound, and against the chunked mode on shapes
that fit in one chunk (where the two modes coincide).
"""
import numpy as np
import pytest

from tests import _layout as LY


def _fused_q(orc, ar, shape):
    """q' in field order: q - r, or the outlier's delta."""
    sec = orc.sections(ar)
    h = sec["header"]
    codes = orc.decode_codes(ar, shape)
    slots = LY.slot_index(shape)
    qp = codes.astype(np.int64)[slots] - h["radius"]
    rec = sec["records"]
    kinds = rec[:, 0] & 1
    inv = np.full(codes.size, -1, dtype=np.int64)
    inv[slots.ravel()] = np.arange(int(np.prod(shape)))
    qp.ravel()[inv[(rec[:, 0] >> 1)[kinds == 0]]] = rec[:, 1][kinds == 0].view(np.int32)
    return qp, rec, kinds, inv, h


@pytest.mark.parametrize("shape", [(9000,), (70, 131), (19, 23, 37), (1, 1), (5,), (3, 2, 1), (40, 1, 33)])
def test_global_recurrence_equals_field_cumsum(orc, shape):
    rng = np.random.default_rng(7)
    x = np.cumsum(rng.standard_normal(shape).astype(np.float32), axis=-1).astype(np.float32)
    st, ar = orc.compress_ex(x, orc.EB_ABS, 2e-3, radius=16, global_lorenzo=True)  # small radius: outliers
    assert orc.parse_header(ar)["flags"] & orc.FLAG_GLOBAL
    qp, rec, kinds, inv, h = _fused_q(orc, ar, shape)
    k = qp
    for ax in range(len(shape)):
        k = np.cumsum(k, axis=ax)
    y_ref = (k.astype(np.float32) * np.float32(2 * np.float32(h["eb_f"]))).astype(np.float32).ravel()
    y_ref[inv[(rec[:, 0] >> 1)[kinds == 1]]] = rec[:, 1][kinds == 1].view(np.float32)
    st, y = orc.decompress(ar, x.size)
    assert st == 0
    assert np.array_equal(y.view(np.uint32), y_ref.view(np.uint32))
    assert np.abs(x.ravel().astype(np.float64) - y).max() <= h["eb_f"]


def _residuals(orc, x):
    """Global-mode residuals of an integer-valued field (eb 0.5: 2eb = 1, k = x)."""
    st, ar = orc.compress_ex(x, orc.EB_ABS, 0.5, global_lorenzo=True, select=orc.SEL_HUFF)
    assert st == 0
    qp, _, _, _, _ = _fused_q(orc, ar, x.shape)
    return qp


def test_global_polynomial_residuals(orc):
    # 1-D linear: residual is the slope after the first element, which is the value
    i = np.arange(5000)
    d = _residuals(orc, (5 + 3 * i).astype(np.float32))
    assert d[0] == 5 and np.all(d[1:] == 3)
    # 2-D planar: zero everywhere but the field's first row and column (chunk edges
    # at multiples of 16 no longer restart the prediction)
    ny, nx = 70, 90
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    f = (3 + 2 * x - 5 * y).astype(np.float32)
    d = _residuals(orc, f)
    assert np.all(d[1:, 1:] == 0)
    assert np.all(d[0, 1:] == 2) and np.all(d[1:, 0] == -5) and d[0, 0] == 3
    d = _residuals(orc, (x * y).astype(np.float32))  # mixed term: residual 1 inside
    assert np.all(d[1:, 1:] == 1)
    # 3-D trilinear
    nz, ny, nx = 20, 19, 21
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = (1 + 2 * x - 3 * y + 4 * z + x * y - 2 * y * z + 3 * x * z).astype(np.float32)
    d = _residuals(orc, f)
    assert np.all(d[1:, 1:, 1:] == 0)
    d = _residuals(orc, (x * y * z).astype(np.float32))
    assert np.all(d[1:, 1:, 1:] == 1)


@pytest.mark.parametrize("shape", [(200,), (16, 16), (8, 8, 8), (5, 7, 3)])
def test_global_equals_chunked_within_one_chunk(orc, shape):
    """A field no larger than one chunk has the same residuals in both modes: the
    archives differ only in the header's mode flag."""
    rng = np.random.default_rng(sum(shape))
    x = np.cumsum(rng.standard_normal(shape).astype(np.float32), axis=-1).astype(np.float32)
    st, a = orc.compress_ex(x, orc.EB_REL, 1e-3)
    st, g = orc.compress_ex(x, orc.EB_REL, 1e-3, global_lorenzo=True)
    assert a.size == g.size
    diff = np.nonzero(a != g)[0]
    assert list(diff) == [60]  # the flags word's low byte
    assert g[60] == a[60] | orc.FLAG_GLOBAL


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_global_error_bound_and_smaller_on_smooth_fields(orc, dtype):
    """The bound holds in global mode, and on a smooth field the archive is smaller
    than the chunked one (no restarts at chunk faces)."""
    y, x = np.meshgrid(np.linspace(0, 3, 300), np.linspace(0, 5, 400), indexing="ij")
    f = (np.sin(x) * np.cos(y) * 100 + 3 * x * y).astype(dtype)
    st, a = orc.compress_ex(f, orc.EB_REL, 1e-5)
    st, g = orc.compress_ex(f, orc.EB_REL, 1e-5, global_lorenzo=True)
    assert g.size < a.size
    if dtype == np.float64:
        st, yv = orc.decompress_f64(g, f.size)
        eb = orc.parse_header(g)["eb_d"]
    else:
        st, yv = orc.decompress(g, f.size)
        eb = orc.parse_header(g)["eb_f"]
    assert st == 0 and np.abs(f.ravel().astype(np.float64) - yv).max() <= eb
