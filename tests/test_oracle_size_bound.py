"""The lower bound on a Huffman block's size that the exhaustive pick relies on.

Every canonical Huffman code is at least one bit long, so a Huffman codec block of m
codes carries at least m bits of codes, i.e. at least m / 16 units in its two
interleaved streams, plus its 16-bit unit count: at least 2 + m / 8 bytes.  The GPU
encoder skips the Huffman size of a block when a run codec is already smaller than
that bound (the pick cannot be Huffman then).  Checked here on the oracle's exact
block sizes, on fields with full and edge blocks and with runs, noise and outliers.
"""
import numpy as np
import pytest


def _sizes(orc, x, eb, radius=512, mode=None):
    vmin, vmax = float(x.min()), float(x.max())
    st, _, ebf, x2, xr = orc.eb_params(orc.EB_REL if mode is None else mode, eb, vmin, vmax)
    assert st == 0
    c = orc.construct(x, ebf, x2, xr, radius)
    vh, lh, _ = orc.run_stats(c["codes"], x.shape, all_blocks=True)
    cl, vl, ll = orc.huffman_lengths(c["hist"]), orc.huffman_lengths(vh), orc.huffman_lengths(lh)
    return orc.block_sizes(c["codes"], x.shape, radius, cl, vl, ll, all_blocks=True)


def _field(shape, seed, zero=True):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(shape).astype(np.float32)
    for ax in range(len(shape)):
        x = np.cumsum(x, axis=ax).astype(np.float32)
    if zero:
        x[tuple(slice(0, s // 2) for s in shape)] = 0.0
    return x


@pytest.mark.parametrize("shape,eb,radius", [((64 * 4096,), 1e-3, 512), ((128, 192), 1e-2, 512),
                                             ((32, 48, 64), 1e-4, 512), ((32, 32, 32), 1e-3, 16)])
def test_huffman_size_at_least_two_plus_m_over_8_full_blocks(orc, shape, eb, radius):
    sizes = _sizes(orc, _field(shape, sum(shape)), eb, radius)
    m = 4096  # every block of these shapes is full
    assert sizes.shape[0] > 1
    assert int(sizes[:, 0].min()) >= 2 + m / 8


def test_huffman_size_bound_is_reached_by_one_bit_codes(orc):
    """An all-zero field gives one symbol, coded in one bit: each 32-lane stream of
    2048 codes is 128 units, so a block is 2 + 2 * 256 = 514 bytes, 516 with the
    4-byte padding -- the bound, up to that padding."""
    x = np.zeros((48, 64, 64), dtype=np.float32)
    sizes = _sizes(orc, x, 0.1, mode=orc.EB_ABS)
    assert sizes.shape[0] == 3 * 4 * 4
    assert np.all(sizes[:, 0] == 516)


def test_huffman_size_bound_on_an_edge_block(orc):
    n = 5 * 4096 + 777  # the last block holds 777 codes
    sizes = _sizes(orc, _field((n,), 7, zero=False), 1e-3)
    assert sizes.shape[0] == 6
    for b in range(6):
        m = 4096 if b < 5 else 777
        assert int(sizes[b, 0]) >= 2 + m / 8, (b, int(sizes[b, 0]))
