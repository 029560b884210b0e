"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than its own formulas:
the error bound (Sec. IV-A1), the partial-sum identity of the reconstruction
(Sec. IV-B2 proof), closed forms of the Lorenzo residual on polynomial fields,
the paper's run-length example (Sec. III-B), brute-force optimal Huffman costs,
Kraft's equality, the redundancy bounds quoted in Sec. III-B1, and a textbook
Huffman instance.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from tests import _layout as LY

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _fields(rng):
    yield rng.standard_normal(5000).astype(np.float32).cumsum()
    yield rng.standard_normal((70, 131)).astype(np.float32).cumsum(0).cumsum(1)
    yield rng.standard_normal((19, 23, 37)).astype(np.float32).cumsum(2)
    yield (rng.standard_normal((33, 65)) * 1e3).astype(np.float32)
    yield np.exp(rng.standard_normal((17, 17, 40))).astype(np.float32)


# ---------------------------------------------------------------------------------
# error bound: |x - x'| <= eb on every element (Sec. IV-A1 prequantization)
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("eb", [1e-2, 1e-3, 1e-4])
@pytest.mark.parametrize("sel", [0, 1, 2, 3, 4])
def test_error_bound_every_element(orc, eb, sel):
    rng = np.random.default_rng(11)
    for x in _fields(rng):
        st, ar = orc.compress(x, orc.EB_REL, eb, select=sel)
        assert st == 0
        h = orc.parse_header(ar)
        st, y = orc.decompress(ar, x.size)
        assert st == 0
        err = np.abs(x.ravel().astype(np.float64) - y.astype(np.float64))
        assert err.max() <= h["eb_f"], (err.max(), h["eb_f"])
        # eb_f is the largest float not above eb * range
        rng_d = float(x.max()) - float(x.min())
        assert h["eb_f"] <= eb * rng_d
        assert float(np.nextafter(np.float32(h["eb_f"]), np.float32(np.inf))) > eb * rng_d


def test_error_bound_absolute_and_small_radius(orc):
    rng = np.random.default_rng(5)
    x = (rng.standard_normal((40, 50)) * 10).astype(np.float32)
    for r in (1, 2, 7, 512):
        st, ar = orc.compress(x, orc.EB_ABS, 0.01, radius=r)
        st, y = orc.decompress(ar, x.size)
        h = orc.parse_header(ar)
        assert np.abs(x.ravel().astype(np.float64) - y).max() <= h["eb_f"]
        if r <= 2:
            assert h["n_out"] > 0  # rough data at tiny radius must produce outliers


def test_prequant_near_half_points_and_patches(orc):
    """Values placed on the rounding boundary at large |k| stress the FP32 fix-up;
    every reconstruction still meets the bound, through a verbatim patch if needed."""
    eb = np.float32(0.0123456789)
    st, ebd, ebf, x2, xr = orc.eb_params(orc.EB_ABS, float(eb))
    assert st == 0
    ks = np.array([1, 2, 3, 1000, 12345, 654321, 3000000, 7000000], dtype=np.float64)
    vals = []
    for k in ks:
        mid = (k + 0.5) * float(x2)
        m32 = np.float32(mid)
        for d in range(-4, 5):
            v = m32
            for _ in range(abs(d)):
                v = np.nextafter(v, np.float32(np.inf if d > 0 else -np.inf))
            vals.extend([v, -v])
    x = np.array(vals, dtype=np.float32)
    patches = 0
    for v in x:
        st, k, p = orc.prequant(float(v), ebf, x2, xr)
        assert st == 0
        rec = np.float32(np.float32(k) * np.float32(x2))
        if p:
            patches += 1
        else:
            assert abs(float(v) - float(rec)) <= ebf
    st, ar = orc.compress(x, orc.EB_ABS, float(eb))
    st, y = orc.decompress(ar, x.size)
    assert np.abs(x.astype(np.float64) - y).max() <= orc.parse_header(ar)["eb_f"]
    assert orc.parse_header(ar)["n_patch"] == patches
    assert patches > 0  # the large-k half points cannot all be met by rounding alone


# ---------------------------------------------------------------------------------
# reconstruction = N-D partial sum of q' per chunk (Sec. IV-B2), equal to the
# oracle's sequential recurrence
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(9000,), (70, 131), (19, 23, 37), (1, 1), (5,), (3, 2, 1)])
def test_recurrence_equals_partial_sum(orc, shape):
    rng = np.random.default_rng(3)
    x = rng.standard_normal(shape).astype(np.float32)
    x = np.cumsum(x, axis=-1).astype(np.float32)
    st, ar = orc.compress(x, orc.EB_ABS, 2e-3, radius=16)  # small radius: outliers
    sec = orc.sections(ar)
    h = sec["header"]
    codes = orc.decode_codes(ar, shape)
    slots = LY.slot_index(shape)
    qp = codes.astype(np.int64)[slots] - h["radius"]
    rec = sec["records"]
    kinds = rec[:, 0] & 1
    out_slots = (rec[:, 0] >> 1)[kinds == 0]
    out_vals = rec[:, 1][kinds == 0].view(np.int32)
    inv = np.full(codes.size, -1, dtype=np.int64)
    inv[slots.ravel()] = np.arange(x.size)
    qp.ravel()[inv[out_slots]] = out_vals
    k = LY.chunk_cumsum(qp, shape)
    y_ref = (k.astype(np.float32) * np.float32(2 * np.float32(h["eb_f"]))).astype(np.float32).ravel()
    p_slots = (rec[:, 0] >> 1)[kinds == 1]
    y_ref[inv[p_slots]] = rec[:, 1][kinds == 1].view(np.float32)
    st, y = orc.decompress(ar, x.size)
    assert np.array_equal(y.view(np.uint32), y_ref.view(np.uint32))


# ---------------------------------------------------------------------------------
# Lorenzo residuals on polynomial fields (Sec. IV-B2 predictors): with eb = 0.5
# (2eb = 1) integer-valued fields prequantize exactly, and the residual is the
# mixed difference of the field inside each chunk.
# ---------------------------------------------------------------------------------
def _codes_field(orc, x, radius=512):
    st, ebd, ebf, x2, xr = orc.eb_params(orc.EB_ABS, 0.5)
    assert (ebf, x2, xr) == (0.5, 1.0, 1.0)
    c = orc.construct(x, ebf, x2, xr, radius)
    slots = LY.slot_index(x.shape)
    q = c["codes"].astype(np.int64) - radius
    out = (c["keys"] & 1) == 0
    q[c["keys"][out] >> 1] = c["vals"][out].view(np.int32)  # outliers carry delta itself
    assert np.all(c["codes"][c["keys"][out] >> 1] == 0)
    return q[slots], c


def test_lorenzo_1d_constant_and_linear(orc):
    n = 1000
    i = np.arange(n)
    start = LY.chunk_start_mask((n,))[2]
    d, _ = _codes_field(orc, np.full(n, 7.0, np.float32))
    assert np.all(d[~start] == 0) and np.all(d[start] == 7)
    d, _ = _codes_field(orc, (5 + 3 * i).astype(np.float32))
    # 1-D linear: the residual is the slope, not zero
    assert np.all(d[~start] == 3)
    assert np.array_equal(d[start], (5 + 3 * i)[start])


def test_lorenzo_2d_planar_and_separable(orc):
    ny, nx = 70, 90
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    _, sy, sx = LY.chunk_start_mask((ny, nx))
    inner = ~sy & ~sx
    f = (3 + 2 * x - 5 * y).astype(np.float32)
    d, _ = _codes_field(orc, f)
    assert np.all(d[inner] == 0)
    assert np.all(d[sy & ~sx] == 2)      # first row of a chunk: x-difference
    assert np.all(d[sx & ~sy] == -5)     # first column: y-difference
    assert np.array_equal(d[sx & sy], f[sx & sy].astype(np.int64))
    g = ((x % 7) * 3 + (y * y) % 11).astype(np.float32)  # g(x) + h(y)
    d, _ = _codes_field(orc, g)
    assert np.all(d[inner] == 0)
    h = (x * y).astype(np.float32)  # mixed term: residual is its mixed difference, 1
    d, _ = _codes_field(orc, h)
    assert np.all(d[inner] == 1)


def test_lorenzo_3d_trilinear(orc):
    nz, ny, nx = 20, 19, 21
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    sz, sy, sx = LY.chunk_start_mask((nz, ny, nx))
    inner = ~sz & ~sy & ~sx
    f = (1 + 2 * x - 3 * y + 4 * z + x * y - 2 * y * z + 3 * x * z).astype(np.float32)
    d, _ = _codes_field(orc, f, radius=512)
    assert np.all(d[inner] == 0)
    d, _ = _codes_field(orc, (x * y * z).astype(np.float32))
    assert np.all(d[inner] == 1)


def test_outlier_keeps_delta(orc):
    """Modified quantization (Sec. IV-B1): an out-of-range delta is stored as the
    outlier itself and its code is 0."""
    x = np.zeros(300, np.float32)
    x[10] = 2000.0
    st, ebd, ebf, x2, xr = orc.eb_params(orc.EB_ABS, 0.5)
    c = orc.construct(x, ebf, x2, xr, 512)
    assert list(c["keys"]) == [20, 22]  # slots 10 and 11, kind 0
    assert list(c["vals"].view(np.int32)) == [2000, -2000]
    assert c["codes"][10] == 0 and c["codes"][11] == 0 and c["codes"][12] == 512


# ---------------------------------------------------------------------------------
# run-length encoding: the paper's worked example (Sec. III-B)
# ---------------------------------------------------------------------------------
def test_rle_worked_example(orc):
    g = json.load(open(os.path.join(GOLDEN, "rle_worked_example.json")))
    letters = {"a": 513, "b": 510, "c": 512}  # codes r+1, r-2, r (radius 512)
    seq = [letters[ch] for ch in g["sequence"]]
    delta = np.array(seq) - 512
    x = np.cumsum(delta).astype(np.float32)  # 1-D Lorenzo residuals equal delta
    st, ar = orc.compress(x, orc.EB_ABS, 0.5, select=orc.SEL_RLE)
    sec = orc.sections(ar)
    p = sec["payload"].view(np.uint16)
    nr = len(g["runs"])
    assert sec["blk_bytes"][0] == 4 * nr
    assert list(p[:nr]) == [letters[v] for v, _ in g["runs"]]
    assert list(p[nr:2 * nr]) == [n for _, n in g["runs"]]
    st, y = orc.decompress(ar, x.size)
    assert np.array_equal(y, x)


# ---------------------------------------------------------------------------------
# Huffman code lengths: optimality by brute force, Kraft, textbook instance,
# redundancy bounds of Sec. III-B1
# ---------------------------------------------------------------------------------
def _brute_min_cost(freq):
    k = len(freq)
    best = None
    for lens in itertools.product(range(1, k), repeat=k):
        if sum(2.0 ** -l for l in lens) <= 1.0 + 1e-12:
            c = sum(f * l for f, l in zip(freq, lens))
            best = c if best is None or c < best else best
    return best


@pytest.mark.parametrize("seed", range(12))
def test_huffman_brute_force_optimal(orc, seed):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(2, 7 if seed < 10 else 8))
    freq = rng.integers(1, 50, size=k).astype(np.uint32)
    if seed % 3 == 0:
        freq[: k // 2] = freq[0]  # ties
    full = np.zeros(1024, np.uint32)
    pos = rng.choice(1024, size=k, replace=False)
    full[pos] = freq
    ln = orc.huffman_lengths(full)
    assert np.count_nonzero(ln) == k
    cost = int((ln[pos].astype(np.int64) * freq).sum())
    assert cost == _brute_min_cost(list(map(int, freq)))
    assert sum(2.0 ** -int(l) for l in ln[pos]) == 1.0  # Kraft equality (full tree)


def test_huffman_textbook(orc):
    g = json.load(open(os.path.join(GOLDEN, "huffman_textbook.json")))
    syms = sorted(g["freq"])
    full = np.zeros(16, np.uint32)
    for i, s in enumerate(syms):
        full[i] = g["freq"][s]
    ln = orc.huffman_lengths(full)
    for i, s in enumerate(syms):
        assert ln[i] == g["lengths"][s]
    assert int((ln[: len(syms)].astype(int) * full[: len(syms)]).sum()) == g["cost"]


def test_huffman_single_and_empty(orc):
    f = np.zeros(1024, np.uint32)
    assert not orc.huffman_lengths(f).any()
    f[77] = 5
    ln = orc.huffman_lengths(f)
    assert ln[77] == 1 and ln.sum() == 1


@pytest.mark.parametrize("seed", range(20))
def test_huffman_redundancy_bounds(orc, seed):
    """R = <b> - H: R <= p1 + 0.086 (Gallager), and R >= 1 - H(p1,1-p1) when
    p1 > 0.4 (Sec. III-B1)."""
    rng = np.random.default_rng(100 + seed)
    k = int(rng.integers(2, 300))
    f = rng.geometric(rng.uniform(0.05, 0.9), size=k).astype(np.float64) ** rng.uniform(0.5, 3)
    if seed % 2:
        f[0] *= rng.uniform(2, 200)
    f = np.maximum(1, np.round(f * 50)).astype(np.uint32)
    full = np.zeros(1024, np.uint32)
    full[:k] = f
    ln = orc.huffman_lengths(full)[:k].astype(np.float64)
    p = f / f.sum()
    H = -(p * np.log2(p)).sum()
    avg = (p * ln).sum()
    R = avg - H
    p1 = p.max()
    assert R >= -1e-12
    assert R <= p1 + 0.086 + 1e-9
    if p1 > 0.4:
        Hb = -(p1 * math.log2(p1) + (1 - p1) * math.log2(1 - p1)) if p1 < 1 else 0.0
        assert R >= 1 - Hb - 1e-9


def test_canonical_codes_prefix_free(orc):
    rng = np.random.default_rng(9)
    f = np.zeros(4096, np.uint32)
    idx = rng.choice(4096, 400, replace=False)
    f[idx] = rng.integers(1, 10000, 400)
    ln = orc.huffman_lengths(f)
    code = orc.canonical_codes(ln)
    words = sorted((int(ln[s]), int(s)) for s in np.nonzero(ln)[0])
    strs = [format(int(code[s]), "0%db" % l) for l, s in words]
    # canonical: ordered by (length, symbol) means codes increase as integers
    # left-aligned at the max length
    L = max(l for l, _ in words)
    vals = [int(code[s]) << (L - l) for l, s in words]
    assert vals == sorted(vals) and len(set(vals)) == len(vals)
    for a, b in zip(strs, strs[1:]):
        assert not b.startswith(a)
    # all codes distinct and prefix-free overall
    ss = sorted(strs)
    for a, b in zip(ss, ss[1:]):
        assert not b.startswith(a)


def test_huffman_only_cr_at_most_32(orc):
    """At least one bit per symbol, so Huffman-only CR <= 32 for FP32 (Sec. II-B1)."""
    x = np.zeros((128, 128), np.float32)
    st, ar = orc.compress(x, orc.EB_ABS, 1.0, select=orc.SEL_HUFF)
    sec = orc.sections(ar)
    assert sec["header"]["payload"] * 8 >= x.size
    st, ar2 = orc.compress(x, orc.EB_ABS, 1.0, select=orc.SEL_EXHAUSTIVE)
    assert ar2.size < ar.size  # runs beat the 1-bit floor on a constant field


# ---------------------------------------------------------------------------------
# lossless coding round trips: every codec reproduces the quant-codes exactly
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("sel", [0, 1, 2, 3, 4])
def test_codec_round_trip_codes(orc, sel):
    rng = np.random.default_rng(21)
    for x in _fields(rng):
        st, ar = orc.compress(x, orc.EB_REL, 1e-3, select=sel)
        h = orc.parse_header(ar)
        st, ebd, ebf, x2, xr = orc.eb_params(orc.EB_REL, 1e-3, float(x.min()), float(x.max()))
        c = orc.construct(x, ebf, x2, xr)
        dec = orc.decode_codes(ar, x.shape)
        assert np.array_equal(dec, c["codes"])
        sec = orc.sections(ar)
        assert np.array_equal(sec["records"][:, 0], c["keys"])
        if sel <= 2:
            assert h["n_codec"][sel] == h["nblk"]


def test_exhaustive_is_minimal(orc):
    rng = np.random.default_rng(4)
    x = rng.standard_normal((200, 300)).astype(np.float32).cumsum(1)
    x[50:120, :] = 0.0
    sizes = []
    for sel in range(5):
        st, ar = orc.compress(x, orc.EB_REL, 1e-2, select=sel)
        sizes.append(orc.parse_header(ar)["payload"])
    assert sizes[4] <= min(sizes[:3])
    st, ar = orc.compress(x, orc.EB_REL, 1e-2, select=4)
    h = orc.parse_header(ar)
    assert h["n_codec"][0] > 0 and (h["n_codec"][1] + h["n_codec"][2]) > 0


# ---------------------------------------------------------------------------------
# selector pieces: fixed-point log2, heuristic on clear-cut histograms, features
# ---------------------------------------------------------------------------------
def test_log2_q16(orc):
    for v in [1, 2, 3, 5, 7, 10, 100, 1000, 4095, 4096, 65535, 1 << 20, 123456789, (1 << 32) - 1]:
        got = orc.log2_q16(v) / 65536.0
        assert abs(got - math.log2(v)) <= 2.0 / 65536.0


def test_heuristic_clear_cases(orc):
    h = np.zeros(1024, np.uint32)
    h[512] = 4096
    assert orc.heuristic_pick(h, 4096) == orc.CODEC_RLE_HUFF  # H=0, R-=1 -> 1.0
    h[:] = 0
    h[500:516] = 256
    assert orc.heuristic_pick(h, 4096) == orc.CODEC_HUFF  # H = 4 bits
    rng = np.random.default_rng(0)
    for _ in range(200):
        h = np.zeros(1024, np.uint32)
        k = int(rng.integers(1, 40))
        h[rng.choice(1024, k, replace=False)] = rng.integers(1, 400, k)
        m = int(h.sum())
        p = h[h > 0] / m
        H = -(p * np.log2(p)).sum()
        p1 = p.max()
        R = 1 + p1 * math.log2(p1) + ((1 - p1) * math.log2(1 - p1) if p1 < 1 else 0) if p1 > 0.4 else 0.0
        est = H + max(R, 0)
        if abs(est - 1.09) > 1e-3:
            want = orc.CODEC_RLE_HUFF if est <= 1.09 else orc.CODEC_HUFF
            assert orc.heuristic_pick(h, m) == want


def test_features_special_cases(orc):
    x = np.zeros(4096, np.float32)
    st, ebd, ebf, x2, xr = orc.eb_params(orc.EB_ABS, 0.5)
    c = orc.construct(x, ebf, x2, xr)
    f = orc.block_features(c["codes"], (4096,))
    assert np.allclose(f[0], [1, 0, 1, 0, 1 / 4096, 0, 0, 0])
    rng = np.random.default_rng(2)
    x = rng.integers(-300, 300, 4096).astype(np.float32)
    c = orc.construct(x, ebf, x2, xr)
    f = orc.block_features(c["codes"], (4096,))[0]
    codes = c["codes"][:4096].astype(np.int64)
    assert f[5] == np.float32(np.count_nonzero(codes == 0)) / np.float32(4096)
    assert f[4] == np.float32(1 + np.count_nonzero(codes[1:] != codes[:-1])) / np.float32(4096)
    hst = np.bincount(codes, minlength=1024)
    p = hst[hst > 0] / 4096
    assert abs(f[1] - (-(p * np.log2(p)).sum())) < 1e-3


def _mado_d(i):
    """Madogram pair distance of position i: 1, 26, ..., 176 (every 25th distance of
    the paper's 1..200, Sec. III-B) by i mod 8."""
    return 1 + 25 * (i % 8)


def _hand_block(r=512):
    """A 4096-code block built by hand: a run of 1000 zero residuals, a run of 100
    outliers (code 0), then a period-8 pattern of residuals -3..4, with |delta| = 300
    at position 2000 and the largest in-range |delta| = r - 1 at position 3000."""
    c = [r] * 1000 + [0] * 100 + [r + (i % 8) - 3 for i in range(1100, 4096)]
    c[2000] = r + 300
    c[3000] = r - (r - 1)
    return c


def test_features_hand_computed_block(orc):
    """All 8 selector features on a block with outliers, runs, known |delta| values and
    a period-8 pattern, against counts written out here from the definitions
    (Sec. III-B: p1, entropy, runs, and the binary-variance madogram)."""
    r, m = 512, 4096
    c = _hand_block(r)
    f = orc.block_features(np.array(c, np.uint16), (m,), r)[0]
    # zero residuals: the first run, plus the pattern's delta = 0 positions (i % 8 == 3);
    # 2000 and 3000 are both 0 mod 8, so neither removes one
    zero = 1000 + sum(1 for i in range(1100, 4096) if i % 8 == 3)
    outl = 100
    deltas = [abs(v - r) for v in c if v != 0]
    absd = sum(deltas)
    assert max(deltas) == r - 1 and len(deltas) == m - outl
    runs = 1 + sum(1 for i in range(1, m) if c[i] != c[i - 1])
    counts = {}
    for v in c:
        counts[v] = counts.get(v, 0) + 1
    pairs = [i for i in range(m) if i + _mado_d(i) < m]
    mism = sum(1 for i in pairs if c[i] != c[i + _mado_d(i)])
    pairs = len(pairs)
    assert f[0] == np.float32(zero) / np.float32(m)
    assert f[2] == np.float32(max(counts.values())) / np.float32(m)
    assert max(counts, key=counts.get) == r  # the zero residual is the top code
    assert f[3] == np.float32(9.0)           # log2(1 + 511), exact in Q16
    assert f[4] == np.float32(runs) / np.float32(m)
    assert f[5] == np.float32(outl) / np.float32(m)
    assert f[6] == np.float32(absd) / np.float32(m * r)  # outliers count 0, denominator m r
    assert f[7] == np.float32(mism) / np.float32(pairs)
    p = np.array(list(counts.values()), np.float64) / m
    assert abs(f[1] - float(-(p * np.log2(p)).sum())) < 1e-3


def test_features_closed_forms(orc):
    """Closed forms: in a pure period-8 block every sampled pair differs except those
    at distance 176 (a multiple of 8, taken by positions 7 mod 8): 7/8 of the pairs,
    whose count is 4096 - 8 = 4088 less the tail of each distance class; a block
    shorter than a distance has no pairs at it; log2(1 + max|delta|) is log2(5) for
    max |delta| = 4."""
    r, m = 512, 4096
    c = np.array([r + (i % 8) - 3 for i in range(m)], np.uint16)
    f = orc.block_features(c, (m,), r)[0]
    # class k (positions k mod 8) has (m - d_k - k + 7) // 8 pairs, d_k = 1 + 25 k
    per_class = [(m - (1 + 25 * k) - k + 7) // 8 for k in range(8)]
    assert f[7] == np.float32(sum(per_class[:7])) / np.float32(sum(per_class))
    assert abs(f[3] - math.log2(5)) < 2 ** -15
    assert f[4] == 1.0  # every element starts a run
    assert f[0] == np.float32(m // 8) / np.float32(m)
    # a 40-element 1-D field alternating two codes: only distances 1 (positions
    # 0, 8, ..., 32: 5 pairs, all differing) and 26 (positions 1, 9: 2 pairs, equal
    # codes since 26 is even) fit inside it
    c = np.array([r + (i % 2) for i in range(40)], np.uint16)
    f = orc.block_features(c, (40,), r)[0]
    assert f[7] == np.float32(5) / np.float32(7)
    assert f[3] == np.float32(1.0)  # log2(1 + 1)


# ---------------------------------------------------------------------------------
# MLP: FP32 forward close to a float64 forward; analytic gradient = finite differences
# ---------------------------------------------------------------------------------
def test_mlp_forward_and_gradient(orc):
    rng = np.random.default_rng(1)
    w = (rng.standard_normal(orc.MLP_PARAMS) * 0.3).astype(np.float32)
    feat = rng.random((64, 8)).astype(np.float32)
    tgt = rng.random((64, 3)).astype(np.float32) * 10
    y = orc.mlp_forward(w, feat)
    W1 = w[:256].reshape(32, 8).astype(np.float64)
    b1 = w[256:288]
    W2 = w[288:1312].reshape(32, 32).astype(np.float64)
    b2 = w[1312:1344]
    W3 = w[1344:1440].reshape(3, 32).astype(np.float64)
    b3 = w[1440:1443]
    h1 = np.maximum(0, feat.astype(np.float64) @ W1.T + b1)
    h2 = np.maximum(0, h1 @ W2.T + b2)
    y64 = h2 @ W3.T + b3
    assert np.allclose(y, y64, rtol=1e-5, atol=1e-5)
    loss, g = orc.mlp_loss_grad(w, feat, tgt)
    assert abs(loss - ((y64 - tgt) ** 2).mean()) < 1e-6 * max(1, loss)
    for i in rng.choice(orc.MLP_PARAMS, 40, replace=False):
        w64 = w.astype(np.float64)
        eps = 1e-7
        wp, wm = w64.copy(), w64.copy()
        wp[i] += eps
        wm[i] -= eps

        def L(ww):
            a = np.maximum(0, feat @ ww[:256].reshape(32, 8).T + ww[256:288])
            a = np.maximum(0, a @ ww[288:1312].reshape(32, 32).T + ww[1312:1344])
            return ((a @ ww[1344:1440].reshape(3, 32).T + ww[1440:1443] - tgt) ** 2).mean()
        fd = (L(wp) - L(wm)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(fd))


# ---------------------------------------------------------------------------------
# learned selection: argmin of the predictions, exact sizes when the two best are
# within the margin; training targets are log2 bits per element
# ---------------------------------------------------------------------------------
def test_learned_pick_rule(orc):
    s = np.array([900, 40, 60], np.uint64)  # exact: RLE smallest
    assert orc.learned_pick([1.0, 5.0, 9.0], s) == orc.CODEC_HUFF       # clear-cut: trust the net
    assert orc.learned_pick([5.0, 9.0, 1.0], s) == orc.CODEC_RLE_HUFF
    assert orc.learned_pick([1.0, 1.01, 9.0], s) == orc.CODEC_RLE       # within 2%: exact sizes
    assert orc.learned_pick([2.0, 2.0, 2.0], s) == orc.CODEC_RLE
    assert orc.learned_pick([1.0, 1.0 + 0.03, 9.0], s) == orc.CODEC_HUFF  # just outside the margin
    # exhaustive ties prefer HUFF, then RLE+Huffman, then RLE
    assert orc.learned_pick([0.0, 0.0, 0.0], np.array([8, 8, 8], np.uint64)) == orc.CODEC_HUFF
    assert orc.learned_pick([0.0, 0.0, 0.0], np.array([12, 8, 8], np.uint64)) == orc.CODEC_RLE_HUFF
    # a NaN prediction neither wins nor triggers the fallback
    assert orc.learned_pick([np.nan, 3.0, 4.0], s) == orc.CODEC_HUFF
    assert orc.learned_pick([3.0, np.nan, 1.0], s) == orc.CODEC_RLE_HUFF


def test_selector_targets_closed_form(orc):
    dims = (3 * 4096 + 100,)
    sizes = np.array([[512, 4, 12], [4096, 64, 2048], [999, 8, np.iinfo(np.uint64).max],
                      [50, 4, 13]], np.uint64)
    tgt, valid = orc.selector_targets(sizes, dims)
    assert valid.tolist() == [1, 1, 0, 1]
    # powers of two are exact: 512 B over 4096 elements = 1 bit each -> 0
    assert tgt[0, 0] == 0.0 and tgt[1, 0] == 3.0 and tgt[0, 1] == np.float32(-7.0)
    m = np.array([4096, 4096, 4096, 100], np.float64)
    want = np.log2(8 * sizes.astype(np.float64)[[0, 1, 3]] / m[[0, 1, 3], None])
    assert np.abs(tgt[[0, 1, 3]] - want).max() <= 2.0 / 65536
    assert tgt[2, 2] == 0.0


def test_learned_mode_reduces_to_other_selectors(orc):
    """A network with zero weights predicts its output bias for every block: a bias
    that strongly favours Huffman gives the forced-Huffman choice on every block, an
    all-equal bias falls back to the exact sizes everywhere (the exhaustive choice).
    Archives then match byte for byte except the header's selector field."""
    rng = np.random.default_rng(21)
    x = rng.standard_normal((40, 90, 70)).astype(np.float32).cumsum(axis=2).astype(np.float32)
    x[:, :, :35] = 0.0
    w = np.zeros(orc.MLP_PARAMS, np.float32)

    def body(ar):
        a = ar.copy()
        a[112:116] = 0
        return a
    w[-3:] = [0.0, 10.0, 10.0]
    _, a_l = orc.compress(x, orc.EB_REL, 1e-3, select=orc.SEL_LEARNED, mlp_w=w)
    _, a_h = orc.compress(x, orc.EB_REL, 1e-3, select=orc.SEL_HUFF)
    assert np.array_equal(body(a_l), body(a_h))
    w[-3:] = [4.0, 4.0, 4.0]
    _, a_l = orc.compress(x, orc.EB_REL, 1e-3, select=orc.SEL_LEARNED, mlp_w=w)
    _, a_e = orc.compress(x, orc.EB_REL, 1e-3, select=orc.SEL_EXHAUSTIVE)
    assert np.array_equal(body(a_l), body(a_e))
    assert orc.parse_header(a_e)["n_codec"][1] > 0  # the zero half is run coded
    # RLE favoured: every run-eligible block is RLE, the others Huffman
    w[-3:] = [10.0, 0.0, 10.0]
    _, a_r = orc.compress(x, orc.EB_REL, 1e-3, select=orc.SEL_LEARNED, mlp_w=w)
    codec = orc.sections(a_r)["codec"]
    st, ebd, ebf, x2, xr = orc.eb_params(orc.EB_REL, 1e-3, float(x.min()), float(x.max()))
    c = orc.construct(x, ebf, x2, xr)
    _, _, nr = orc.run_stats(c["codes"], x.shape, all_blocks=False)
    nblk, _ = orc.geometry(x.shape)
    bz, by, bx = np.meshgrid(np.arange(3), np.arange(6), np.arange(5), indexing="ij")
    m = (np.minimum(16, 40 - 16 * bz) * np.minimum(16, 90 - 16 * by) * np.minimum(16, 70 - 16 * bx)).ravel()
    assert m.size == nblk
    elig = 4 * nr.astype(np.int64) <= m
    assert np.array_equal(codec, np.where(elig, orc.CODEC_RLE, orc.CODEC_HUFF).astype(np.uint8))


# ---------------------------------------------------------------------------------
# interleaved Huffman stream layout, closed form: with a two-symbol book every code
# is one bit, so each of the 32 lanes tops up one 16-bit unit at steps 0, 16, 32, ...
# and a stream is lane 0..31's unit 0, then their unit 1, and so on.  A Huffman
# block is a u16 unit count of stream A (the first 2048 codes), stream A, stream B
# (the other 2048), padded to 4 bytes.
# ---------------------------------------------------------------------------------
def test_interleaved_stream_layout_one_bit_codes(orc):
    rng = np.random.default_rng(12)
    n = 4096
    d = rng.integers(0, 2, n)                 # residuals 0/1 -> codes 512/513
    x = np.zeros(n, np.float32)
    for c0 in range(0, n, 256):               # prediction restarts at every chunk
        x[c0:c0 + 256] = np.cumsum(d[c0:c0 + 256])
    st, ar = orc.compress(x, orc.EB_ABS, 0.5, select=orc.SEL_HUFF)
    sec = orc.sections(ar)
    books = sec["books"]
    assert books[512] == 1 and books[513] == 1 and books[:1024].sum() == 2
    units = sec["payload"].view(np.uint16)
    assert units.size == 1 + 2 * 32 * 4 + 1    # count, 2 streams x 64 bits per lane, pad
    assert units[0] == 128 and units[-1] == 0

    def stream(sym):
        expect = np.zeros((4, 32), np.uint16)
        for lane in range(32):
            bits = sym[lane::32]               # the lane's symbols, one bit each
            for k in range(4):
                v = 0
                for b in bits[16 * k:16 * k + 16]:
                    v = (v << 1) | int(b)
                expect[k, lane] = v
        return expect.ravel()
    assert np.array_equal(units[1:129], stream(d[:2048]))
    assert np.array_equal(units[129:257], stream(d[2048:]))
    st, y = orc.decompress(ar, n)
    assert np.array_equal(y, x)
