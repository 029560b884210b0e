"""GPU path vs CPU oracle: byte-identical archives and bit-identical reconstructions.

All inputs are seeded and synthetic; every call goes through the C ABI
(libcszp.so) via the ctypes binding.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_12912_gb300 import api
    api.workspace_bytes((1,))
    return api


def _field(kind, shape, seed):
    rng = np.random.default_rng(seed)
    if kind == "walk":
        x = rng.standard_normal(shape).astype(np.float32)
        for ax in range(len(shape)):
            x = np.cumsum(x, axis=ax).astype(np.float32)
        return x
    if kind == "noise":
        return (rng.standard_normal(shape) * 100).astype(np.float32)
    if kind == "sparse":
        x = rng.standard_normal(shape).astype(np.float32).cumsum(axis=-1).astype(np.float32)
        mask = rng.random(shape) < 0.5
        x[mask] = 0.0
        return x
    if kind == "lognormal":
        return np.exp(rng.standard_normal(shape)).astype(np.float32)
    raise ValueError(kind)


def _gpu_archive(api, x, eb, mode, radius, sel, weights=None):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    ar, nb, st = api.compress(xd, eb=eb, eb_mode=mode, radius=radius, select=sel, weights=weights,
                              raise_on_error=False)
    torch.cuda.synchronize()
    return st, ar, nb


def _check(api, orc, x, eb=1e-3, mode="rel", radius=512, sel="exhaustive"):
    st, ar, nb = _gpu_archive(api, x, eb, mode, radius, sel)
    ost, ref = orc.compress(x, orc.EB_REL if mode == "rel" else orc.EB_ABS, eb, radius=radius,
                            select=api.SELECT[sel], raise_on_error=False)
    assert st == ost, (st, ost)
    if st:
        return
    g = ar[:nb].cpu().numpy()
    if g.size != ref.size or not np.array_equal(g, ref):
        # locate the first differing section for the report
        hs = orc.sections(ref)
        diff = np.nonzero(g[: min(g.size, ref.size)] != ref[: min(g.size, ref.size)])[0]
        raise AssertionError(f"archive differs: gpu {g.size} B, oracle {ref.size} B, first diff at "
                             f"{diff[:5] if diff.size else 'tail'}; oracle header {hs['header']}")
    y, dst = api.decompress(ar, nb)
    torch.cuda.synchronize()
    ost, yr = orc.decompress(ref, x.size)
    assert np.array_equal(y.cpu().numpy().ravel().view(np.uint32), yr.view(np.uint32))
    eb_f = orc.parse_header(ref)["eb_f"]
    assert np.abs(x.ravel().astype(np.float64) - yr.astype(np.float64)).max() <= eb_f


@pytest.mark.parametrize("shape", [(5000,), (4096,), (1,), (12289,), (70, 131), (64, 64), (1, 1), (129, 65),
                                   (19, 23, 37), (16, 16, 16), (1, 1, 1), (33, 17, 70)])
@pytest.mark.parametrize("kind", ["walk", "sparse"])
def test_parity_shapes(gpu, orc, shape, kind):
    x = _field(kind, shape, 7 + len(shape))
    mode = "abs" if x.size == 1 or float(x.max()) == float(x.min()) else "rel"
    _check(gpu, orc, x, eb=1e-3 if mode == "rel" else 0.05, mode=mode)


@pytest.mark.parametrize("sel", ["huff", "rle", "rle_huff", "heuristic", "exhaustive"])
@pytest.mark.parametrize("shape", [(20000,), (150, 210), (40, 40, 41)])
def test_parity_selectors(gpu, orc, sel, shape):
    x = _field("sparse", shape, 3)
    _check(gpu, orc, x, eb=1e-2, sel=sel)


@pytest.mark.parametrize("radius", [1, 2, 16, 100, 512])
def test_parity_radius(gpu, orc, radius):
    x = _field("noise", (90, 111), 5)
    _check(gpu, orc, x, eb=1e-3, radius=radius)


@pytest.mark.parametrize("eb", [1e-1, 1e-2, 1e-4, 1e-6])
def test_parity_error_bounds(gpu, orc, eb):
    x = _field("lognormal", (24, 50, 50), 9)
    _check(gpu, orc, x, eb=eb)


def test_parity_patches(gpu, orc):
    """Values on the FP32 rounding boundary at large |k| need verbatim patches."""
    eb = 0.0123456789
    st, ebd, ebf, x2, xr = orc.eb_params(orc.EB_ABS, eb)
    vals = []
    for k in [1, 3, 1000, 654321, 3000000, 7000000]:
        m32 = np.float32((k + 0.5) * float(x2))
        for d in range(-3, 4):
            v = m32
            for _ in range(abs(d)):
                v = np.nextafter(v, np.float32(np.inf if d > 0 else -np.inf))
            vals.extend([v, -v])
    x = np.array(vals * 50, dtype=np.float32)
    _check(gpu, orc, x, eb=eb, mode="abs")
    assert orc.parse_header(orc.compress(x, orc.EB_ABS, eb)[1])["n_patch"] > 0


def test_status_codes(gpu, orc):
    x = _field("walk", (64, 64), 1)
    bad = x.copy()
    bad[3, 3] = np.nan
    assert _gpu_archive(gpu, bad, 1e-3, "rel", 512, "exhaustive")[0] == 2
    assert _gpu_archive(gpu, bad, 1e-3, "abs", 512, "exhaustive")[0] == 2
    const = np.full((50, 50), 2.5, np.float32)
    assert _gpu_archive(gpu, const, 1e-3, "rel", 512, "exhaustive")[0] == 1
    big = np.array([0.0, 1e7, 0.0], np.float32)
    assert _gpu_archive(gpu, big, 0.5, "abs", 512, "exhaustive")[0] == 3
    # archive capacity too small
    xd = torch.from_numpy(x).cuda()
    small = torch.empty(2000, dtype=torch.uint8, device="cuda")
    _, _, st = gpu.compress(xd, 1e-6, out=small, raise_on_error=False)
    assert st == 5


def test_corrupt_archives(gpu, orc):
    x = _field("sparse", (90, 140), 8)
    st, ar, nb = _gpu_archive(gpu, x, 1e-2, "rel", 64, "exhaustive")
    good = ar[:nb].clone()
    # truncation and header damage are rejected on the host
    _, st = gpu.decompress(good[:nb - 1].clone(), nb - 1, dims=x.shape, raise_on_error=False)
    assert st == 4
    for off, val in [(0, 0), (4, 9), (6, 4), (52, 0), (56, 7), (60, 16)]:
        bad = good.clone()
        bad[off] = val
        _, st = gpu.decompress(bad, nb, dims=x.shape, raise_on_error=False)
        assert st == 4, off
    # random payload / section damage: the GPU agrees with the oracle on corrupt-or-not,
    # and never faults
    rng = np.random.default_rng(3)
    ref = good.cpu().numpy()
    for _ in range(60):
        bad = ref.copy()
        i = int(rng.integers(128, bad.size))
        bad[i] ^= np.uint8(1 << int(rng.integers(0, 8)))
        ost, yo = orc.decompress(bad, x.size, raise_on_error=False)
        y, gst = gpu.decompress(torch.from_numpy(bad).cuda(), nb, dims=x.shape, raise_on_error=False)
        torch.cuda.synchronize()
        assert gst in (0, 4)
        if ost == 0 and gst == 0:
            assert np.array_equal(y.cpu().numpy().ravel().view(np.uint32), yo.view(np.uint32))


def test_cross_decode(gpu, orc):
    """GPU decodes oracle archives and the oracle decodes GPU archives."""
    x = _field("walk", (3, 70, 90), 4)
    st, ref = orc.compress(x, orc.EB_REL, 1e-3, radius=32)
    y, st = gpu.decompress(torch.from_numpy(ref).cuda(), ref.size)
    ost, yo = orc.decompress(ref, x.size)
    assert np.array_equal(y.cpu().numpy().ravel().view(np.uint32), yo.view(np.uint32))


def test_parity_deep_huffman_codes(gpu, orc):
    """Residual counts following the Fibonacci numbers give a maximally deep Huffman
    tree (codes far longer than the 12-bit lookup table), exercising the decoder's
    long-code search and multi-unit top-ups."""
    fib = [1, 1]
    while len(fib) < 28:
        fib.append(fib[-1] + fib[-2])
    rng = np.random.default_rng(17)
    deltas = np.concatenate([np.full(c, i - 14, np.int64) for i, c in enumerate(fib)])
    rng.shuffle(deltas)
    n = deltas.size - deltas.size % 256
    deltas = deltas[:n]
    x = np.empty(n, np.float32)
    for c0 in range(0, n, 256):  # prediction restarts at every 256-element chunk
        x[c0:c0 + 256] = np.cumsum(deltas[c0:c0 + 256])
    for sel in ("huff", "exhaustive"):
        _check(gpu, orc, x, eb=0.5, mode="abs", sel=sel)
    st, ar = orc.compress(x, orc.EB_ABS, 0.5, select=orc.SEL_HUFF)
    books = orc.sections(ar)["books"][:1024]
    assert books.max() >= 24  # deep enough to leave the lookup table far behind
