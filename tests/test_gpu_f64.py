"""GPU parity of the double-precision input path (csz_compress_f64 / csz_decompress_f64).

Archives byte-identical to the oracle's orc_compress_f64 and reconstructions
bit-identical to orc_decompress_f64, across dimensionalities, edge blocks, selectors,
bound modes, fields at the half points of the quantization step, and a 256^3 field;
plus the status codes of the type checks and guards.
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
    return api


def _parity(api, orc, x, eb, mode="rel", sel="exhaustive"):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    ar, nb, st = api.compress(xd, eb, mode, select=sel, raise_on_error=False)
    torch.cuda.synchronize()
    ost, ref = orc.compress_f64(x, orc.EB_REL if mode == "rel" else orc.EB_ABS, eb, select=api.SELECT[sel],
                                raise_on_error=False)
    assert st == ost
    if st:
        return st
    g = ar[:nb].cpu().numpy()
    assert g.size == ref.size and np.array_equal(g, ref)
    y, _ = api.decompress(ar, nb)
    assert y.dtype == torch.float64
    st, yr = orc.decompress_f64(ref, x.size)
    assert np.array_equal(y.cpu().numpy().ravel().view(np.uint64), yr.view(np.uint64))
    eb_d = api.header(ar)["eb_d"]
    assert float(np.abs(x.ravel() - yr).max()) <= eb_d
    return 0


def _walk(shape, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(shape)
    for ax in range(len(shape)):
        x = np.cumsum(x, axis=ax)
    return x * scale


@pytest.mark.parametrize("shape", [(5000,), (8192,), (70, 131), (128, 192), (19, 23, 37), (32, 48, 64)])
@pytest.mark.parametrize("eb", [1e-3, 1e-6])
def test_f64_parity_shapes(gpu, orc, shape, eb):
    x = _walk(shape, sum(shape))
    x[tuple(slice(0, max(1, s // 3)) for s in shape)] = 0.0
    assert _parity(gpu, orc, x, eb) == 0


@pytest.mark.parametrize("sel", ["huff", "rle", "rle_huff", "heuristic", "exhaustive"])
def test_f64_parity_selectors(gpu, orc, sel):
    x = _walk((40, 64, 80), 7, 1e3)
    x[:, :32, :] = 0.0
    assert _parity(gpu, orc, x, 1e-4, sel=sel) == 0


def test_f64_half_points_and_abs(gpu, orc):
    eb = 0.37
    st, eb_d, step, rstep = orc.eb_params_f64(orc.EB_ABS, eb)
    vals = []
    for k in [0, 1, 3, 1000, 12345, 2 ** 20 + 7, 2 ** 26 - 5, -1, -777]:
        for base in (2 * eb, step):
            c = (k + 0.5) * base
            for u in range(-3, 4):
                vals.append(c + u * np.spacing(c))
    x = np.array(vals * 40)
    assert _parity(gpu, orc, x, eb, mode="abs") == 0


def test_f64_fullsize_256cubed(gpu, orc):
    """A 256^3 double log-normal field (4096 codec blocks, many tiles per construct CTA),
    rel eb 1e-6: archive and reconstruction equal to the oracle's."""
    from paper_2105_12912_gb300 import synth
    x = synth.make_field(synth.workload_3d(n=256, seed=5, eb=1e-6), "cpu").numpy().astype(np.float64)
    x = x * (1.0 + 1e-9 * np.arange(x.size).reshape(x.shape) / x.size)  # values FP32 cannot hold
    assert _parity(gpu, orc, x, 1e-6) == 0


def test_f64_statuses(gpu, orc):
    from paper_2105_12912_gb300 import _lib
    x = _walk((3000,), 3)
    x[17] = np.nan
    assert _parity(gpu, orc, x, 1e-3) == 2  # CSZ_E_NONFINITE
    big = np.array([0.0, 2.0 ** 27 * 0.2 * 1.01, 0.0])
    assert _parity(gpu, orc, big, 0.1, mode="abs") == 3  # CSZ_E_RANGE
    assert _parity(gpu, orc, np.full(500, 2.5), 1e-3) == 1  # CSZ_E_ARG: no value range
    # an archive of one type decoded as the other
    xd = torch.from_numpy(_walk((5000,), 4)).cuda()
    ar64, nb64, _ = gpu.compress(xd, 1e-4)
    ar32, nb32, _ = gpu.compress(xd.float(), 1e-4)
    assert gpu.elem_bytes(bytes(ar64[:128].cpu().numpy().tobytes())) == 8
    assert gpu.elem_bytes(bytes(ar32[:128].cpu().numpy().tobytes())) == 4
    _, st = gpu.decompress(ar64, nb64, out=torch.empty(5000, dtype=torch.float32, device="cuda"),
                           raise_on_error=False)
    assert st == _lib.E_ARG
    _, st = gpu.decompress(ar32, nb32, out=torch.empty(5000, dtype=torch.float64, device="cuda"),
                           raise_on_error=False)
    assert st == _lib.E_ARG
