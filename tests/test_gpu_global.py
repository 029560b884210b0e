"""GPU parity of global (unchunked) Lorenzo prediction (CSZ_FLAG_GLOBAL_LORENZO).

Construction reads each tile's halo (the elements one step before it on every axis)
so prediction restarts only at the field's faces; reconstruction is the N-D partial
sum over the whole field, by per-axis passes with a decoupled look-back along x.
Archives must be byte-identical to the oracle's (orc_compress_ex, global) and
reconstructions bit-identical to the oracle's sequential recurrence.
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


def _parity(api, orc, x, eb, mode="rel", sel="exhaustive", radius=512):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    ar, nb, st = api.compress(xd, eb, mode, select=sel, radius=radius, global_lorenzo=True, raise_on_error=False)
    torch.cuda.synchronize()
    ost, ref = orc.compress_ex(x, orc.EB_REL if mode == "rel" else orc.EB_ABS, eb, radius=radius,
                               select=api.SELECT[sel], global_lorenzo=True, raise_on_error=False)
    assert st == ost
    if st:
        return st
    assert api.header(ar)["flags"] & 8
    assert nb == ref.size and np.array_equal(ar[:nb].cpu().numpy(), ref)
    y, _ = api.decompress(ar, nb)
    st, yr = orc.decompress(ref, x.size)
    assert np.array_equal(y.cpu().numpy().ravel().view(np.uint32), yr.view(np.uint32))
    assert float(np.abs(x.ravel().astype(np.float64) - yr).max()) <= api.header(ar)["eb_f"]
    return 0


def _walk(shape, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(shape).astype(np.float32)
    for ax in range(len(shape)):
        x = np.cumsum(x, axis=ax).astype(np.float32)
    return x


@pytest.mark.parametrize("shape", [(5000,), (1 << 22,), (70, 131), (128, 192), (1800, 3600), (19, 23, 37),
                                   (40, 90, 70), (128, 128, 128), (1, 1), (3, 1, 5)])
def test_global_parity_shapes(gpu, orc, shape):
    x = _walk(shape, sum(shape))
    x[tuple(slice(0, max(1, s // 3)) for s in shape)] = 0.0
    if x.size == 1:
        assert _parity(gpu, orc, x, 1e-3, mode="abs") == 0  # one value has no range for a relative bound
    else:
        assert _parity(gpu, orc, x, 1e-4) == 0


@pytest.mark.parametrize("sel", ["huff", "rle", "rle_huff", "heuristic", "exhaustive"])
def test_global_parity_selectors_and_outliers(gpu, orc, sel):
    x = _walk((40, 64, 80), 11)
    x[:, :32, :] = 0.0
    assert _parity(gpu, orc, x, 1e-3, sel=sel) == 0
    assert _parity(gpu, orc, x, 1e-4, sel=sel, radius=8) == 0  # many outliers


def test_global_patches_and_lognormal(gpu, orc):
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
    assert _parity(gpu, orc, x, eb, mode="abs") == 0
    from paper_2105_12912_gb300 import synth
    y = synth.make_field(synth.workload_3d(n=160, seed=9, eb=1e-4), "cpu").numpy()
    assert _parity(gpu, orc, y, 1e-4) == 0


def test_global_smaller_and_refusals(gpu):
    """On a smooth field the global predictor's archive is smaller (no restarts at the
    8^3 chunk faces).  (On rough fields the lower-order predictors of the chunk faces
    can win: the 3-D mixed difference sums 8 noisy terms.)"""
    z, y, x = torch.meshgrid(*[torch.linspace(0, 4, 128, device="cuda")] * 3, indexing="ij")
    x = (torch.sin(x) * torch.cos(y) * torch.sin(0.7 * z) * 100 + x * y * z).contiguous()
    _, nb_c, _ = gpu.compress(x, 1e-5)
    _, nb_g, _ = gpu.compress(x, 1e-5, global_lorenzo=True)
    assert nb_g < nb_c
    _, _, st = gpu.compress(x.double(), 1e-4, global_lorenzo=True, raise_on_error=False)
    assert st == 1  # CSZ_E_ARG: double fields use chunked prediction
