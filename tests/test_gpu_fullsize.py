"""GPU parity at the workloads' full sizes, through the same API calls bench.py times.

* 1-D 2^20 random walk + sines (rel eb 1e-3) and 2-D 1800x3600 GRF k^-3 with 20% zeros
  (rel eb 1e-4, each codec forced and the exhaustive choice): archives byte-identical
  to the oracle's, reconstructions bit-identical.
* 3-D 512^3 log-normal field (rel eb 1e-2 and 1e-4): too large for the scalar oracle in
  a test, so the error bound is checked on every element on the GPU, and sampled
  codec blocks are compressed by the oracle as standalone 16^3 fields with the same
  absolute bound -- prediction is chunk-local, so a block's reconstruction does not
  depend on the rest of the field -- and must match the GPU bit for bit.
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


def _full_parity(api, orc, x_cpu, eb, sel):
    xd = x_cpu.cuda()
    ar, nb, _ = api.compress(xd, eb, "rel", select=sel)
    y, _ = api.decompress(ar, nb)
    torch.cuda.synchronize()
    st, ref = orc.compress(x_cpu.numpy(), orc.EB_REL, eb, select=api.SELECT[sel])
    assert st == 0
    g = ar[:nb].cpu().numpy()
    assert g.size == ref.size and np.array_equal(g, ref)
    st, yr = orc.decompress(ref, x_cpu.numel())
    assert np.array_equal(y.cpu().numpy().ravel().view(np.uint32), yr.view(np.uint32))
    eb_f = api.header(ar)["eb_f"]
    assert float((x_cpu.double() - y.cpu().double()).abs().max()) <= eb_f


def test_fullsize_1d_walk_sines(gpu, orc):
    from paper_2105_12912_gb300 import synth
    spec = synth.workload_1d()
    x = synth.make_field(spec, "cpu")
    assert x.numel() == 1 << 20
    _full_parity(gpu, orc, x, spec.eb, "exhaustive")


@pytest.mark.parametrize("sel", ["exhaustive", "huff", "rle", "rle_huff"])
def test_fullsize_2d_grf(gpu, orc, sel):
    from paper_2105_12912_gb300 import synth
    spec = synth.workload_2d()
    x = synth.make_field(spec, "cpu")
    assert tuple(x.shape) == (1800, 3600)
    assert float((x == 0).float().mean()) >= 0.2
    _full_parity(gpu, orc, x, spec.eb, sel)


@pytest.mark.parametrize("eb", [1e-2, 1e-4])
def test_fullsize_3d_lognormal(gpu, orc, eb):
    from paper_2105_12912_gb300 import synth
    spec = synth.workload_3d(eb=eb)
    x = synth.make_field(spec, "cuda")
    assert tuple(x.shape) == (512, 512, 512)
    ar, nb, _ = gpu.compress(x, eb, "rel")
    y, _ = gpu.decompress(ar, nb)
    torch.cuda.synchronize()
    h = gpu.header(ar)
    err = (x.double() - y.double()).abs().max().item()
    assert err <= h["eb_f"]
    assert h["nblk"] == 32 ** 3
    # sampled blocks through the oracle as standalone fields with the same bound
    rng = np.random.default_rng(int(eb * 1e6))
    picks = [(0, 0, 0), (31, 31, 31)] + [tuple(int(v) for v in rng.integers(0, 32, 3)) for _ in range(14)]
    for bz, by, bx in picks:
        sub = x[16 * bz:16 * bz + 16, 16 * by:16 * by + 16, 16 * bx:16 * bx + 16].contiguous().cpu()
        st, ref = orc.compress(sub.numpy(), orc.EB_ABS, h["eb_d"])
        assert st == 0
        assert orc.parse_header(ref)["eb_f"] == h["eb_f"]
        st, yr = orc.decompress(ref, sub.numel())
        got = y[16 * bz:16 * bz + 16, 16 * by:16 * by + 16, 16 * bx:16 * bx + 16].contiguous().cpu()
        assert np.array_equal(got.numpy().ravel().view(np.uint32), yr.view(np.uint32)), (bz, by, bx)
