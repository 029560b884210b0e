"""GPU parity at the workloads' full sizes, through the same API calls bench.py times.

* 1-D 2^20 random walk + sines (rel eb 1e-3) and 2-D 1800x3600 GRF k^-3 with 20% zeros
  (rel eb 1e-4, each codec forced and the exhaustive choice): archives byte-identical
  to the oracle's, reconstructions bit-identical.
* 3-D 512^3 log-normal field (rel eb 1e-2 and 1e-4): the whole archive byte-identical
  to the oracle's (codes, outlier and patch records, streams, books, selection) and
  the whole reconstruction bit-identical to the oracle's sequential recurrence.  The
  field has 32768 codec blocks, far more than the persistent construction grid, so
  every construct CTA draws many ticketed tiles and the payload look-back spans the
  whole field.
* 3-D 160x256x256 GRF with zero blocks (2560 codec blocks, more than four times the
  resident construct grid of 608 CTAs) under every selector, the learned one included.
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
    assert h["nblk"] == 32 ** 3
    xh = x.cpu()
    del x
    st, ref = orc.compress(xh.numpy(), orc.EB_REL, eb)
    assert st == 0
    assert ref.size == nb and np.array_equal(ar[:nb].cpu().numpy(), ref)
    st, yr = orc.decompress(ref, xh.numel())
    assert st == 0
    assert np.array_equal(y.cpu().numpy().ravel().view(np.uint32), yr.view(np.uint32))
    assert float((xh.double() - y.cpu().double()).abs().max()) <= h["eb_f"]


@pytest.fixture(scope="module")
def learned_weights(gpu):
    """Selector weights trained on the method's own sizes from four small fields."""
    from paper_2105_12912_gb300 import selector, synth
    rows = selector.collect_rows(
        [(lambda s=s: synth.make_field(synth.workload_selector(s, dims=(48, 96, 96)), "cuda"), 1e-3, "rel")
         for s in range(1000, 1004)])
    w, _, _ = selector.train(rows, seed=3, steps=600)
    return w


@pytest.mark.parametrize("sel", ["exhaustive", "heuristic", "learned", "huff", "rle", "rle_huff"])
def test_3d_many_tiles_every_selector(gpu, orc, learned_weights, sel):
    """2560 codec blocks (160x256x256): every construct CTA takes several tiles and the
    look-back places payloads over thousands of blocks; archive and reconstruction
    must equal the oracle's under every selector."""
    from paper_2105_12912_gb300 import synth
    spec = synth.workload_selector(1234, dims=(160, 256, 256))
    xh = synth.make_field(spec, "cpu")
    xd = xh.cuda()
    w = learned_weights if sel == "learned" else None
    ar, nb, _ = gpu.compress(xd, 1e-3, "rel", select=sel, weights=w)
    y, _ = gpu.decompress(ar, nb)
    torch.cuda.synchronize()
    assert gpu.header(ar)["nblk"] == 2560
    st, ref = orc.compress(xh.numpy(), orc.EB_REL, 1e-3, select=gpu.SELECT[sel],
                           mlp_w=None if w is None else w.cpu().numpy())
    assert st == 0
    assert ref.size == nb and np.array_equal(ar[:nb].cpu().numpy(), ref)
    st, yr = orc.decompress(ref, xh.numel())
    assert np.array_equal(y.cpu().numpy().ravel().view(np.uint32), yr.view(np.uint32))
