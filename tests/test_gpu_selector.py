"""Learned codec selector on the GPU: training rows, inference and gradient against the
CPU oracle, LEARNED-mode archives against the oracle, and what training gains.

Parity bars: features, targets, sizes and network outputs bit-exact (both sides use
the same integer ratios, the same fixed-point logarithm and the same FMA chains);
the FP32 gradient within 1e-4 of the oracle's double-precision gradient (relative to
its largest component); archives byte-identical.
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


def _sparse_field(shape, seed, zero_frac=0.4):
    """Random walk along x with whole codec blocks (1-D 4096, 2-D 64^2, 3-D 16^3) zeroed."""
    rng = np.random.default_rng(seed)
    x = np.cumsum(rng.standard_normal(shape).astype(np.float32), axis=-1).astype(np.float32)
    edge = {1: 4096, 2: 64, 3: 16}[len(shape)]
    grid = [(s + edge - 1) // edge for s in shape]
    for idx in zip(*np.nonzero(rng.random(grid) < zero_frac)):
        x[tuple(slice(edge * i, edge * i + edge) for i in idx)] = 0.0
    return x


def _oracle_rows(orc, x, eb, radius=512):
    vmin, vmax = float(x.min()), float(x.max())
    st, ebd, ebf, x2, xr = orc.eb_params(orc.EB_REL, eb, vmin, vmax)
    assert st == 0
    c = orc.construct(x, ebf, x2, xr, radius)
    vh, lh, _ = orc.run_stats(c["codes"], x.shape, all_blocks=False)
    cl, vl, ll = orc.huffman_lengths(c["hist"]), orc.huffman_lengths(vh), orc.huffman_lengths(lh)
    sizes = orc.block_sizes(c["codes"], x.shape, radius, cl, vl, ll, all_blocks=False)
    feat = orc.block_features(c["codes"], x.shape, radius)
    tgt, valid = orc.selector_targets(sizes, x.shape)
    return feat, tgt, sizes, valid


@pytest.mark.parametrize("shape,eb,radius", [((40, 90, 70), 1e-3, 512), ((150, 210), 1e-2, 512),
                                             ((30000,), 1e-3, 64), ((33, 17, 70), 1e-4, 512)])
def test_selector_rows_match_oracle(gpu, orc, shape, eb, radius):
    x = _sparse_field(shape, 5)
    rows = gpu.selector_rows(torch.from_numpy(x).cuda(), eb, "rel", radius=radius)
    feat, tgt, sizes, valid = _oracle_rows(orc, x, eb, radius)
    assert np.array_equal(rows["valid"].cpu().numpy(), valid)
    assert np.array_equal(rows["feat"].cpu().numpy().view(np.uint32), feat.view(np.uint32))
    assert np.array_equal(rows["target"].cpu().numpy().view(np.uint32), tgt.view(np.uint32))
    gs = rows["sizes"].cpu().numpy().view(np.uint32).astype(np.uint64)
    gs[gs == 0xFFFFFFFF] = np.iinfo(np.uint64).max
    assert np.array_equal(gs, sizes)
    assert valid.any() and not valid.all()


def test_selector_predict_bit_exact(gpu, orc):
    rng = np.random.default_rng(4)
    w = (rng.standard_normal(gpu.MLP_PARAMS) * 0.4).astype(np.float32)
    feat = rng.random((3001, 8)).astype(np.float32) * np.array([1, 10, 1, 1, 1, 1, 1, 1], np.float32)
    y = gpu.selector_predict(torch.from_numpy(w).cuda(), torch.from_numpy(feat).cuda()).cpu().numpy()
    assert np.array_equal(y.view(np.uint32), orc.mlp_forward(w, feat).view(np.uint32))


def test_selector_gradient_check(gpu, orc):
    """FP32 GPU gradient of the mean squared error against the oracle's double-precision
    backward pass, on real training rows with some rows masked out."""
    from paper_2105_12912_gb300 import selector
    x = _sparse_field((64, 128, 128), 6)
    rows = gpu.selector_rows(torch.from_numpy(x).cuda(), 1e-3, "rel")
    valid = rows["valid"].clone()
    valid[::7] = 0
    for seed in (0, 1):
        w = selector.init_weights(seed)
        w += 0.05 * torch.randn(w.shape, generator=torch.Generator().manual_seed(seed)).cuda()
        loss, g = gpu.selector_grad(w, rows["feat"], rows["target"], valid)
        keep = valid.cpu().numpy().astype(bool)
        ref_loss, ref_g = orc.mlp_loss_grad(w.cpu().numpy(), rows["feat"].cpu().numpy()[keep],
                                            rows["target"].cpu().numpy()[keep])
        g = g.cpu().numpy().astype(np.float64)
        assert abs(loss - ref_loss) <= 1e-5 * max(1.0, abs(ref_loss))
        assert np.abs(g - ref_g).max() <= 1e-4 * np.abs(ref_g).max()
        # every parameter group receives gradient
        assert np.abs(ref_g[:256]).max() > 0 and np.abs(ref_g[1344:1443]).max() > 0


def test_selector_training_is_reproducible_and_descends(gpu):
    from paper_2105_12912_gb300 import selector
    x = _sparse_field((48, 96, 96), 8)
    rows = gpu.selector_rows(torch.from_numpy(x).cuda(), 1e-3, "rel")
    w1, l0, l1 = selector.train(rows, seed=3, steps=300)
    w2, _, _ = selector.train(rows, seed=3, steps=300)
    assert torch.equal(w1, w2)
    assert l1 < 0.25 * l0


@pytest.mark.parametrize("kind", ["trained", "random", "tie"])
def test_learned_archives_match_oracle(gpu, orc, kind):
    from paper_2105_12912_gb300 import selector
    x = _sparse_field((40, 90, 70), 9)
    xd = torch.from_numpy(x).cuda()
    if kind == "trained":
        rows = gpu.selector_rows(torch.from_numpy(_sparse_field((48, 96, 96), 10)).cuda(), 1e-3, "rel")
        w, _, _ = selector.train(rows, seed=1, steps=400)
    elif kind == "random":
        w = selector.init_weights(7) * 3.0
    else:  # zero weights, equal output bias: every decision falls back to exact sizes
        w = torch.zeros(gpu.MLP_PARAMS, device="cuda")
        w[-3:] = 2.5
    ar, nb, _ = gpu.compress(xd, 1e-3, "rel", select="learned", weights=w)
    st, ref = orc.compress(x, orc.EB_REL, 1e-3, select=orc.SEL_LEARNED, mlp_w=w.cpu().numpy())
    assert st == 0
    assert np.array_equal(ar[:nb].cpu().numpy(), ref)
    y, _ = gpu.decompress(ar, nb)
    st, yr = orc.decompress(ref, x.size)
    assert np.array_equal(y.cpu().numpy().ravel().view(np.uint32), yr.view(np.uint32))


def test_training_gains_over_heuristic(gpu):
    """Trained on the method's own sizes from 8 fields, evaluated on 4 held-out fields
    (3-D GRF k^-3 with 0-60% zero 16^3 blocks, rel eb 1e-3): the learned selector's
    archives are smaller than the paper's heuristic's and within 1% of exhaustive."""
    from paper_2105_12912_gb300 import selector, synth

    def fields(seeds):
        return [(lambda s=s: synth.make_field(synth.workload_selector(s, dims=(48, 160, 160)), "cuda"), 1e-3, "rel")
                for s in seeds]
    rows = selector.collect_rows(fields(range(1000, 1008)))
    w, l0, l1 = selector.train(rows, seed=0, steps=1500)
    rep = selector.evaluate(w, fields(range(2000, 2004)))
    assert l1 < l0
    assert rep["bytes"]["learned"] < rep["bytes"]["heuristic"], rep
    assert rep["regret_vs_exhaustive"] <= 0.01, rep


def test_fullsize_selector_workload(gpu, orc):
    """The learned-selector configuration at full size: 3-D 100x500x500 GRF k^-3 fields
    with 0-60% zero 16^3 blocks, rel eb 1e-3; trained on the method's own sizes from
    64 fields (seeds 1000-1063), evaluated on 16 held-out fields (seeds 2000-2015).
    LEARNED archives of two held-out fields are byte-identical to the oracle's; over
    all 16 the size regret against exhaustive selection is at most 1% and the archives
    are smaller than the paper's heuristic's."""
    from paper_2105_12912_gb300 import selector, synth

    def fields(seeds):
        return [(lambda s=s: synth.make_field(synth.workload_selector(s), "cuda"), 1e-3, "rel") for s in seeds]
    rows = selector.collect_rows(fields(range(1000, 1064)))
    assert rows["feat"].shape[0] == 64 * 7 * 32 * 32
    w, l0, l1 = selector.train(rows, seed=0, steps=3000, lr=1e-2)
    assert l1 < 0.5 * l0
    del rows
    for s in (2000, 2007):
        xh = synth.make_field(synth.workload_selector(s), "cpu")
        ar, nb, _ = gpu.compress(xh.cuda(), 1e-3, "rel", select="learned", weights=w)
        st, ref = orc.compress(xh.numpy(), orc.EB_REL, 1e-3, select=orc.SEL_LEARNED, mlp_w=w.cpu().numpy())
        assert st == 0
        assert ref.size == nb and np.array_equal(ar[:nb].cpu().numpy(), ref), s
        y, _ = gpu.decompress(ar, nb)
        st, yr = orc.decompress(ref, xh.numel())
        assert np.array_equal(y.cpu().numpy().ravel().view(np.uint32), yr.view(np.uint32)), s
    rep = selector.evaluate(w, fields(range(2000, 2016)))
    assert rep["regret_vs_exhaustive"] <= 0.01, rep
    assert rep["bytes"]["learned"] < rep["bytes"]["heuristic"], rep
