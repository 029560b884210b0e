"""Batched compression, replayed as a CUDA graph: one persistent launch for all fields
(plan "persistent") or one launch per stage (plan "staged").

Every field's archive from the batch must be byte-identical to what the single-field
call writes (and, for a sample, to the oracle's), under both plans, across mixed
dimensionalities, REL/ABS bounds, shapes whose rows TMA cannot describe (x extent not
a multiple of 4, offset base pointers), fields with errors (which must not disturb the
others), and repeated graph replays with new data in the same buffers.
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


def _mixed_fields(seed=0):
    rng = np.random.default_rng(seed)
    shapes = [(5000,), (4096,), (1,), (70000,), (70, 131), (64, 64), (129, 65), (300, 301), (19, 23, 37),
              (16, 16, 16), (33, 17, 70), (40, 64, 64), (3, 5, 7), (1000,), (2, 3)]
    out = []
    for i, sh in enumerate(shapes):
        x = rng.standard_normal(sh).astype(np.float32)
        for ax in range(len(sh)):
            x = np.cumsum(x, axis=ax).astype(np.float32)
        if i % 3 == 0:
            x[tuple(slice(0, max(1, s // 2)) for s in sh)] = 0.0
        mode = "abs" if x.size == 1 or float(x.max()) == float(x.min()) else ("rel" if i % 4 else "abs")
        eb = [1e-2, 1e-3, 1e-4][i % 3] if mode == "rel" else 0.05
        out.append((x, eb, mode))
    return out


def _single(api, x, eb, mode, sel="exhaustive", weights=None):
    ar, nb, st = api.compress(x, eb, mode, select=sel, weights=weights, raise_on_error=False)
    return st, ar[:nb].cpu().numpy() if st == 0 else None


PLANS = ["persistent", "staged"]


@pytest.mark.parametrize("plan", PLANS)
@pytest.mark.parametrize("sel", ["exhaustive", "heuristic", "huff", "rle_huff"])
def test_batch_matches_single_field_calls(gpu, sel, plan):
    fields = _mixed_fields(1)
    xs = [torch.from_numpy(x).cuda() for x, _, _ in fields]
    bc = gpu.BatchCompressor(xs, [e for _, e, _ in fields], [m for _, _, m in fields], select=sel, plan=plan,
                             autotune=False)
    assert bc.info()["persistent"] == (plan == "persistent")
    bc.run()
    sizes, stats = bc.results()
    for i, (x, eb, mode) in enumerate(fields):
        st, ref = _single(gpu, xs[i], eb, mode, sel)
        assert stats[i] == st, (i, stats[i], st)
        assert sizes[i] == ref.size
        assert np.array_equal(bc.archives[i][:sizes[i]].cpu().numpy(), ref), i


def test_batch_matches_oracle_and_replays(gpu, orc):
    fields = _mixed_fields(2)
    xs = [torch.from_numpy(x).cuda() for x, _, _ in fields]
    bc = gpu.BatchCompressor(xs, [e for _, e, _ in fields], [m for _, _, m in fields])
    for rep in range(3):
        if rep == 2:  # new data in the same buffers
            for x in xs:
                x.mul_(1.5).add_(0.25)
        bc.run()
        sizes, stats = bc.results()
        assert all(s == 0 for s in stats)
        for i in (0, 4, 8, 11):
            _, eb, mode = fields[i]
            xh = xs[i].cpu().numpy()
            st, ref = orc.compress(xh, orc.EB_REL if mode == "rel" else orc.EB_ABS, eb)
            assert st == 0
            assert np.array_equal(bc.archives[i][:sizes[i]].cpu().numpy(), ref), (rep, i)
            y, _ = gpu.decompress(bc.archives[i], sizes[i])
            st, yr = orc.decompress(ref, xh.size)
            assert np.array_equal(y.cpu().numpy().ravel().view(np.uint32), yr.view(np.uint32))


@pytest.mark.parametrize("plan", PLANS)
def test_batch_without_tma_layouts(gpu, plan):
    """Rows whose byte pitch is not a multiple of 16 and base pointers off 16 bytes
    take the thread-loaded path."""
    rng = np.random.default_rng(3)
    base = torch.from_numpy(rng.standard_normal(200000).astype(np.float32).cumsum()).cuda()
    xs = [base[1:1 + 150 * 203].view(150, 203), base[3:3 + 9 * 31 * 33].view(9, 31, 33), base[5:5 + 77777],
          base[:64 * 64].view(64, 64)]
    bc = gpu.BatchCompressor(xs, 1e-3, "rel", autotune=False, plan=plan)
    bc.run()
    sizes, stats = bc.results()
    for i, x in enumerate(xs):
        st, ref = _single(gpu, x, 1e-3, "rel")
        assert stats[i] == 0 and st == 0
        assert np.array_equal(bc.archives[i][:sizes[i]].cpu().numpy(), ref), i


@pytest.mark.parametrize("plan", PLANS)
def test_batch_errors_stay_per_field(gpu, plan):
    rng = np.random.default_rng(4)
    good = torch.from_numpy(rng.standard_normal((64, 70)).astype(np.float32).cumsum(1)).cuda()
    nan = good.clone()
    nan[3, 3] = float("nan")
    const = torch.full((50, 50), 2.5, device="cuda")
    big = torch.tensor([0.0, 1e7, 0.0], device="cuda")
    xs = [good, nan, const, big, good.clone()]
    bc = gpu.BatchCompressor(xs, [1e-3, 1e-3, 1e-3, 0.5, 1e-3], ["rel", "rel", "rel", "abs", "rel"], plan=plan,
                             autotune=False)
    bc.run()
    sizes, stats = bc.results()
    assert stats == [0, 2, 1, 3, 0]
    st, ref = _single(gpu, good, 1e-3, "rel")
    assert np.array_equal(bc.archives[0][:sizes[0]].cpu().numpy(), ref)
    assert np.array_equal(bc.archives[4][:sizes[4]].cpu().numpy(), ref)


@pytest.mark.parametrize("plan", PLANS)
def test_batch_learned_selector(gpu, orc, plan):
    from paper_2105_12912_gb300 import selector
    fields = _mixed_fields(5)
    xs = [torch.from_numpy(x).cuda() for x, _, _ in fields]
    w = selector.init_weights(2) * 2.0
    bc = gpu.BatchCompressor(xs, [e for _, e, _ in fields], [m for _, _, m in fields], select="learned", weights=w,
                             plan=plan, autotune=False)
    bc.run()
    sizes, stats = bc.results()
    for i, (x, eb, mode) in enumerate(fields):
        st, ref = orc.compress(x, orc.EB_REL if mode == "rel" else orc.EB_ABS, eb, select=orc.SEL_LEARNED,
                               mlp_w=w.cpu().numpy())
        assert stats[i] == st == 0
        assert np.array_equal(bc.archives[i][:sizes[i]].cpu().numpy(), ref), i


def test_batch_autotune_info(gpu):
    """The autotuner times both plans and keeps one; the archives do not depend on it."""
    fields = _mixed_fields(6)
    xs = [torch.from_numpy(x).cuda() for x, _, _ in fields]
    bc = gpu.BatchCompressor(xs, 1e-3, "abs")
    info = bc.info()
    assert info["construct_grid"] > 0 and info["tuned_ms"][0] > 0 and info["persist_ms"][0] > 0
    assert info["grid"] > 0
    bc.run()
    sizes, stats = bc.results()
    assert stats == [0] * len(xs)
    for i, x in enumerate(xs):
        st, ref = _single(gpu, x, 1e-3, "abs")
        assert st == 0 and np.array_equal(bc.archives[i][:sizes[i]].cpu().numpy(), ref), i


def test_batch_round_trip(gpu, orc):
    """Batched compression then batched decompression: every field bit-identical to
    the single-field decompression of the same archive, within the bound, and
    identical again after a replay with new data in the same buffers."""
    fields = _mixed_fields(7)
    xs = [torch.from_numpy(x).cuda() for x, _, _ in fields]
    bc = gpu.BatchCompressor(xs, [e for _, e, _ in fields], [m for _, _, m in fields])
    bd = gpu.BatchDecompressor(bc.archives, [tuple(x.shape) for x in xs])
    for rep in range(2):
        if rep == 1:
            for x in xs:
                x.mul_(-0.75).add_(3.0)
        bc.run()
        sizes, stats = bc.results()
        assert all(v == 0 for v in stats)
        bd.run()
        assert bd.results() == [0] * len(xs)
        for i, x in enumerate(xs):
            y, st = gpu.decompress(bc.archives[i], sizes[i])
            assert st == 0
            assert torch.equal(bd.outs[i].view(torch.int32), y.view(torch.int32)), (rep, i)
            eb_f = gpu.header(bc.archives[i])["eb_f"]
            assert float((x.double() - bd.outs[i].double()).abs().max()) <= eb_f


@pytest.mark.parametrize("nd", [1, 2, 3])
def test_batch_round_trip_common_dimensionality(gpu, orc, nd):
    """Batches whose fields share a dimensionality decode full Huffman blocks with the
    fused reconstruction (and the chunked set-up): bit-identical to the oracle's
    decompression of each archive, including edge blocks, run blocks, outliers and a
    field with more than 1024 codec blocks (several set-up chunks)."""
    rng = np.random.default_rng(40 + nd)
    shapes = {1: [(5000,), (4096 * 1100 + 17,), (1,), (70000,)],
              2: [(70, 131), (64, 64), (2200, 2100), (300, 301)],
              3: [(19, 23, 37), (16, 16, 16), (160, 130, 70), (40, 64, 64)]}[nd]
    xs, ebs, modes = [], [], []
    for i, sh in enumerate(shapes):
        x = rng.standard_normal(sh).astype(np.float32)
        for ax in range(len(sh)):
            x = np.cumsum(x, axis=ax).astype(np.float32)
        if i % 2 == 0:
            x[tuple(slice(0, max(1, s // 2)) for s in sh)] = 0.0
        xs.append(torch.from_numpy(x).cuda())
        ebs.append(1e-3 if x.size > 1 else 0.1)
        modes.append("rel" if x.size > 1 else "abs")
    bc = gpu.BatchCompressor(xs, ebs, modes, radius=64, autotune=False)  # small radius: outliers
    bc.run()
    sizes, stats = bc.results()
    assert all(v == 0 for v in stats)
    bd = gpu.BatchDecompressor(bc.archives, [tuple(x.shape) for x in xs], archive_bytes=sizes)
    bd.run()
    assert bd.results() == [0] * len(xs)
    for i, x in enumerate(xs):
        st, yr = orc.decompress(bc.archives[i][:sizes[i]].cpu().numpy(), x.numel())
        assert st == 0
        assert np.array_equal(bd.outs[i].cpu().numpy().ravel().view(np.uint32), yr.view(np.uint32)), i


def test_batch_decoder_tuning(gpu):
    """The decoder's CTA shape (8, 16 or 32 warps) never changes the output: after
    tuning, the batch decompression equals the single-field decompressions bit for
    bit, for a mixed batch and for one of a common dimensionality."""
    for fields in (_mixed_fields(11), _mixed_fields(12)[8:12]):
        xs = [torch.from_numpy(x).cuda() for x, _, _ in fields]
        bc = gpu.BatchCompressor(xs, [e for _, e, _ in fields], [m for _, _, m in fields], autotune=False)
        bc.run()
        sizes, stats = bc.results()
        assert all(v == 0 for v in stats)
        bd = gpu.BatchDecompressor(bc.archives, [tuple(x.shape) for x in xs], archive_bytes=sizes)
        warps, ms = bd.tune()
        assert warps in (8, 16, 32) and all(t > 0 for t in ms)
        bd.run()
        assert bd.results() == [0] * len(xs)
        for i in range(len(xs)):
            y, _ = gpu.decompress(bc.archives[i], sizes[i])
            assert torch.equal(bd.outs[i].view(torch.int32), y.view(torch.int32)), (warps, i)


def test_batch_decompress_bad_header_isolated(gpu):
    fields = _mixed_fields(8)[:6]
    xs = [torch.from_numpy(x).cuda() for x, _, _ in fields]
    bc = gpu.BatchCompressor(xs, [e for _, e, _ in fields], [m for _, _, m in fields], autotune=False)
    bc.run()
    sizes, _ = bc.results()
    bad = [a.clone() for a in bc.archives]
    bad[2][0] ^= 0xFF           # magic
    bad[4][64] ^= 0x01          # block count
    shapes = [tuple(x.shape) for x in xs]
    shapes[5] = tuple(int(d) + 1 for d in shapes[5])  # shape that does not match the header
    outs = [torch.empty(sh, device="cuda") for sh in shapes]
    bd = gpu.BatchDecompressor(bad, shapes, archive_bytes=sizes, outs=outs)
    bd.run()
    st = bd.results()
    assert st[2] == 4 and st[4] == 4 and st[5] == 4
    for i in (0, 1, 3):
        assert st[i] == 0
        y, _ = gpu.decompress(bc.archives[i], sizes[i])
        assert torch.equal(bd.outs[i].view(torch.int32), y.view(torch.int32))


@pytest.mark.parametrize("plan", PLANS)
def test_batch_traced_launches_match_graph(gpu, plan):
    """With tracing on, batch calls launch their kernels one by one (each with CUDA
    events); archives and reconstructions must equal the graph replays'."""
    fields = _mixed_fields(9)[:8]
    xs = [torch.from_numpy(x).cuda() for x, _, _ in fields]
    bc = gpu.BatchCompressor(xs, [e for _, e, _ in fields], [m for _, _, m in fields], autotune=False, plan=plan)
    bd = gpu.BatchDecompressor(bc.archives, [tuple(x.shape) for x in xs])
    bc.run()
    bd.run()
    sizes, stats = bc.results()
    assert stats == [0] * len(xs) and bd.results() == [0] * len(xs)
    ref_ar = [a[:n].clone() for a, n in zip(bc.archives, sizes)]
    ref_out = [o.clone() for o in bd.outs]
    gpu.trace_enable(True)
    try:
        gpu.trace_read(reset=True)
        bc.run()
        bd.run()
        torch.cuda.synchronize()
        tr = gpu.trace_read(reset=True)
    finally:
        gpu.trace_enable(False)
    sizes2, stats2 = bc.results()
    assert sizes2 == sizes and stats2 == stats and bd.results() == [0] * len(xs)
    for i in range(len(xs)):
        assert torch.equal(bc.archives[i][:sizes[i]], ref_ar[i])
        assert torch.equal(bd.outs[i].view(torch.int32), ref_out[i].view(torch.int32))
    comp = ("batch_persistent",) if plan == "persistent" else ("range", "construct", "codebook", "encode")
    for k in comp + ("dec_header", "dec_setup", "stream_decode", "reconstruct"):
        ms, cnt = tr[k]
        assert cnt == 1 and ms > 0, (k, tr[k])
    other = ("range", "construct", "codebook", "encode") if plan == "persistent" else ("batch_persistent",)
    for k in other:
        assert tr[k][1] == 0, (k, tr[k])


@pytest.mark.parametrize("plan", PLANS)
@pytest.mark.parametrize("nd", [1, 2, 3])
def test_batch_of_one_dimensionality(gpu, nd, plan):
    """A batch whose fields share their dimensionality runs the specialised
    construction kernel; archives must still equal the single-field calls'."""
    shapes = {1: [(5000,), (70001,), (4096,)], 2: [(70, 131), (64, 64), (300, 301)],
              3: [(19, 23, 37), (16, 16, 16), (40, 64, 64)]}[nd]
    rng = np.random.default_rng(10 + nd)
    xs = []
    for sh in shapes:
        x = rng.standard_normal(sh).astype(np.float32)
        for ax in range(len(sh)):
            x = np.cumsum(x, axis=ax).astype(np.float32)
        xs.append(torch.from_numpy(x).cuda())
    bc = gpu.BatchCompressor(xs, 1e-3, "rel", autotune=False, plan=plan)
    bc.run()
    sizes, stats = bc.results()
    for i, x in enumerate(xs):
        st, ref = _single(gpu, x, 1e-3, "rel")
        assert stats[i] == 0 and st == 0
        assert np.array_equal(bc.archives[i][:sizes[i]].cpu().numpy(), ref), i


def test_batch256_matches_single_field_calls_and_oracle(gpu, orc):
    """The real mixed batch (256 fields, seeds 100-355, 2.65e9 elements, 10.6 GB): every
    archive of the batched path, under the one-launch plan and the staged plan alike,
    equals the single-field call's byte for byte, and the largest 1-D, 2-D and 3-D
    fields equal the oracle's archives, with reconstructions bit-identical to the
    oracle's recurrence."""
    from paper_2105_12912_gb300 import synth
    specs = synth.workload_batch(256)
    xs = [synth.make_field(sp, "cuda") for sp in specs]
    caps = [min(gpu.max_archive_bytes(tuple(x.shape)), 6 * x.numel() + (1 << 20)) for x in xs]
    runs = {}
    for plan in PLANS:
        bc = gpu.BatchCompressor(xs, [sp.eb for sp in specs], [sp.eb_mode for sp in specs], archive_caps=caps,
                                 plan=plan, autotune=False)
        assert bc.info()["persistent"] == (plan == "persistent")
        bc.run()
        sizes, stats = bc.results()
        assert all(s == 0 for s in stats), (plan, stats)
        runs[plan] = (bc.archives, sizes)
        del bc.workspace
    sizes = runs["persistent"][1]
    assert runs["staged"][1] == sizes
    ws = gpu.Workspace(xs[0].device)
    arc = torch.empty(max(caps), dtype=torch.uint8, device="cuda")
    for i, (x, sp) in enumerate(zip(xs, specs)):
        ar, nb, _ = gpu.compress(x, sp.eb, sp.eb_mode, out=arc[:caps[i]], workspace=ws)
        assert nb == sizes[i], i
        for plan in PLANS:
            assert torch.equal(ar[:nb], runs[plan][0][i][:nb]), (plan, i)
    del arc, ws
    archives = runs["persistent"][0]
    largest = {}
    for i, x in enumerate(xs):
        nd = x.dim()
        if nd not in largest or x.numel() > xs[largest[nd]].numel():
            largest[nd] = i
    for nd, i in sorted(largest.items()):
        xh = xs[i].cpu().numpy()
        sp = specs[i]
        st, ref = orc.compress(xh, orc.EB_REL, sp.eb)
        assert st == 0
        assert ref.size == sizes[i] and np.array_equal(archives[i][:sizes[i]].cpu().numpy(), ref), (nd, i)
        y, _ = gpu.decompress(archives[i], sizes[i])
        st, yr = orc.decompress(ref, xh.size)
        assert np.array_equal(y.cpu().numpy().ravel().view(np.uint32), yr.view(np.uint32)), (nd, i)
