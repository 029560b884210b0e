"""Compression that returns the header, and decompression with no host round trip.

csz_compress_with_header must return exactly the device archive's first 128 bytes;
csz_decompress_async, given that host copy, must reconstruct bit-identically to
csz_decompress and report its status in a device word; a host copy that parses but
is not this archive's header must come back as CSZ_E_CORRUPT from the device check,
and one that does not parse must be refused on the host before any launch.
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


def _field(shape, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(shape).astype(np.float32)
    for ax in range(len(shape)):
        x = np.cumsum(x, axis=ax).astype(np.float32)
    return torch.from_numpy(x).cuda()


@pytest.mark.parametrize("shape", [(70001,), (130, 257), (20, 33, 47)])
def test_header_and_async_round_trip(gpu, shape):
    x = _field(shape, 1)
    ar, nb, hdr = gpu.compress_with_header(x, 1e-3, "rel")
    ar2, nb2, _ = gpu.compress(x, 1e-3, "rel")
    assert nb == nb2 and torch.equal(ar[:nb], ar2[:nb2])
    assert hdr == bytes(ar[:128].cpu().numpy().tobytes())
    ref, st = gpu.decompress(ar, nb)
    assert st == 0
    out = torch.full_like(x, float("nan"))
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    gpu.decompress_async(ar, nb, hdr, out, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert torch.equal(out.view(torch.int32), ref.view(torch.int32))


def test_async_back_to_back(gpu):
    """Several asynchronous decompressions in a row, one synchronisation at the end."""
    xs = [_field((64, 300), s) for s in range(3)]
    packs = [gpu.compress_with_header(x, 1e-4, "rel", out=torch.empty(1 << 20, dtype=torch.uint8, device="cuda"))
             for x in xs]
    outs = [torch.empty_like(x) for x in xs]
    status = torch.full((3,), -1, dtype=torch.int32, device="cuda")
    ws = gpu.Workspace(torch.device("cuda"))
    for i, (ar, nb, hdr) in enumerate(packs):
        gpu.decompress_async(ar, nb, hdr, outs[i], status[i:i + 1], workspace=ws)
    torch.cuda.synchronize()
    assert status.tolist() == [0, 0, 0]
    for i, (ar, nb, _) in enumerate(packs):
        ref, _ = gpu.decompress(ar, nb)
        assert torch.equal(outs[i].view(torch.int32), ref.view(torch.int32))


def test_async_header_of_another_archive_is_corrupt(gpu):
    x = _field((96, 200), 5)
    ar, nb, hdr = gpu.compress_with_header(x, 1e-3, "rel")
    forged = bytearray(hdr)
    forged[32] ^= 0x01  # the user's bound (parses, but is not this archive's header)
    out = torch.empty_like(x)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    gpu.decompress_async(ar, nb, bytes(forged), out, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 4  # CSZ_E_CORRUPT


def test_async_unparsable_header_refused_on_host(gpu):
    x = _field((5000,), 6)
    ar, nb, hdr = gpu.compress_with_header(x, 1e-3, "rel")
    bad = bytearray(hdr)
    bad[0] ^= 0xFF  # magic
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    with pytest.raises(RuntimeError):
        gpu.decompress_async(ar, nb, bytes(bad), torch.empty_like(x), status)
    torch.cuda.synchronize()
    assert int(status.item()) == -1  # nothing was launched
