"""csz_decompress_static: decompression for callers that cannot allocate device memory.

Such callers (an I/O filter plug-in handed only its input and output buffers, or an
application whose device memory is all held by its own pool) cannot provide the
workspace csz_decompress needs; this entry point runs on a scratch array the library
holds instead.  These tests call it through the C ABI and compare it with
csz_decompress, bit for bit (the tolerance of every other reconstruction test), on
two calls in a row.  The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_12912_gb300 import api as A
    return A


def _static(lib, ar, nb, out):
    st = lib.csz_decompress_static(C.c_void_p(ar.data_ptr()), nb, C.c_void_p(out.data_ptr()), out.numel(),
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st


@pytest.mark.parametrize("shape", [(262144,), (300, 200), (40, 40, 40), (1,), (65, 63)])
def test_static_matches_workspace_decompress(api, shape):
    from paper_2105_12912_gb300 import _lib
    lib = _lib.lib()
    rng = np.random.default_rng(sum(shape))
    x = rng.standard_normal(shape).astype(np.float32).cumsum(axis=-1).astype(np.float32)
    x[..., : max(1, shape[-1] // 3)] = 0.0
    xd = torch.from_numpy(x).cuda()
    mode = "abs" if x.size == 1 else "rel"
    ar, nb, _ = api.compress(xd, 1e-3, mode)
    ref, st = api.decompress(ar, nb)
    torch.cuda.synchronize()
    assert st == 0
    # a different archive in between, so the shared array holds another call's data
    other = torch.from_numpy(rng.standard_normal(4096).astype(np.float32)).cuda()
    oar, onb, _ = api.compress(other, 1e-2)
    for _ in range(2):
        out = torch.full_like(xd, float("nan"))
        assert _static(lib, ar, nb, out) == 0
        assert torch.equal(out.view(torch.int32), ref.view(torch.int32))
        oout = torch.empty_like(other)
        assert _static(lib, oar, onb, oout) == 0


@pytest.mark.parametrize("over,at", [
    ((64 * 4096 + 1,), (64 * 4096,)),            # 1-D: 65 blocks / 64 blocks
    ((512, 576), (512, 512)),                    # 2-D: 8 x 9 = 72 blocks / 8 x 8 = 64
    ((64, 64, 65), (64, 64, 64)),                # 3-D: 4 x 4 x 5 = 80 blocks / 4^3 = 64
    ((16, 16, 1040), (16, 16, 1024)),            # 3-D: 1 x 1 x 65 / 1 x 1 x 64
])
def test_static_block_limit(api, over, at):
    """One block over the 64-block limit is refused with CSZ_E_CAPACITY before any
    device work; exactly 64 blocks decompress, bit-identical to csz_decompress."""
    from paper_2105_12912_gb300 import _lib
    lib = _lib.lib()
    n = int(np.prod(over))
    x = torch.linspace(0, 1, n, device="cuda").reshape(over)
    ar, nb, _ = api.compress(x, 1e-3)
    out = torch.empty_like(x)
    assert _static(lib, ar, nb, out) == 5  # CSZ_E_CAPACITY
    n = int(np.prod(at))
    y = torch.linspace(0, 1, n, device="cuda").reshape(at)
    ar, nb, _ = api.compress(y, 1e-3)
    out = torch.full_like(y, float("nan"))
    assert _static(lib, ar, nb, out) == 0
    ref, _ = api.decompress(ar, nb)
    assert torch.equal(out.view(torch.int32), ref.view(torch.int32))
