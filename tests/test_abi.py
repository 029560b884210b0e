"""The C-ABI library loads without a GPU and exports every function the public
headers declare; host-only calls (sizes, status names, header parsing) work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2105_12912_gb300 import build
    build.build()
    from paper_2105_12912_gb300 import _lib
    return _lib.lib()


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(csz_[a-z0-9_]+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert {"csz_compress", "csz_decompress", "csz_archive_info", "csz_max_archive_bytes",
            "csz_workspace_bytes", "csz_status_string"} <= names
    for n in sorted(names):
        assert hasattr(L, n), n


def test_sizes_and_status(L):
    from paper_2105_12912_gb300 import _lib
    d = _lib.dims_array((1800, 3600))
    assert L.csz_max_archive_bytes(2, d) > 0
    ws = L.csz_workspace_bytes(2, d)
    nblk = 29 * 57
    assert ws >= nblk * 4096 * 2
    assert L.csz_workspace_bytes(2, _lib.dims_array((0, 5))) == 0
    assert L.csz_max_archive_bytes(4, d) == 0
    assert L.csz_status_string(0) == b"ok"
    assert L.csz_status_string(4) == b"corrupt archive"


def test_archive_info_reads_oracle_header(L, orc):
    x = np.random.default_rng(0).standard_normal((33, 65)).astype(np.float32)
    st, ar = orc.compress(x, orc.EB_REL, 1e-3)
    from paper_2105_12912_gb300 import api
    dims, eb, tot = api.archive_info(bytes(ar[:128]))
    h = orc.parse_header(ar)
    assert dims == (33, 65) and eb == h["eb_d"] and tot == ar.size
    bad = bytearray(ar[:128])
    bad[0] ^= 1
    with pytest.raises(Exception):
        api.archive_info(bytes(bad))


def test_no_gpu_calls_fail_cleanly(L):
    """Without a device the compute entry points return a status instead of crashing."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2105_12912_gb300 import _lib
    d = _lib.dims_array((64,))
    nb = C.c_size_t()
    st = L.csz_compress(None, 1, d, 1, 1e-3, None, None, 0, None, 0, C.byref(nb), None)
    assert st == 1  # null pointers are rejected before any CUDA call


def test_async_and_selftest_argument_checks_need_no_device(L, orc):
    """The asynchronous decompression parses its host header copy before any launch:
    missing pointers are CSZ_E_ARG, a copy that does not parse (or disagrees with the
    byte count) is CSZ_E_CORRUPT, all without touching a device.  The wait self-test
    rejects bad arguments the same way."""
    import numpy as np
    x = np.cumsum(np.random.default_rng(5).standard_normal(5000)).astype(np.float32)
    st, ar = orc.compress(x, orc.EB_REL, 1e-3)
    assert st == 0
    hdr = (C.c_uint8 * 128).from_buffer_copy(bytes(ar[:128]))
    fake = C.c_void_p(0x1000)  # never dereferenced: every case below fails on the host
    status = C.c_void_p(0x2000)
    # missing pointers
    assert L.csz_decompress_async(None, ar.size, hdr, fake, 5000, fake, 1 << 20, status, None) == 1
    assert L.csz_decompress_async(fake, ar.size, None, fake, 5000, fake, 1 << 20, status, None) == 1
    assert L.csz_decompress_async(fake, ar.size, hdr, fake, 5000, fake, 1 << 20, None, None) == 1
    # a header copy that does not parse, or does not fit the byte count
    bad = bytearray(ar[:128])
    bad[0] ^= 0xFF
    badh = (C.c_uint8 * 128).from_buffer_copy(bytes(bad))
    assert L.csz_decompress_async(fake, ar.size, badh, fake, 5000, fake, 1 << 20, status, None) == 4
    assert L.csz_decompress_async(fake, ar.size - 1, hdr, fake, 5000, fake, 1 << 20, status, None) == 4
    # output or workspace too small
    assert L.csz_decompress_async(fake, ar.size, hdr, fake, 4999, fake, 1 << 20, status, None) == 5
    assert L.csz_decompress_async(fake, ar.size, hdr, fake, 5000, fake, 16, status, None) == 5
    # the self-test's argument checks
    assert L.csz_wait_selftest(3, 100, fake, 512, None) == 1
    assert L.csz_wait_selftest(0, 0, fake, 512, None) == 1
    assert L.csz_wait_selftest(0, 100, fake, 64, None) == 1
    assert L.csz_wait_selftest(0, 100, None, 512, None) == 1
