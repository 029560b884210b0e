"""Failure path on the GPU without a fault: a bounded wait that nothing satisfies
(the look-back of a tile whose predecessor never publishes; an mbarrier phase no
copy completes; a field hand-over of the batched persistent kernel that no phase
releases) gives up, leaves the timeout status, and the kernel returns; the context
stays usable for the next compression."""
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


@pytest.mark.parametrize("which", [0, 1, 2])
def test_bounded_wait_reports_timeout(gpu, which):
    assert gpu.wait_selftest(which, spin_limit=500) == 7  # CSZ_E_TIMEOUT
    # the context is intact: an ordinary round trip still works
    x = torch.from_numpy(np.cumsum(np.random.default_rng(which).standard_normal(20000)).astype(np.float32)).cuda()
    ar, nb, st = gpu.compress(x, 1e-3, "rel")
    assert st == 0
    y, st = gpu.decompress(ar, nb)
    assert st == 0
    assert float((x.double() - y.double()).abs().max()) <= gpu.header(ar)["eb_f"]


def test_selftest_rejects_bad_arguments(gpu):
    assert gpu.wait_selftest(3) == 1  # CSZ_E_ARG
    assert gpu.wait_selftest(0, spin_limit=0) == 1
