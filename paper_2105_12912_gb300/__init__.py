"""cszp: GB300-native error-bounded lossy compressor (cuSZ+ data-parallel path).

    from paper_2105_12912_gb300 import api
    archive, nbytes, _ = api.compress(field_cuda_f32, eb=1e-4, eb_mode="rel")
    field, _ = api.decompress(archive, nbytes)

The compute path is libcszp.so (hand-written sm_103a kernels behind a C ABI, see
include/cszp.h); this package is its thin ctypes binding plus seeded synthetic
field generators (synth).
"""
__all__ = ["api", "synth"]
