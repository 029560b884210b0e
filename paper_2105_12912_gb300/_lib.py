"""ctypes loader of libcszp.so (the CUDA library).  No fallback: if the library is
missing the import of the binding fails with a message saying how to build it."""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libcszp.so")

OK, E_ARG, E_NONFINITE, E_RANGE, E_CORRUPT, E_CAPACITY, E_CUDA, E_TIMEOUT = range(8)
STATUS_NAMES = ["ok", "E_ARG", "E_NONFINITE", "E_RANGE", "E_CORRUPT", "E_CAPACITY", "E_CUDA", "E_TIMEOUT"]


class csz_options(C.Structure):
    _fields_ = [("radius", C.c_uint32), ("select", C.c_uint32), ("selector_weights", C.c_void_p),
                ("flags", C.c_uint32), ("reserved", C.c_uint32 * 3)]


class csz_field(C.Structure):
    _fields_ = [("d_field", C.c_void_p), ("ndim", C.c_int), ("dims", C.c_uint64 * 3), ("eb_mode", C.c_int),
                ("eb", C.c_double), ("d_archive", C.c_void_p), ("archive_cap", C.c_size_t)]


class csz_dfield(C.Structure):
    _fields_ = [("d_archive", C.c_void_p), ("archive_bytes", C.c_size_t), ("d_out", C.c_void_p),
                ("out_cap_elems", C.c_uint64), ("ndim", C.c_int), ("dims", C.c_uint64 * 3)]


class CszError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{what}: {name}")
        self.status = status


_lib = None

# name -> (restype, argtypes); the exported C ABI of include/cszp.h
SIGNATURES = {
    "csz_max_archive_bytes": (C.c_size_t, [C.c_int, C.POINTER(C.c_uint64)]),
    "csz_workspace_bytes": (C.c_size_t, [C.c_int, C.POINTER(C.c_uint64)]),
    "csz_compress": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_uint64), C.c_int, C.c_double,
                               C.POINTER(csz_options), C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t,
                               C.POINTER(C.c_size_t), C.c_void_p]),
    "csz_archive_info": (C.c_int, [C.c_void_p, C.c_size_t, C.POINTER(C.c_int), C.POINTER(C.c_uint64),
                                   C.POINTER(C.c_double), C.POINTER(C.c_uint64)]),
    "csz_decompress": (C.c_int, [C.c_void_p, C.c_size_t, C.c_void_p, C.c_uint64, C.c_void_p, C.c_size_t,
                                 C.c_void_p]),
    "csz_compress_with_header": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_uint64), C.c_int, C.c_double,
                                           C.POINTER(csz_options), C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t,
                                           C.POINTER(C.c_size_t), C.c_void_p, C.c_void_p]),
    "csz_decompress_async": (C.c_int, [C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p,
                                       C.c_size_t, C.c_void_p, C.c_void_p]),
    "csz_compress_f64": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_uint64), C.c_int, C.c_double,
                                   C.POINTER(csz_options), C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t,
                                   C.POINTER(C.c_size_t), C.c_void_p]),
    "csz_decompress_f64": (C.c_int, [C.c_void_p, C.c_size_t, C.c_void_p, C.c_uint64, C.c_void_p, C.c_size_t,
                                     C.c_void_p]),
    "csz_archive_elem_bytes": (C.c_int, [C.c_void_p, C.c_size_t]),
    "csz_wait_selftest": (C.c_int, [C.c_int, C.c_uint32, C.c_void_p, C.c_size_t, C.c_void_p]),
    "csz_decompress_static": (C.c_int, [C.c_void_p, C.c_size_t, C.c_void_p, C.c_uint64, C.c_void_p]),
    "csz_selector_rows": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_uint64), C.c_int, C.c_double, C.c_uint32,
                                    C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p]),
    "csz_selector_workspace_bytes": (C.c_size_t, [C.c_uint64]),
    "csz_selector_predict": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]),
    "csz_selector_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p,
                                    C.POINTER(C.c_double), C.c_void_p, C.c_size_t, C.c_void_p]),
    "csz_selector_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint32,
                                     C.c_float, C.c_void_p, C.c_size_t, C.POINTER(C.c_double), C.c_void_p]),
    "csz_batch_workspace_bytes": (C.c_size_t, [C.c_int, C.POINTER(csz_field)]),
    "csz_batch_create": (C.c_int, [C.c_int, C.POINTER(csz_field), C.POINTER(csz_options), C.c_void_p, C.c_size_t,
                                   C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
    "csz_batch_compress": (C.c_int, [C.c_void_p, C.c_void_p]),
    "csz_batch_results": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_int), C.c_void_p]),
    "csz_batch_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "csz_batch_plan": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "csz_batch_destroy": (None, [C.c_void_p]),
    "csz_batch_last_error": (C.c_char_p, []),
    "csz_batch_dec_workspace_bytes": (C.c_size_t, [C.c_int, C.POINTER(csz_dfield)]),
    "csz_batch_dec_tune": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "csz_batch_dec_create": (C.c_int, [C.c_int, C.POINTER(csz_dfield), C.c_void_p, C.c_size_t, C.c_void_p,
                                       C.POINTER(C.c_void_p)]),
    "csz_batch_decompress": (C.c_int, [C.c_void_p, C.c_void_p]),
    "csz_batch_dec_results": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.c_void_p]),
    "csz_batch_dec_destroy": (None, [C.c_void_p]),
    "csz_status_string": (C.c_char_p, [C.c_int]),
    "csz_kernel_count": (C.c_int, []),
    "csz_kernel_name": (C.c_char_p, [C.c_int]),
    "csz_trace_enable": (C.c_int, [C.c_int]),
    "csz_trace_read": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_uint64), C.c_int]),
}


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libcszp.so not found at {LIB_PATH}; build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def dims_array(dims):
    d = (C.c_uint64 * 3)()
    for i, v in enumerate(dims):
        d[i] = int(v)
    return d
