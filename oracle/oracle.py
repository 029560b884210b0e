"""ctypes binding of the scalar C oracle.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py.  The product path (paper_2105_12912_gb300) never
imports this module, and this module never imports the product package.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK, E_ARG, E_NONFINITE, E_RANGE, E_CORRUPT, E_CAPACITY = range(6)
EB_ABS, EB_REL = 0, 1
SEL_HUFF, SEL_RLE, SEL_RLE_HUFF, SEL_HEURISTIC, SEL_EXHAUSTIVE, SEL_LEARNED = range(6)
CODEC_HUFF, CODEC_RLE, CODEC_RLE_HUFF = range(3)
MLP_PARAMS = 32 * 8 + 32 + 32 * 32 + 32 + 3 * 32 + 3
SLOTS = 4096

_lib = None

_u8p = C.POINTER(C.c_uint8)
_u16p = C.POINTER(C.c_uint16)
_u32p = C.POINTER(C.c_uint32)
_u64p = C.POINTER(C.c_uint64)
_i32p = C.POINTER(C.c_int32)
_f32p = C.POINTER(C.c_float)
_f64p = C.POINTER(C.c_double)


class OracleError(RuntimeError):
    def __init__(self, status, what=""):
        super().__init__(f"oracle {what} failed with status {status}")
        self.status = status


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        sig = {
            "orc_max_archive_bytes": (C.c_size_t, [C.c_int, _u64p]),
            "orc_compress": (C.c_int, [_f32p, C.c_int, _u64p, C.c_int, C.c_double, C.c_uint32, C.c_int,
                                       _f32p, _u8p, C.c_size_t, C.POINTER(C.c_size_t)]),
            "orc_decompress": (C.c_int, [_u8p, C.c_size_t, _f32p, C.c_uint64]),
            "orc_value_range": (C.c_int, [_f32p, C.c_uint64, _f32p, _f32p]),
            "orc_eb_params": (C.c_int, [C.c_int, C.c_double, C.c_float, C.c_float, _f64p, _f32p, _f32p, _f32p]),
            "orc_prequant": (C.c_int, [C.c_float, C.c_float, C.c_float, C.c_float, _i32p, C.POINTER(C.c_int)]),
            "orc_geometry": (C.c_int, [C.c_int, _u64p, _u64p, _u64p]),
            "orc_construct": (C.c_int, [_f32p, C.c_int, _u64p, C.c_float, C.c_float, C.c_float, C.c_uint32,
                                        _u16p, _u32p, _u32p, C.c_uint64, _u64p, _u32p]),
            "orc_run_stats": (C.c_int, [_u16p, C.c_int, _u64p, C.c_int, _u32p, _u32p, _u32p]),
            "orc_huffman_lengths": (C.c_int, [_u32p, C.c_int, _u8p]),
            "orc_canonical_codes": (C.c_int, [_u8p, C.c_int, _u64p]),
            "orc_block_sizes": (C.c_int, [_u16p, C.c_int, _u64p, C.c_uint32, _u8p, _u8p, _u8p, C.c_uint32, C.c_int,
                                          _u64p]),
            "orc_block_features": (C.c_int, [_u16p, C.c_int, _u64p, C.c_uint32, _f32p]),
            "orc_heuristic_pick": (C.c_int, [_u32p, C.c_int, C.c_uint32]),
            "orc_log2_q16": (C.c_uint32, [C.c_uint64]),
            "orc_mlp_forward": (None, [_f32p, _f32p, C.c_uint64, _f32p]),
            "orc_mlp_loss_grad_f64": (C.c_double, [_f32p, _f32p, _f32p, C.c_uint64, _f64p]),
            "orc_decode_codes": (C.c_int, [_u8p, C.c_size_t, _u16p, C.c_uint64]),
            "orc_selector_targets": (C.c_int, [_u64p, C.c_int, _u64p, _f32p, _u8p]),
            "orc_learned_pick": (C.c_int, [_f32p, _u64p]),
            "orc_compress_f64": (C.c_int, [_f64p, C.c_int, _u64p, C.c_int, C.c_double, C.c_uint32, C.c_int,
                                           _f32p, _u8p, C.c_size_t, C.POINTER(C.c_size_t)]),
            "orc_decompress_f64": (C.c_int, [_u8p, C.c_size_t, _f64p, C.c_uint64]),
            "orc_eb_params_f64": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_double, _f64p, _f64p, _f64p]),
            "orc_prequant_f64": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_double, _i32p]),
            "orc_compress_ex": (C.c_int, [_f32p, _f64p, C.c_int, _u64p, C.c_int, C.c_double, C.c_uint32, C.c_int,
                                          _f32p, C.c_int, _u8p, C.c_size_t, C.POINTER(C.c_size_t)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _dims(dims):
    d = np.zeros(3, dtype=np.uint64)
    d[: len(dims)] = dims
    return d


def geometry(dims):
    nb, ne = C.c_uint64(), C.c_uint64()
    st = lib().orc_geometry(len(dims), _p(_dims(dims), _u64p), C.byref(nb), C.byref(ne))
    if st:
        raise OracleError(st, "geometry")
    return nb.value, ne.value


def max_archive_bytes(dims):
    return int(lib().orc_max_archive_bytes(len(dims), _p(_dims(dims), _u64p)))


def compress(x: np.ndarray, eb_mode=EB_REL, eb=1e-4, radius=512, select=SEL_EXHAUSTIVE, mlp_w=None,
             raise_on_error=True):
    """Returns (status, archive bytes as np.uint8 array)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    dims = x.shape
    cap = max_archive_bytes(dims) if x.size else 1024
    out = np.zeros(max(cap, 1), dtype=np.uint8)
    nbytes = C.c_size_t(0)
    w = None if mlp_w is None else np.ascontiguousarray(mlp_w, dtype=np.float32)
    st = lib().orc_compress(_p(x, _f32p), x.ndim, _p(_dims(dims), _u64p), int(eb_mode), float(eb), int(radius),
                            int(select), None if w is None else _p(w, _f32p), _p(out, _u8p), out.size,
                            C.byref(nbytes))
    if st and raise_on_error:
        raise OracleError(st, "compress")
    return st, out[: nbytes.value].copy() if st == OK else out[:0]


def decompress(ar: np.ndarray, n: int, raise_on_error=True):
    ar = np.ascontiguousarray(ar, dtype=np.uint8)
    out = np.zeros(max(n, 1), dtype=np.float32)
    st = lib().orc_decompress(_p(ar, _u8p), ar.size, _p(out, _f32p), n)
    if st and raise_on_error:
        raise OracleError(st, "decompress")
    return st, out[:n]


def value_range(x):
    x = np.ascontiguousarray(x, dtype=np.float32).ravel()
    lo, hi = C.c_float(), C.c_float()
    st = lib().orc_value_range(_p(x, _f32p), x.size, C.byref(lo), C.byref(hi))
    return st, lo.value, hi.value


def eb_params(eb_mode, eb, vmin=0.0, vmax=0.0):
    ebd, ebf, x2, xr = C.c_double(), C.c_float(), C.c_float(), C.c_float()
    st = lib().orc_eb_params(int(eb_mode), float(eb), float(vmin), float(vmax), C.byref(ebd), C.byref(ebf),
                             C.byref(x2), C.byref(xr))
    return st, ebd.value, ebf.value, x2.value, xr.value


def prequant(x, eb_f, ebx2_f, ebx2_r):
    k, p = C.c_int32(), C.c_int()
    st = lib().orc_prequant(C.c_float(x), C.c_float(eb_f), C.c_float(ebx2_f), C.c_float(ebx2_r), C.byref(k),
                            C.byref(p))
    return st, k.value, p.value


def construct(x, eb_f, ebx2_f, ebx2_r, radius=512):
    """Returns dict(codes[nblk*4096] u16, keys u32, vals u32, hist[1024])."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    nblk, ne = geometry(x.shape)
    codes = np.zeros(nblk * SLOTS, dtype=np.uint16)
    cap = 2 * ne + 1
    keys = np.zeros(cap, dtype=np.uint32)
    vals = np.zeros(cap, dtype=np.uint32)
    nrec = C.c_uint64()
    hist = np.zeros(1024, dtype=np.uint32)
    st = lib().orc_construct(_p(x, _f32p), x.ndim, _p(_dims(x.shape), _u64p), C.c_float(eb_f), C.c_float(ebx2_f),
                             C.c_float(ebx2_r), int(radius), _p(codes, _u16p), _p(keys, _u32p), _p(vals, _u32p),
                             cap, C.byref(nrec), _p(hist, _u32p))
    if st:
        raise OracleError(st, "construct")
    n = nrec.value
    return {"codes": codes, "keys": keys[:n].copy(), "vals": vals[:n].copy(), "hist": hist, "nblk": nblk}


def run_stats(codes, dims, all_blocks=True):
    nblk, _ = geometry(dims)
    codes = np.ascontiguousarray(codes, dtype=np.uint16)
    vh = np.zeros(1024, dtype=np.uint32)
    lh = np.zeros(4096, dtype=np.uint32)
    nr = np.zeros(nblk, dtype=np.uint32)
    st = lib().orc_run_stats(_p(codes, _u16p), len(dims), _p(_dims(dims), _u64p), int(all_blocks), _p(vh, _u32p),
                             _p(lh, _u32p), _p(nr, _u32p))
    if st:
        raise OracleError(st, "run_stats")
    return vh, lh, nr


def huffman_lengths(freq):
    f = np.ascontiguousarray(freq, dtype=np.uint32)
    ln = np.zeros(f.size, dtype=np.uint8)
    st = lib().orc_huffman_lengths(_p(f, _u32p), f.size, _p(ln, _u8p))
    if st:
        raise OracleError(st, "huffman_lengths")
    return ln


def canonical_codes(lengths):
    ln = np.ascontiguousarray(lengths, dtype=np.uint8)
    code = np.zeros(ln.size, dtype=np.uint64)
    st = lib().orc_canonical_codes(_p(ln, _u8p), ln.size, _p(code, _u64p))
    if st:
        raise OracleError(st, "canonical_codes")
    return code


def block_sizes(codes, dims, radius, code_len, val_len, len_len, all_blocks=True):
    nblk, _ = geometry(dims)
    out = np.zeros((nblk, 3), dtype=np.uint64)
    c = np.ascontiguousarray(codes, dtype=np.uint16)
    a, b, d = (np.ascontiguousarray(v, dtype=np.uint8) for v in (code_len, val_len, len_len))
    st = lib().orc_block_sizes(_p(c, _u16p), len(dims), _p(_dims(dims), _u64p), int(radius), _p(a, _u8p),
                               _p(b, _u8p), _p(d, _u8p), 32, int(all_blocks), _p(out, _u64p))
    if st:
        raise OracleError(st, "block_sizes")
    return out


def block_features(codes, dims, radius=512):
    nblk, _ = geometry(dims)
    out = np.zeros((nblk, 8), dtype=np.float32)
    c = np.ascontiguousarray(codes, dtype=np.uint16)
    st = lib().orc_block_features(_p(c, _u16p), len(dims), _p(_dims(dims), _u64p), int(radius), _p(out, _f32p))
    if st:
        raise OracleError(st, "block_features")
    return out


def heuristic_pick(block_hist, m):
    h = np.ascontiguousarray(block_hist, dtype=np.uint32)
    return int(lib().orc_heuristic_pick(_p(h, _u32p), h.size, int(m)))


def log2_q16(v):
    return int(lib().orc_log2_q16(int(v)))


def mlp_forward(w, feat):
    w = np.ascontiguousarray(w, dtype=np.float32)
    f = np.ascontiguousarray(feat, dtype=np.float32).reshape(-1, 8)
    out = np.zeros((f.shape[0], 3), dtype=np.float32)
    lib().orc_mlp_forward(_p(w, _f32p), _p(f, _f32p), f.shape[0], _p(out, _f32p))
    return out


def mlp_loss_grad(w, feat, target):
    w = np.ascontiguousarray(w, dtype=np.float32)
    f = np.ascontiguousarray(feat, dtype=np.float32).reshape(-1, 8)
    t = np.ascontiguousarray(target, dtype=np.float32).reshape(-1, 3)
    g = np.zeros(MLP_PARAMS, dtype=np.float64)
    loss = lib().orc_mlp_loss_grad_f64(_p(w, _f32p), _p(f, _f32p), _p(t, _f32p), f.shape[0], _p(g, _f64p))
    return float(loss), g


def selector_targets(sizes, dims):
    """Training targets (log2 bits per element, Q16-exact) and the run-eligible mask."""
    nblk, _ = geometry(dims)
    sz = np.ascontiguousarray(sizes, dtype=np.uint64).reshape(nblk, 3)
    tgt = np.zeros((nblk, 3), dtype=np.float32)
    valid = np.zeros(nblk, dtype=np.uint8)
    st = lib().orc_selector_targets(_p(sz, _u64p), len(dims), _p(_dims(dims), _u64p), _p(tgt, _f32p),
                                    _p(valid, _u8p))
    if st:
        raise OracleError(st, "selector_targets")
    return tgt, valid


def learned_pick(y, sizes):
    yy = np.ascontiguousarray(y, dtype=np.float32).reshape(3)
    s = np.ascontiguousarray(sizes, dtype=np.uint64).reshape(3)
    return int(lib().orc_learned_pick(_p(yy, _f32p), _p(s, _u64p)))


def decode_codes(ar, dims):
    nblk, _ = geometry(dims)
    ar = np.ascontiguousarray(ar, dtype=np.uint8)
    codes = np.zeros(nblk * SLOTS, dtype=np.uint16)
    st = lib().orc_decode_codes(_p(ar, _u8p), ar.size, _p(codes, _u16p), codes.size)
    if st:
        raise OracleError(st, "decode_codes")
    return codes


def parse_header(ar):
    """Header fields of an archive (plain struct unpacking; used by tests)."""
    import struct
    b = bytes(np.asarray(ar[:128], dtype=np.uint8))
    magic, ver, ndim, mode = struct.unpack_from("<IHBB", b, 0)
    dims = struct.unpack_from("<3Q", b, 8)
    eb_user, eb_d = struct.unpack_from("<2d", b, 32)
    eb_f, = struct.unpack_from("<f", b, 48)
    radius, lanes, flags = struct.unpack_from("<3I", b, 52)
    nblk, nrec, nout, npatch, payload, total = struct.unpack_from("<6Q", b, 64)
    select, nh, nr, nrh = struct.unpack_from("<4I", b, 112)
    return dict(magic=magic, version=ver, ndim=ndim, eb_mode=mode, dims=dims[:ndim], eb_user=eb_user, eb_d=eb_d,
                eb_f=eb_f, radius=radius, lanes=lanes, flags=flags, nblk=nblk, n_rec=nrec, n_out=nout,
                n_patch=npatch, payload=payload, total=total, select=select, n_codec=(nh, nr, nrh))


def sections(ar):
    """Split an archive into its sections (tests)."""
    h = parse_header(ar)
    a8 = lambda v: (v + 7) & ~7
    nblk = h["nblk"]
    off_bb = 128 + a8(nblk)
    off_rec = off_bb + a8(4 * nblk)
    off_pay = off_rec + 8 * h["n_rec"]
    off_books = off_pay + a8(h["payload"])
    ar = np.asarray(ar, dtype=np.uint8)
    rec = ar[off_rec:off_pay].view(np.uint32).reshape(-1, 2) if h["n_rec"] else np.zeros((0, 2), np.uint32)
    return dict(header=h, codec=ar[128:128 + nblk], blk_bytes=ar[off_bb:off_bb + 4 * nblk].view(np.uint32),
                records=rec, payload=ar[off_pay:off_pay + h["payload"]], books=ar[off_books:h["total"]])


# ---- double-precision fields ----------------------------------------------------------
FLAG_F64 = 4


def compress_f64(x: np.ndarray, eb_mode=EB_REL, eb=1e-4, radius=512, select=SEL_EXHAUSTIVE, mlp_w=None,
                 raise_on_error=True):
    """Double-precision field -> (status, archive bytes as np.uint8 array)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    dims = x.shape
    cap = max_archive_bytes(dims) if x.size else 1024
    out = np.zeros(max(cap, 1), dtype=np.uint8)
    nbytes = C.c_size_t(0)
    w = None if mlp_w is None else np.ascontiguousarray(mlp_w, dtype=np.float32)
    st = lib().orc_compress_f64(_p(x, _f64p), x.ndim, _p(_dims(dims), _u64p), int(eb_mode), float(eb), int(radius),
                                int(select), None if w is None else _p(w, _f32p), _p(out, _u8p), out.size,
                                C.byref(nbytes))
    if st and raise_on_error:
        raise OracleError(st, "compress_f64")
    return st, out[: nbytes.value].copy() if st == 0 else None


def decompress_f64(ar: np.ndarray, n: int, raise_on_error=True):
    ar = np.ascontiguousarray(ar, dtype=np.uint8)
    out = np.zeros(max(n, 1), dtype=np.float64)
    st = lib().orc_decompress_f64(_p(ar, _u8p), ar.size, _p(out, _f64p), n)
    if st and raise_on_error:
        raise OracleError(st, "decompress_f64")
    return st, out[:n]


def eb_params_f64(eb_mode, eb, vmin=0.0, vmax=0.0):
    """(status, eb_d, step, rstep)"""
    ebd, step, rstep = C.c_double(), C.c_double(), C.c_double()
    st = lib().orc_eb_params_f64(int(eb_mode), float(eb), float(vmin), float(vmax), C.byref(ebd), C.byref(step),
                                 C.byref(rstep))
    return st, ebd.value, step.value, rstep.value


def prequant_f64(x, eb_d, step, rstep):
    """(status, k)"""
    k = C.c_int32()
    st = lib().orc_prequant_f64(float(x), float(eb_d), float(step), float(rstep), C.byref(k))
    return st, k.value


# ---- general entry (FP32 or double; chunked or global Lorenzo) ------------------------
FLAG_GLOBAL = 8


def compress_ex(x: np.ndarray, eb_mode=EB_REL, eb=1e-4, radius=512, select=SEL_EXHAUSTIVE, mlp_w=None,
                global_lorenzo=False, raise_on_error=True):
    """(status, archive) for an FP32 or float64 field; global_lorenzo selects the
    unchunked predictor (archive flag FLAG_GLOBAL)."""
    f64 = np.asarray(x).dtype == np.float64
    x = np.ascontiguousarray(x, dtype=np.float64 if f64 else np.float32)
    dims = x.shape
    cap = max_archive_bytes(dims) if x.size else 1024
    out = np.zeros(max(cap, 1), dtype=np.uint8)
    nbytes = C.c_size_t(0)
    w = None if mlp_w is None else np.ascontiguousarray(mlp_w, dtype=np.float32)
    st = lib().orc_compress_ex(None if f64 else _p(x, _f32p), _p(x, _f64p) if f64 else None, x.ndim,
                               _p(_dims(dims), _u64p), int(eb_mode), float(eb), int(radius), int(select),
                               None if w is None else _p(w, _f32p), 1 if global_lorenzo else 0, _p(out, _u8p),
                               out.size, C.byref(nbytes))
    if st and raise_on_error:
        raise OracleError(st, "compress_ex")
    return st, out[: nbytes.value].copy() if st == 0 else None
