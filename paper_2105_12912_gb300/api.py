"""Python binding of the cszp C ABI (argument marshalling only).

PyTorch provides device memory and streams; every step of compression and
decompression runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
from functools import lru_cache

import torch

from . import _lib as L

EB_MODES = {"abs": 0, "rel": 1}
SELECT = {"huff": 0, "rle": 1, "rle_huff": 2, "heuristic": 3, "exhaustive": 4, "learned": 5}
CODECS = ("huff", "rle", "rle_huff")
MLP_PARAMS = 1443


def _check(st: int, what: str):
    if st != L.OK:
        raise L.CszError(st, what)


def _stream_ptr(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# per-shape values and marshalled argument blocks are kept, so a call on a shape seen
# before spends no time on them (the C side only reads them)
@lru_cache(maxsize=1024)
def _dims_c(dims: tuple):
    return L.dims_array(dims)


@lru_cache(maxsize=1024)
def _max_archive_bytes(dims: tuple) -> int:
    return int(L.lib().csz_max_archive_bytes(len(dims), _dims_c(dims)))


@lru_cache(maxsize=1024)
def _workspace_bytes(dims: tuple) -> int:
    return int(L.lib().csz_workspace_bytes(len(dims), _dims_c(dims)))


def max_archive_bytes(dims) -> int:
    return _max_archive_bytes(tuple(int(d) for d in dims))


def workspace_bytes(dims) -> int:
    return _workspace_bytes(tuple(int(d) for d in dims))


_opt_cache = {}


FLAG_GLOBAL_LORENZO = 1


def _options(radius, select, weights, flags=0):
    if weights is not None:
        if not (weights.is_cuda and weights.dtype == torch.float32 and weights.numel() == MLP_PARAMS):
            raise ValueError("weights must be a float32 CUDA tensor of 1443 parameters")
    key = (int(radius), SELECT[select] if isinstance(select, str) else int(select),
           weights.data_ptr() if weights is not None else 0, int(flags))
    opt = _opt_cache.get(key)
    if opt is None:
        opt = L.csz_options()
        opt.radius, opt.select, opt.flags = key[0], key[1], key[3]
        if weights is not None:
            opt.selector_weights = C.c_void_p(key[2])
        _opt_cache[key] = opt
    return opt


class Workspace:
    """Device scratch for one stream, grown on demand and reused across calls."""

    def __init__(self, device=None):
        self.device = torch.device(device or "cuda")
        self.buf = None

    def get(self, nbytes: int) -> torch.Tensor:
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        return self.buf


_default_ws = {}


def _ws(device, ws):
    if ws is not None:
        return ws
    key = torch.device(device).index
    if key not in _default_ws:
        _default_ws[key] = Workspace(device)
    return _default_ws[key]


def compress(field: torch.Tensor, eb: float, eb_mode: str = "rel", radius: int = 512,
             select: str = "exhaustive", weights: torch.Tensor | None = None, out: torch.Tensor | None = None,
             workspace: Workspace | None = None, stream=None, raise_on_error: bool = True,
             global_lorenzo: bool = False):
    """Compress a contiguous FP32 or float64 CUDA tensor (1-3 dims; float64 goes to
    csz_compress_f64).  Returns (archive, nbytes, status): archive is a uint8 CUDA
    tensor whose first nbytes bytes hold the archive."""
    if not (field.is_cuda and field.dtype in (torch.float32, torch.float64) and field.is_contiguous()):
        raise ValueError("field must be a contiguous float32 or float64 CUDA tensor")
    dims = tuple(field.shape)
    if out is None:
        out = torch.empty(max_archive_bytes(dims) or 1, dtype=torch.uint8, device=field.device)
    ws = _ws(field.device, workspace).get(workspace_bytes(dims) or 256)
    opt = _options(radius, select, weights, FLAG_GLOBAL_LORENZO if global_lorenzo else 0)
    nbytes = C.c_size_t(0)
    fn = L.lib().csz_compress_f64 if field.dtype == torch.float64 else L.lib().csz_compress
    st = fn(C.c_void_p(field.data_ptr()), len(dims), _dims_c(dims),
                              EB_MODES[eb_mode] if isinstance(eb_mode, str) else int(eb_mode), float(eb),
                              C.byref(opt), C.c_void_p(ws.data_ptr()), ws.numel(), C.c_void_p(out.data_ptr()),
                              out.numel(), C.byref(nbytes), _stream_ptr(stream))
    if raise_on_error:
        _check(st, "csz_compress")
    return out, int(nbytes.value), st


def archive_info(archive_host_head: bytes):
    """(dims, eb_abs, total_bytes) from the first 128 bytes of an archive."""
    buf = (C.c_uint8 * len(archive_host_head)).from_buffer_copy(archive_host_head)
    nd = C.c_int()
    dims = (C.c_uint64 * 3)()
    eb = C.c_double()
    tot = C.c_uint64()
    st = L.lib().csz_archive_info(C.cast(buf, C.c_void_p), len(archive_host_head), C.byref(nd), dims,
                                  C.byref(eb), C.byref(tot))
    _check(st, "csz_archive_info")
    return tuple(int(dims[i]) for i in range(nd.value)), float(eb.value), int(tot.value)


def decompress(archive: torch.Tensor, nbytes: int | None = None, out: torch.Tensor | None = None,
               dims=None, workspace: Workspace | None = None, stream=None, raise_on_error: bool = True):
    """Decompress a uint8 CUDA archive.  Returns (field, status)."""
    if not (archive.is_cuda and archive.dtype == torch.uint8):
        raise ValueError("archive must be a uint8 CUDA tensor")
    if nbytes is None:
        nbytes = archive.numel()
    if dims is None or out is None:
        head = bytes(archive[:128].cpu().numpy().tobytes())
        if dims is None:
            dims, _, _ = archive_info(head)
        if out is None:
            esz = elem_bytes(head)
            out = torch.empty(tuple(dims), dtype=torch.float64 if esz == 8 else torch.float32,
                              device=archive.device)
    ws = _ws(archive.device, workspace).get(workspace_bytes(dims) or 256)
    f64 = out.dtype == torch.float64
    fn = L.lib().csz_decompress_f64 if f64 else L.lib().csz_decompress
    st = fn(C.c_void_p(archive.data_ptr()), int(nbytes), C.c_void_p(out.data_ptr()), out.numel(),
            C.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream))
    if raise_on_error:
        _check(st, "csz_decompress_f64" if f64 else "csz_decompress")
    return out, st


def elem_bytes(archive_host_head: bytes) -> int:
    """4 (FP32) or 8 (double) for the field an archive holds; 0 if the header is invalid."""
    buf = (C.c_uint8 * len(archive_host_head)).from_buffer_copy(archive_host_head)
    return int(L.lib().csz_archive_elem_bytes(C.cast(buf, C.c_void_p), len(archive_host_head)))


def compress_with_header(field: torch.Tensor, eb: float, eb_mode: str = "rel", radius: int = 512,
                         select: str = "exhaustive", weights: torch.Tensor | None = None,
                         out: torch.Tensor | None = None, workspace: Workspace | None = None, stream=None,
                         global_lorenzo: bool = False):
    """compress() that also returns the archive's 128-byte header as bytes (copied in
    the same synchronisation), for decompress_async.  Returns (archive, nbytes, header)."""
    if not (field.is_cuda and field.dtype == torch.float32 and field.is_contiguous()):
        raise ValueError("field must be a contiguous float32 CUDA tensor")
    dims = tuple(field.shape)
    if out is None:
        out = torch.empty(max_archive_bytes(dims) or 1, dtype=torch.uint8, device=field.device)
    ws = _ws(field.device, workspace).get(workspace_bytes(dims) or 256)
    opt = _options(radius, select, weights, FLAG_GLOBAL_LORENZO if global_lorenzo else 0)
    nbytes = C.c_size_t(0)
    hdr = (C.c_uint8 * 128)()
    st = L.lib().csz_compress_with_header(
        C.c_void_p(field.data_ptr()), len(dims), _dims_c(dims),
        EB_MODES[eb_mode] if isinstance(eb_mode, str) else int(eb_mode), float(eb), C.byref(opt),
        C.c_void_p(ws.data_ptr()), ws.numel(), C.c_void_p(out.data_ptr()), out.numel(), C.byref(nbytes), hdr,
        _stream_ptr(stream))
    _check(st, "csz_compress_with_header")
    return out, int(nbytes.value), bytes(hdr)


def decompress_async(archive: torch.Tensor, nbytes: int, header_bytes: bytes, out: torch.Tensor,
                     status: torch.Tensor, workspace: Workspace | None = None, stream=None) -> None:
    """Decompress without host synchronisation: the archive's header comes from the
    host copy `header_bytes` (128 bytes), the outcome lands in `status` (an int32 CUDA
    tensor of one element, a csz_status value) when the stream reaches it."""
    if not (archive.is_cuda and archive.dtype == torch.uint8):
        raise ValueError("archive must be a uint8 CUDA tensor")
    if not (status.is_cuda and status.dtype == torch.int32 and status.numel() >= 1):
        raise ValueError("status must be an int32 CUDA tensor")
    if len(header_bytes) < 128:
        raise ValueError("header_bytes must hold the archive's 128-byte header")
    hb = (C.c_uint8 * 128).from_buffer_copy(bytes(header_bytes[:128]))
    ws = _ws(archive.device, workspace).get(workspace_bytes(tuple(out.shape)) or 256)
    st = L.lib().csz_decompress_async(C.c_void_p(archive.data_ptr()), int(nbytes), hb, C.c_void_p(out.data_ptr()),
                                      out.numel(), C.c_void_p(ws.data_ptr()), ws.numel(),
                                      C.c_void_p(status.data_ptr()), _stream_ptr(stream))
    _check(st, "csz_decompress_async")


def wait_selftest(which: int, spin_limit: int = 1000, stream=None) -> int:
    """Run one bounded wait that nothing satisfies (0: look-back, 1: mbarrier) and
    return the resulting status (CSZ_E_TIMEOUT = 7 when the wait gave up)."""
    scratch = torch.empty(512, dtype=torch.uint8, device="cuda")
    return int(L.lib().csz_wait_selftest(int(which), int(spin_limit), C.c_void_p(scratch.data_ptr()),
                                         scratch.numel(), _stream_ptr(stream)))


def header(archive) -> dict:
    """Parsed 128-byte archive header (from a CUDA/CPU uint8 tensor or bytes)."""
    import struct
    if isinstance(archive, torch.Tensor):
        archive = bytes(archive[:128].cpu().numpy().tobytes())
    b = bytes(archive[:128])
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


# ---------------------------------------------------------------------------------
# batched compression (one launch per stage for all fields, replayed as a CUDA graph)
# ---------------------------------------------------------------------------------
BATCH_AUTOTUNE, BATCH_STAGED, BATCH_PERSISTENT = 1, 2, 4
BATCH_PLANS = {"auto": 0, "staged": BATCH_STAGED, "persistent": BATCH_PERSISTENT}


class BatchCompressor:
    """Compresses a fixed list of device fields together.  Construction lays out the
    workspace, uploads the per-field tables, chooses the plan (one persistent launch,
    or one launch per stage; plan="auto" lets the autotuner time both), and captures
    it as a graph; run() replays it (no host synchronisation); results() reads sizes
    and statuses.  The field tensors are referenced, not copied: overwrite them in
    place between runs to compress new data of the same shapes."""

    def __init__(self, fields, ebs, eb_modes="rel", select="exhaustive", radius=512, weights=None,
                 autotune=True, archive_caps=None, stream=None, plan="auto"):
        n = len(fields)
        if n == 0:
            raise ValueError("empty batch")
        ebs = list(ebs) if hasattr(ebs, "__len__") else [ebs] * n
        modes = list(eb_modes) if isinstance(eb_modes, (list, tuple)) else [eb_modes] * n
        dev = fields[0].device
        self.fields = list(fields)
        self.archives = []
        arr = (L.csz_field * n)()
        for i, x in enumerate(self.fields):
            if not (x.is_cuda and x.dtype == torch.float32 and x.is_contiguous() and 1 <= x.dim() <= 3):
                raise ValueError("fields must be contiguous float32 CUDA tensors of 1-3 dims")
            cap = int(archive_caps[i]) if archive_caps is not None else max_archive_bytes(tuple(x.shape))
            a = torch.empty(max(cap, 1), dtype=torch.uint8, device=dev)
            self.archives.append(a)
            f = arr[i]
            f.d_field = x.data_ptr()
            f.ndim = x.dim()
            for k, d in enumerate(x.shape):
                f.dims[k] = int(d)
            f.eb_mode = EB_MODES[modes[i]] if isinstance(modes[i], str) else int(modes[i])
            f.eb = float(ebs[i])
            f.d_archive = a.data_ptr()
            f.archive_cap = a.numel()
        self._arr = arr
        wsb = int(L.lib().csz_batch_workspace_bytes(n, arr))
        if wsb == 0:
            raise ValueError("invalid field in batch")
        self.workspace = torch.empty(wsb, dtype=torch.uint8, device=dev)
        opt = L.csz_options()
        opt.radius = int(radius)
        opt.select = SELECT[select] if isinstance(select, str) else int(select)
        self.weights = weights
        if weights is not None:
            if not (weights.is_cuda and weights.dtype == torch.float32 and weights.numel() == MLP_PARAMS):
                raise ValueError("weights must be a float32 CUDA tensor of 1443 parameters")
            opt.selector_weights = C.c_void_p(weights.data_ptr())
        h = C.c_void_p()
        st = L.lib().csz_batch_create(n, arr, C.byref(opt), C.c_void_p(self.workspace.data_ptr()), wsb,
                                      (BATCH_AUTOTUNE if autotune else 0) | BATCH_PLANS[plan],
                                      _stream_ptr(stream), C.byref(h))
        if st != L.OK:
            raise L.CszError(st, "csz_batch_create (" + L.lib().csz_batch_last_error().decode() + ")")
        self._h = h
        self.n = n

    def run(self, stream=None):
        _check(L.lib().csz_batch_compress(self._h, _stream_ptr(stream)), "csz_batch_compress")

    def results(self, stream=None):
        """(sizes, statuses): per-field archive bytes and csz_status values."""
        sizes = (C.c_uint64 * self.n)()
        stats = (C.c_int * self.n)()
        L.lib().csz_batch_results(self._h, sizes, stats, _stream_ptr(stream))
        return [int(v) for v in sizes], [int(v) for v in stats]

    def info(self):
        g = C.c_int()
        ms = (C.c_double * 4)()
        L.lib().csz_batch_info(self._h, C.byref(g), ms)
        p, pg = C.c_int(), C.c_int()
        pms = (C.c_double * 4)()
        L.lib().csz_batch_plan(self._h, C.byref(p), C.byref(pg), pms)
        return {"construct_grid": int(g.value), "tuned_ms": [float(v) for v in ms],
                "persistent": bool(p.value), "grid": int(pg.value), "persist_ms": [float(v) for v in pms]}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            L.lib().csz_batch_destroy(h)
            self._h = None


class BatchDecompressor:
    """Decompresses a fixed list of archives into fields of known shapes together
    (one launch per stage, replayed as a CUDA graph).  The archive tensors are
    referenced: overwrite them in place (same shapes) to decompress new data."""

    def __init__(self, archives, shapes, archive_bytes=None, outs=None, stream=None):
        n = len(archives)
        if n == 0 or len(shapes) != n:
            raise ValueError("one shape per archive")
        dev = archives[0].device
        self.archives = list(archives)
        self.outs = list(outs) if outs is not None else [torch.empty(tuple(sh), dtype=torch.float32, device=dev)
                                                          for sh in shapes]
        arr = (L.csz_dfield * n)()
        for i, (a, sh, o) in enumerate(zip(self.archives, shapes, self.outs)):
            if not (a.is_cuda and a.dtype == torch.uint8):
                raise ValueError("archives must be uint8 CUDA tensors")
            if not (o.is_cuda and o.dtype == torch.float32 and o.is_contiguous()):
                raise ValueError("outputs must be contiguous float32 CUDA tensors")
            f = arr[i]
            f.d_archive = a.data_ptr()
            f.archive_bytes = int(archive_bytes[i]) if archive_bytes is not None else a.numel()
            f.d_out = o.data_ptr()
            f.out_cap_elems = o.numel()
            f.ndim = len(sh)
            for k, d in enumerate(sh):
                f.dims[k] = int(d)
        self._arr = arr
        wsb = int(L.lib().csz_batch_dec_workspace_bytes(n, arr))
        if wsb == 0:
            raise ValueError("invalid shape in batch")
        self.workspace = torch.empty(wsb, dtype=torch.uint8, device=dev)
        h = C.c_void_p()
        st = L.lib().csz_batch_dec_create(n, arr, C.c_void_p(self.workspace.data_ptr()), wsb, _stream_ptr(stream),
                                          C.byref(h))
        if st != L.OK:
            raise L.CszError(st, "csz_batch_dec_create (" + L.lib().csz_batch_last_error().decode() + ")")
        self._h = h
        self.n = n

    def run(self, stream=None):
        _check(L.lib().csz_batch_decompress(self._h, _stream_ptr(stream)), "csz_batch_decompress")

    def results(self, stream=None):
        stats = (C.c_int * self.n)()
        L.lib().csz_batch_dec_results(self._h, stats, _stream_ptr(stream))
        return [int(v) for v in stats]

    def tune(self, stream=None):
        """Times the decoder's CTA shapes on the archives now in the buffers, keeps the
        fastest (csz_batch_dec_tune).  Returns (warps per CTA, [ms of 8, 16, 32 warps])."""
        warps = C.c_int()
        ms = (C.c_double * 3)()
        _check(L.lib().csz_batch_dec_tune(self._h, _stream_ptr(stream), C.byref(warps), ms), "csz_batch_dec_tune")
        return int(warps.value), [float(v) for v in ms]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            L.lib().csz_batch_dec_destroy(h)
            self._h = None


# ---------------------------------------------------------------------------------
# learned selector: training rows, inference, gradient, training
# ---------------------------------------------------------------------------------
def _f32_cuda(t, name, shape=None):
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}")
    return C.c_void_p(t.data_ptr())


def nblocks(dims) -> int:
    d = [int(v) for v in dims]
    if len(d) == 1:
        return -(-d[0] // 4096)
    if len(d) == 2:
        return -(-d[0] // 64) * -(-d[1] // 64)
    return -(-d[0] // 16) * -(-d[1] // 16) * -(-d[2] // 16)


def selector_rows(field: torch.Tensor, eb: float, eb_mode: str = "rel", radius: int = 512, out=None,
                  workspace: Workspace | None = None, stream=None):
    """Training rows of the learned selector for every codec block of `field`:
    dict(feat [nblk,8] f32, target [nblk,3] f32 (log2 bits/element), sizes [nblk,3] i32
    (exact bytes, -1 where a codec does not apply), valid [nblk] u8).  `out` may hold
    preallocated tensors of those shapes (views into larger buffers are fine)."""
    if not (field.is_cuda and field.dtype == torch.float32 and field.is_contiguous()):
        raise ValueError("field must be a contiguous float32 CUDA tensor")
    dims = tuple(field.shape)
    nb = nblocks(dims)
    dev = field.device
    if out is None:
        out = dict(feat=torch.empty((nb, 8), dtype=torch.float32, device=dev),
                   target=torch.empty((nb, 3), dtype=torch.float32, device=dev),
                   sizes=torch.empty((nb, 3), dtype=torch.int32, device=dev),
                   valid=torch.empty(nb, dtype=torch.uint8, device=dev))
    for k, shp in (("feat", (nb, 8)), ("target", (nb, 3)), ("sizes", (nb, 3)), ("valid", (nb,))):
        t = out[k]
        if not (t.is_cuda and t.is_contiguous() and tuple(t.shape) == shp):
            raise ValueError(f"out[{k!r}] must be a contiguous CUDA tensor of shape {shp}")
    ws = _ws(dev, workspace).get(workspace_bytes(dims) or 256)
    st = L.lib().csz_selector_rows(C.c_void_p(field.data_ptr()), len(dims), L.dims_array(dims),
                                   EB_MODES[eb_mode] if isinstance(eb_mode, str) else int(eb_mode), float(eb),
                                   int(radius), C.c_void_p(ws.data_ptr()), ws.numel(),
                                   C.c_void_p(out["feat"].data_ptr()), C.c_void_p(out["target"].data_ptr()),
                                   C.c_void_p(out["sizes"].data_ptr()), C.c_void_p(out["valid"].data_ptr()),
                                   _stream_ptr(stream))
    _check(st, "csz_selector_rows")
    return out


def selector_predict(weights: torch.Tensor, feat: torch.Tensor, stream=None) -> torch.Tensor:
    """Network outputs [n,3] for feature rows [n,8] (the encoder's own forward pass)."""
    n = feat.shape[0]
    out = torch.empty((n, 3), dtype=torch.float32, device=feat.device)
    st = L.lib().csz_selector_predict(_f32_cuda(weights, "weights", (MLP_PARAMS,)), _f32_cuda(feat, "feat", (n, 8)),
                                      n, C.c_void_p(out.data_ptr()), _stream_ptr(stream))
    _check(st, "csz_selector_predict")
    return out


def _valid_ptr(valid, n):
    if valid is None:
        return None
    if not (valid.is_cuda and valid.dtype == torch.uint8 and valid.is_contiguous() and valid.numel() == n):
        raise ValueError("valid must be a contiguous uint8 CUDA tensor with one entry per row")
    return C.c_void_p(valid.data_ptr())


def _train_ws(n, device):
    return torch.empty(int(L.lib().csz_selector_workspace_bytes(n)), dtype=torch.uint8, device=device)


def selector_grad(weights, feat, target, valid=None, stream=None):
    """(mean squared error, its gradient [1443]) over the rows with valid != 0."""
    n = feat.shape[0]
    grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device=feat.device)
    ws = _train_ws(n, feat.device)
    loss = C.c_double(0.0)
    st = L.lib().csz_selector_grad(_f32_cuda(weights, "weights", (MLP_PARAMS,)), _f32_cuda(feat, "feat", (n, 8)),
                                   _f32_cuda(target, "target", (n, 3)), _valid_ptr(valid, n), n,
                                   C.c_void_p(grad.data_ptr()), C.byref(loss), C.c_void_p(ws.data_ptr()),
                                   ws.numel(), _stream_ptr(stream))
    _check(st, "csz_selector_grad")
    return float(loss.value), grad


def selector_train(weights, feat, target, valid=None, steps: int = 2000, lr: float = 3e-3, stream=None):
    """Full-batch Adam on `weights` in place; returns the loss at the last step."""
    n = feat.shape[0]
    ws = _train_ws(n, feat.device)
    loss = C.c_double(0.0)
    st = L.lib().csz_selector_train(_f32_cuda(weights, "weights", (MLP_PARAMS,)), _f32_cuda(feat, "feat", (n, 8)),
                                    _f32_cuda(target, "target", (n, 3)), _valid_ptr(valid, n), n, int(steps),
                                    float(lr), C.c_void_p(ws.data_ptr()), ws.numel(), C.byref(loss),
                                    _stream_ptr(stream))
    _check(st, "csz_selector_train")
    return float(loss.value)


def status_string(st: int) -> str:
    return L.lib().csz_status_string(int(st)).decode()


def kernel_names():
    n = L.lib().csz_kernel_count()
    return [L.lib().csz_kernel_name(i).decode() for i in range(n)]


def trace_enable(on: bool = True):
    L.lib().csz_trace_enable(1 if on else 0)


def trace_read(reset: bool = True):
    """{kernel name: (total ms while tracing, launches)}"""
    n = L.lib().csz_kernel_count()
    ms = (C.c_double * n)()
    cnt = (C.c_uint64 * n)()
    L.lib().csz_trace_read(ms, cnt, 1 if reset else 0)
    names = kernel_names()
    return {names[i]: (float(ms[i]), int(cnt[i])) for i in range(n)}
