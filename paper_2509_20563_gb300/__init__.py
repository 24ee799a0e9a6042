"""GB300-native error-bounded lossy compression (FZMod-Default hot path).

Thin Python binding of ``libfz.so`` (the C ABI declared in ``include/fz.h``).
Every stage of compression and decompression runs in the library's CUDA
kernels; this module only marshals arguments: torch supplies device memory
and the current CUDA stream.  If the library has not been built the binding
raises instead of falling back to anything else.

The raw C entry points are available under their C names (``fz_compress``,
``fz_decompress``, ...) through :func:`lib`; :func:`compress` and
:func:`decompress` wrap them for torch tensors.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

__all__ = ["lib", "Context", "compress", "decompress", "lorenzo_quantize", "huffman_codebook", "stream_info",
           "block_report", "mlp_grad", "mlp_adam", "compress_batch", "decompress_batch", "FzError", "HEADER_BYTES",
           "stream_check", "set_spin_limit", "selftest_bounded_wait", "error_stats", "histogram",
           "SELECTOR_WEIGHTS"]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfz.so")
HEADER_BYTES = 256
SELECTOR_WEIGHTS = 2372  # W1[64][32], b1[64], W2[4][64], b2[4]
SELECTOR_FEATURES = 32

STATUS = {0: "FZ_OK", 1: "FZ_EINVAL", 2: "FZ_ENOMEM", 3: "FZ_ECUDA", 4: "FZ_EBUFFER", 5: "FZ_ECORRUPT",
          6: "FZ_ETIMEOUT", 7: "FZ_EUNSUPPORTED"}
PREDICTORS = {"lorenzo1": 0, "lorenzo2": 1, "interp_linear": 2, "interp_cubic": 3, "ginterp": 4, "mlp": 16,
              "exhaustive": 17}

_lock = threading.Lock()
_lib = None


class FzError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


class Pipeline(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("predictor", C.c_uint32), ("radius", C.c_uint32),
                ("block", C.c_uint32 * 3), ("chunk", C.c_uint32), ("encoder", C.c_uint32),
                ("selector_weights", C.c_void_p)]


class ErrorReport(C.Structure):
    """fz_error_report: reconstruction statistics of fz_error_stats."""
    _fields_ = [("max_abs_err", C.c_double), ("sse", C.c_double), ("x_min", C.c_double), ("x_max", C.c_double),
                ("psnr_db", C.c_double), ("n_finite", C.c_uint64), ("n_nonfinite_mismatch", C.c_uint64)]


_u64p = C.POINTER(C.c_uint64)
_vp = C.c_void_p


def _declare(L):
    L.fz_status_str.restype = C.c_char_p
    L.fz_status_str.argtypes = [C.c_int]
    L.fz_ctx_create.argtypes = [C.c_int, C.POINTER(C.c_void_p)]
    L.fz_ctx_destroy.argtypes = [_vp]
    L.fz_compress_bound.restype = C.c_uint64
    L.fz_compress_bound.argtypes = [C.c_uint32, _u64p]
    L.fz_compress.argtypes = [_vp, _vp, C.c_uint32, _u64p, C.c_uint32, C.c_double, C.POINTER(Pipeline), _vp,
                              C.c_uint64, _u64p, _vp, _vp]
    L.fz_decompress.argtypes = [_vp, _vp, C.c_uint64, _vp, _vp, C.c_uint64, _vp]
    L.fz_stream_info.argtypes = [_vp, C.c_uint64, C.POINTER(C.c_uint32), _u64p, C.POINTER(C.c_double),
                                 C.POINTER(C.c_uint32)]
    L.fz_lorenzo_quantize.argtypes = [_vp, _vp, C.c_uint32, _u64p, C.c_uint32, C.c_double, C.POINTER(Pipeline),
                                      _vp, _vp, _vp, _u64p, _u64p, C.POINTER(C.c_double), _vp]
    L.fz_huffman_codebook.argtypes = [_vp, _vp, C.c_uint32, _vp, _vp, _vp]
    L.fz_block_report.argtypes = [_vp, _vp, _u64p, C.c_uint32, C.c_double, C.c_uint32, _vp, _vp, _vp, _vp]
    L.fz_mlp_grad.argtypes = [_vp, _vp, _vp, _vp, C.c_uint32, _vp, C.POINTER(C.c_float), _vp]
    L.fz_mlp_adam.argtypes = [_vp, _vp, _vp, _vp, _vp, C.c_uint32, C.c_float, C.c_float, C.c_float, C.c_float,
                              _vp, _vp]
    L.fz_compress_batch_bound.restype = C.c_uint64
    L.fz_compress_batch_bound.argtypes = [C.c_uint32, _vp, _vp]
    L.fz_compress_batch.argtypes = [_vp, C.c_uint32, _vp, _vp, _vp, C.c_uint32, _vp, C.POINTER(Pipeline), _vp,
                                    C.c_uint64, _vp, _vp]
    L.fz_decompress_batch.argtypes = [_vp, C.c_uint32, _vp, _vp, _vp, _vp, _vp]
    L.fz_ctx_set_batch_options.argtypes = [_vp, C.c_int, C.c_int]
    L.fz_decompress_noalloc.argtypes = [_vp, C.c_uint64, _vp, _vp, C.c_uint64, _vp]
    L.fz_ctx_set_profiling.argtypes = [_vp, C.c_int]
    L.fz_stream_check.argtypes = [_vp, C.c_uint64]
    L.fz_error_stats.argtypes = [_vp, _vp, _vp, C.c_uint64, C.POINTER(ErrorReport), _vp]
    L.fz_histogram.argtypes = [_vp, _vp, C.c_uint64, C.c_uint32, C.c_uint32, _vp, _vp]
    L.fz_ctx_set_spin_limit.argtypes = [_vp, C.c_longlong]
    L.fz_selftest_bounded_wait.argtypes = [_vp, _vp]
    L.fz_ctx_get_profile.argtypes = [_vp, _vp]
    for name in ("fz_ctx_create", "fz_ctx_destroy", "fz_compress", "fz_decompress", "fz_stream_info",
                 "fz_lorenzo_quantize", "fz_huffman_codebook", "fz_block_report", "fz_mlp_grad", "fz_mlp_adam",
                 "fz_ctx_set_profiling", "fz_ctx_get_profile", "fz_compress_batch", "fz_decompress_batch",
                 "fz_ctx_set_batch_options", "fz_decompress_noalloc"):
        getattr(L, name).restype = C.c_int


def lib():
    """The loaded libfz.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libfz.so is not built ({LIB_PATH}); run paper_2509_20563_gb300.build.build()")
            L = C.CDLL(LIB_PATH)
            _declare(L)
            _lib = L
    return _lib


def _check(st: int, what: str):
    if st != 0:
        raise FzError(st, what)


class Context:
    """Owns an fz_ctx (device workspace) for one CUDA device."""

    def __init__(self, device: int = 0):
        h = C.c_void_p()
        _check(lib().fz_ctx_create(int(device), C.byref(h)), "fz_ctx_create")
        self.handle = h
        self.device = int(device)

    def close(self):
        if getattr(self, "handle", None):
            lib().fz_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_ctxs: dict[int, Context] = {}


def _ctx(device: int) -> Context:
    with _lock:
        c = _ctxs.get(device)
    if c is None:
        c = Context(device)
        with _lock:
            _ctxs[device] = c
    return c


def _dims(shape):
    d = (C.c_uint64 * 3)(1, 1, 1)
    for a, s in enumerate(reversed(shape)):
        d[a] = int(s)
    return d


ENCODERS = {"huffman": 0, "shuffle": 1}


def _pipeline(predictor="lorenzo1", radius=512, selector_weights=None, chunk=0, block=None,
              encoder="huffman") -> Pipeline:
    p = Pipeline()
    p.struct_size = C.sizeof(Pipeline)
    p.predictor = PREDICTORS[predictor] if isinstance(predictor, str) else int(predictor)
    p.radius = int(radius)
    p.chunk = int(chunk)
    p.encoder = ENCODERS[encoder] if isinstance(encoder, str) else int(encoder)
    for a, b in enumerate(block or ()):
        p.block[a] = int(b)
    p.selector_weights = selector_weights.data_ptr() if selector_weights is not None else None
    return p


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def compress_bound(shape) -> int:
    return int(lib().fz_compress_bound(len(shape), _dims(shape)))


def compress(x: torch.Tensor, eb: float, mode: str = "rel", predictor="lorenzo1", radius: int = 512,
             out: torch.Tensor | None = None, stream=None, selector_weights=None, chunk: int = 0,
             block=None, encoder: str = "huffman") -> torch.Tensor:
    """Compress a contiguous float32 CUDA tensor (1-3 dims, last axis fastest).
    ``chunk`` is the Huffman chunk in symbols (0: the library's default),
    ``block`` the predictor block (x, y, z extents; None: the default) and
    ``encoder`` "huffman" or "shuffle" (FZMod-Speed's bit-shuffle encoder).
    Returns a uint8 CUDA tensor holding exactly the stream; its host header
    copy is attached as ``.fz_header`` (bytes)."""
    if not (x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
        raise ValueError("compress expects a contiguous float32 CUDA tensor")
    if not 1 <= x.dim() <= 3:
        raise ValueError("1 to 3 dimensions")
    bound = compress_bound(x.shape)
    if out is None:
        out = torch.empty(bound, dtype=torch.uint8, device=x.device)
    nbytes = C.c_uint64()
    hdr = C.create_string_buffer(HEADER_BYTES)
    pipe = _pipeline(predictor, radius, selector_weights, chunk, block, encoder)
    st = lib().fz_compress(_ctx(x.device.index or 0).handle, C.c_void_p(x.data_ptr()), x.dim(), _dims(x.shape),
                           1 if mode == "rel" else 0, float(eb), C.byref(pipe), C.c_void_p(out.data_ptr()),
                           out.numel(), C.byref(nbytes), hdr, _stream(stream))
    _check(st, "fz_compress")
    res = out[: nbytes.value]
    res.fz_header = hdr.raw
    return res


def stream_info(header: bytes):
    ndim, dims, eb_abs, flags = C.c_uint32(), (C.c_uint64 * 3)(), C.c_double(), C.c_uint32()
    buf = C.create_string_buffer(bytes(header[:HEADER_BYTES]), HEADER_BYTES)
    _check(lib().fz_stream_info(buf, HEADER_BYTES, C.byref(ndim), dims, C.byref(eb_abs), C.byref(flags)),
           "fz_stream_info")
    shape = tuple(int(dims[a]) for a in range(ndim.value))[::-1]
    return shape, eb_abs.value, flags.value


def error_stats(x: torch.Tensor, y: torch.Tensor, stream=None, ctx: "Context | None" = None) -> dict:
    """Reconstruction statistics of y against x (fz_error_stats): max abs
    error, sum of squared errors, value range, PSNR (dB), finite count and
    non-finite mismatches."""
    if not (x.is_cuda and y.is_cuda and x.dtype == torch.float32 and y.dtype == torch.float32
            and x.is_contiguous() and y.is_contiguous() and x.numel() == y.numel()):
        raise ValueError("error_stats expects two contiguous float32 CUDA tensors of the same size")
    r = ErrorReport()
    c = ctx if ctx is not None else _ctx(x.device.index or 0)
    _check(lib().fz_error_stats(c.handle, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), x.numel(),
                                C.byref(r), _stream(stream)), "fz_error_stats")
    return {f: getattr(r, f) for f, _ in ErrorReport._fields_}


HIST_METHODS = {"private": 0, "topk": 1}


def histogram(codes: torch.Tensor, nsym: int, method: str = "private", stream=None,
              ctx: "Context | None" = None) -> torch.Tensor:
    """Counts of a contiguous uint16 code array on the GPU (fz_histogram);
    returns an int64 CUDA tensor of nsym counts."""
    if not (codes.is_cuda and codes.dtype in (torch.int16, torch.uint16) and codes.is_contiguous()):
        raise ValueError("histogram expects a contiguous 16-bit CUDA tensor")
    out = torch.empty(int(nsym), dtype=torch.int64, device=codes.device)
    c = ctx if ctx is not None else _ctx(codes.device.index or 0)
    _check(lib().fz_histogram(c.handle, C.c_void_p(codes.data_ptr()), codes.numel(), int(nsym),
                              HIST_METHODS[method], C.c_void_p(out.data_ptr()), _stream(stream)), "fz_histogram")
    return out


def stream_check(header: bytes, stream_bytes: int) -> int:
    """Host-only validation of a stream header against a stream length
    (fz_stream_check); returns the status code (0 = valid)."""
    buf = C.create_string_buffer(bytes(header[:HEADER_BYTES]), HEADER_BYTES)
    return int(lib().fz_stream_check(buf, int(stream_bytes)))


def set_spin_limit(cycles: int, device: int = 0) -> None:
    """Bound of the device-side look-back waits of the default context
    (clock cycles; 0 restores the library default)."""
    _check(lib().fz_ctx_set_spin_limit(_ctx(device).handle, int(cycles)), "fz_ctx_set_spin_limit")


def selftest_bounded_wait(device: int = 0, stream=None) -> int:
    """Run the bounded-wait self-test (fz_selftest_bounded_wait); returns
    its status code, FZ_ETIMEOUT (6) when the wait gave up as designed."""
    return int(lib().fz_selftest_bounded_wait(_ctx(device).handle, _stream(stream)))


def decompress(buf: torch.Tensor, out: torch.Tensor | None = None, header: bytes | None = None,
               stream=None) -> torch.Tensor:
    """Reconstruct the float32 field from a compressed stream on the GPU."""
    if not (buf.is_cuda and buf.dtype == torch.uint8):
        raise ValueError("decompress expects a uint8 CUDA tensor")
    header = header if header is not None else getattr(buf, "fz_header", None)
    if header is None:
        header = bytes(buf[:HEADER_BYTES].cpu().numpy())
    shape, _, _ = stream_info(header)
    n = 1
    for s in shape:
        n *= s
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=buf.device)
    hb = C.create_string_buffer(bytes(header[:HEADER_BYTES]), HEADER_BYTES)
    st = lib().fz_decompress(_ctx(buf.device.index or 0).handle, C.c_void_p(buf.data_ptr()), buf.numel(), hb,
                             C.c_void_p(out.data_ptr()), out.numel(), _stream(stream))
    _check(st, "fz_decompress")
    return out


def _batch_shapes(xs):
    n = len(xs)
    ndim = (C.c_uint32 * n)()
    dims = (C.c_uint64 * (3 * n))()
    for j, x in enumerate(xs):
        ndim[j] = x.dim()
        d = _dims(x.shape)
        for a in range(3):
            dims[3 * j + a] = d[a]
    return ndim, dims


def compress_batch(xs, eb, mode: str = "rel", predictor="lorenzo1", radius: int = 512, out=None, stream=None,
                   ctx: Context | None = None, chunk: int = 0):
    """Compress a list of contiguous float32 CUDA tensors (1-3 dims each) in
    one batched call.  ``eb`` is one bound or one per field; ``chunk`` 0
    lets the autotuner pick the Huffman chunk per kind of field.  Returns the
    packed uint8 buffer and the stream offsets (n+1 ints); stream j is
    ``buf[off[j]:off[j] + its total_bytes]``, byte-identical to ``compress``
    of field j with the chunk its header records."""
    xs = list(xs)
    n = len(xs)
    if n == 0:
        raise ValueError("empty batch")
    for x in xs:
        if not (x.is_cuda and x.dtype == torch.float32 and x.is_contiguous() and 1 <= x.dim() <= 3):
            raise ValueError("compress_batch expects contiguous float32 CUDA tensors of 1 to 3 dims")
    ndim, dims = _batch_shapes(xs)
    bound = int(lib().fz_compress_batch_bound(n, ndim, dims))
    if out is None:
        out = torch.empty(bound, dtype=torch.uint8, device=xs[0].device)
    ebs = [float(eb)] * n if isinstance(eb, (int, float)) else [float(e) for e in eb]
    ptrs = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
    ebarr = (C.c_double * n)(*ebs)
    offs = (C.c_uint64 * (n + 1))()
    pipe = _pipeline(predictor, radius, chunk=chunk)
    c = ctx if ctx is not None else _ctx(xs[0].device.index or 0)
    st = lib().fz_compress_batch(c.handle, n, ptrs, ndim, dims, 1 if mode == "rel" else 0, ebarr, C.byref(pipe),
                                 C.c_void_p(out.data_ptr()), out.numel(), offs, _stream(stream))
    _check(st, "fz_compress_batch")
    return out, [int(offs[j]) for j in range(n + 1)]


def decompress_batch(buf: torch.Tensor, offsets, outs=None, stream=None, ctx: Context | None = None):
    """Reconstruct every stream of a packed batch buffer; returns the list of
    float32 CUDA tensors (shapes from the stream headers)."""
    n = len(offsets) - 1
    if outs is None:
        host = [bytes(buf[offsets[j]: offsets[j] + HEADER_BYTES].cpu().numpy()) for j in range(n)]
        outs = [torch.empty(stream_info(h)[0], dtype=torch.float32, device=buf.device) for h in host]
    ptrs = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    caps = (C.c_uint64 * n)(*[o.numel() for o in outs])
    offs = (C.c_uint64 * (n + 1))(*[int(o) for o in offsets])
    c = ctx if ctx is not None else _ctx(buf.device.index or 0)
    st = lib().fz_decompress_batch(c.handle, n, C.c_void_p(buf.data_ptr()), offs, ptrs, caps, _stream(stream))
    _check(st, "fz_decompress_batch")
    return outs


class Profile(C.Structure):
    """fz_profile: per-stage times of the last calls, launch and plan counts."""
    _fields_ = [("n_compress", C.c_uint32), ("n_decompress", C.c_uint32),
                ("compress_names", (C.c_char * 16) * 12), ("compress_ms", C.c_float * 12),
                ("decompress_names", (C.c_char * 16) * 12), ("decompress_ms", C.c_float * 12),
                ("launches", C.c_uint64), ("batch_plans", C.c_uint32), ("batch_graphs", C.c_uint32),
                ("batch_tune", C.c_int32 * 4), ("batch_chunk", C.c_uint32 * 2)]


def profile(device: int = 0, ctx: Context | None = None) -> Profile:
    c = ctx if ctx is not None else _ctx(device)
    p = Profile()
    _check(lib().fz_ctx_get_profile(c.handle, C.byref(p)), "fz_ctx_get_profile")
    return p


def set_batch_options(autotune: bool = True, graphs: bool = True, device: int = 0, ctx: Context | None = None):
    c = ctx if ctx is not None else _ctx(device)
    _check(lib().fz_ctx_set_batch_options(c.handle, int(autotune), int(graphs)), "fz_ctx_set_batch_options")


def decompress_noalloc(buf: torch.Tensor, out: torch.Tensor | None = None, header: bytes | None = None,
                       stream=None) -> torch.Tensor:
    """Like :func:`decompress`, through the entry point that allocates
    nothing on the device (fixed scratch; see ``fz_decompress_noalloc``).
    ``out`` is allocated here (by torch) when not given; pass it to keep the
    call itself free of allocations."""
    if not (buf.is_cuda and buf.dtype == torch.uint8):
        raise ValueError("decompress_noalloc expects a uint8 CUDA tensor")
    header = header if header is not None else getattr(buf, "fz_header", None)
    if out is None:
        h = header if header is not None else bytes(buf[:HEADER_BYTES].cpu().numpy())
        out = torch.empty(stream_info(h)[0], dtype=torch.float32, device=buf.device)
    hb = C.create_string_buffer(bytes(header[:HEADER_BYTES]), HEADER_BYTES) if header is not None else None
    with torch.cuda.device(buf.device):
        st = lib().fz_decompress_noalloc(C.c_void_p(buf.data_ptr()), buf.numel(), hb, C.c_void_p(out.data_ptr()),
                                         out.numel(), _stream(stream))
    _check(st, "fz_decompress_noalloc")
    return out


def lorenzo_quantize(x: torch.Tensor, eb: float, mode: str = "rel", predictor="lorenzo1", radius: int = 512,
                     stream=None):
    """Stage call: (codes u16 block-major, anchors i32, hist u64, n_out, n_exc, eb_abs)."""
    ndim = x.dim()
    blk = {1: (1024,), 2: (32, 32), 3: (8, 8, 8)}[ndim]
    nb = 1
    for s, b in zip(x.shape, blk):
        nb *= -(-s // b)
    bs = 1
    for b in blk:
        bs *= b
    codes = torch.empty(nb * bs, dtype=torch.int16, device=x.device)
    anchors = torch.empty(nb, dtype=torch.int32, device=x.device)
    hist = torch.zeros(2 * radius, dtype=torch.int64, device=x.device)
    no, ne, eba = C.c_uint64(), C.c_uint64(), C.c_double()
    pipe = _pipeline(predictor, radius)
    st = lib().fz_lorenzo_quantize(_ctx(x.device.index or 0).handle, C.c_void_p(x.data_ptr()), ndim, _dims(x.shape),
                                   1 if mode == "rel" else 0, float(eb), C.byref(pipe), C.c_void_p(codes.data_ptr()),
                                   C.c_void_p(anchors.data_ptr()), C.c_void_p(hist.data_ptr()), C.byref(no),
                                   C.byref(ne), C.byref(eba), _stream(stream))
    _check(st, "fz_lorenzo_quantize")
    return codes, anchors, hist, no.value, ne.value, eba.value


def huffman_codebook(hist: torch.Tensor, stream=None):
    """Stage call: (lengths u8, canonical codewords u32 as int32) for a u64 histogram."""
    nsym = hist.numel()
    lens = torch.empty(nsym, dtype=torch.uint8, device=hist.device)
    codes = torch.empty(nsym, dtype=torch.int32, device=hist.device)
    st = lib().fz_huffman_codebook(_ctx(hist.device.index or 0).handle, C.c_void_p(hist.data_ptr()), nsym,
                                   C.c_void_p(lens.data_ptr()), C.c_void_p(codes.data_ptr()), _stream(stream))
    _check(st, "fz_huffman_codebook")
    return lens, codes


# ---------------------------------------------------------------- selector
def block_report(x: torch.Tensor, eb: float, mode: str = "rel", radius: int = 512, costs: bool = True,
                 features: bool = True, stream=None):
    """Per-block exhaustive-trial labels (u8), trial costs (int32 [nb, 4])
    and bfloat16 features (int16 bits [nb, 32]) of a 3D float32 CUDA field."""
    if x.dim() != 3:
        raise ValueError("block_report needs a 3D field")
    nb = 1
    for s_ in x.shape:
        nb *= -(-s_ // 8)
    lab = torch.empty(nb, dtype=torch.uint8, device=x.device)
    cst = torch.empty((nb, 4), dtype=torch.int32, device=x.device) if costs else None
    fea = torch.empty((nb, SELECTOR_FEATURES), dtype=torch.int16, device=x.device) if features else None
    st = lib().fz_block_report(_ctx(x.device.index or 0).handle, C.c_void_p(x.data_ptr()), _dims(x.shape),
                               1 if mode == "rel" else 0, float(eb), int(radius), C.c_void_p(lab.data_ptr()),
                               C.c_void_p(cst.data_ptr()) if cst is not None else None,
                               C.c_void_p(fea.data_ptr()) if fea is not None else None, _stream(stream))
    _check(st, "fz_block_report")
    return lab, cst, fea


def mlp_grad(w: torch.Tensor, feat: torch.Tensor, labels: torch.Tensor, grad: torch.Tensor | None = None,
             want_loss: bool = True, stream=None):
    """Gradient (float32 [2372]) and loss of the selector objective."""
    if grad is None:
        grad = torch.empty(SELECTOR_WEIGHTS, dtype=torch.float32, device=w.device)
    loss = C.c_float()
    st = lib().fz_mlp_grad(_ctx(w.device.index or 0).handle, C.c_void_p(w.data_ptr()), C.c_void_p(feat.data_ptr()),
                           C.c_void_p(labels.data_ptr()), labels.numel(), C.c_void_p(grad.data_ptr()),
                           C.byref(loss) if want_loss else None, _stream(stream))
    _check(st, "fz_mlp_grad")
    return grad, (loss.value if want_loss else None)


def mlp_adam(w, grad, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
             w_bf16: torch.Tensor | None = None, stream=None):
    st = lib().fz_mlp_adam(_ctx(w.device.index or 0).handle, C.c_void_p(w.data_ptr()), C.c_void_p(grad.data_ptr()),
                           C.c_void_p(m.data_ptr()), C.c_void_p(v.data_ptr()), int(step), float(lr), float(beta1),
                           float(beta2), float(eps), C.c_void_p(w_bf16.data_ptr()) if w_bf16 is not None else None,
                           _stream(stream))
    _check(st, "fz_mlp_adam")
