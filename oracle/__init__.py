"""CPU oracle of the compression path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` import this package.  It compiles ``fz_oracle.c`` (and, for the
learned selector, ``fz_oracle_mlp.c``) with gcc into ``oracle/_build`` and
wraps the C functions with ctypes and numpy.  Nothing here touches the CUDA
library, and the CUDA library never loads this one.

The C sources are built with ``-O2 -ffp-contract=off -fno-fast-math`` so that
every binary32 operation is one IEEE-754 operation, as the method requires.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SOURCES = ["fz_oracle.c"]
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, EBUFFER, ECORRUPT, EUNSUPPORTED = 0, 1, 2, 4, 5, 7


def _extra_sources():
    return [s for s in ("fz_oracle_mlp.c",) if os.path.exists(os.path.join(_HERE, s))]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, plain C11); returns its path."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES + _extra_sources()]
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB):
        lib_t = os.path.getmtime(_LIB)
        if all(os.path.getmtime(s) <= lib_t for s in srcs):
            return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


u8p = C.POINTER(C.c_uint8)
u16p = C.POINTER(C.c_uint16)
u32p = C.POINTER(C.c_uint32)
i32p = C.POINTER(C.c_int32)
i64p = C.POINTER(C.c_int64)
u64p = C.POINTER(C.c_uint64)
f32p = C.POINTER(C.c_float)


def _declare(L):
    L.orc_range.argtypes = [f32p, C.c_uint64, f32p, f32p, C.POINTER(C.c_int)]
    L.orc_constants.argtypes = [C.c_double, f32p, f32p, f32p]
    L.orc_constants.restype = None
    L.orc_prequant_one.argtypes = [C.c_float, C.c_float, C.c_float, C.c_float, i32p]
    L.orc_prequant.argtypes = [f32p, C.c_uint64, C.c_float, C.c_float, C.c_float, i32p, u8p]
    L.orc_prequant.restype = None
    L.orc_block_shape.argtypes = [C.c_uint32, u32p]
    L.orc_block_shape.restype = None
    L.orc_lorenzo_block.argtypes = [C.c_int, C.c_uint32, u32p, i32p, u8p, i64p]
    L.orc_lorenzo_block.restype = None
    L.orc_lorenzo_block_inverse.argtypes = [C.c_int, C.c_uint32, u32p, i64p]
    L.orc_lorenzo_block_inverse.restype = None
    L.orc_huffman_lengths.argtypes = [u64p, C.c_uint32, u8p]
    L.orc_canonical_codes.argtypes = [u8p, C.c_uint32, u32p]
    L.orc_compress_bound.argtypes = [C.c_uint32, u64p]
    L.orc_compress_bound.restype = C.c_uint64
    L.orc_compress.argtypes = [f32p, C.c_uint32, u64p, C.c_uint32, C.c_double, C.c_uint32, C.c_uint32,
                               u8p, C.c_uint64, u64p]
    L.orc_decompress.argtypes = [u8p, C.c_uint64, f32p, C.c_uint64]
    L.orc_stream_info.argtypes = [u8p, C.c_uint64, u32p, u64p, u64p]
    L.orc_quantize_stage.argtypes = [f32p, C.c_uint32, u64p, C.c_float, C.c_float, C.c_float, C.c_uint32,
                                     C.c_uint32, u16p, i32p, u64p, u64p, u64p]
    L.orc_encode.argtypes = [u16p, C.c_uint64, C.c_uint64, u8p, C.c_uint32, u32p, C.c_uint64, u32p, u64p]
    L.orc_decode.argtypes = [u32p, C.c_uint64, u8p, C.c_uint32, C.c_uint64, u16p]
    if hasattr(L, "orc_mlp_forward"):
        from . import mlp as _mlp  # noqa: F401  (declares its own symbols)
        _mlp._declare(L)


def _p(a, t):
    return a.ctypes.data_as(t)


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


def _chk(st, what):
    if st != OK:
        raise OracleError(st, what)


def _dims3(dims):
    d = np.ones(3, dtype=np.uint64)
    d[: len(dims)] = dims
    return d


# ---------------------------------------------------------------- stages
def value_range(x: np.ndarray):
    x = np.ascontiguousarray(x, dtype=np.float32).ravel()
    lo, hi, same = C.c_float(), C.c_float(), C.c_int()
    anyf = lib().orc_range(_p(x, f32p), x.size, C.byref(lo), C.byref(hi), C.byref(same))
    return bool(anyf), lo.value, hi.value, bool(same.value)


def constants(eb_abs: float):
    a, b, c = C.c_float(), C.c_float(), C.c_float()
    lib().orc_constants(float(eb_abs), C.byref(a), C.byref(b), C.byref(c))
    return np.float32(a.value), np.float32(b.value), np.float32(c.value)


def prequant(x: np.ndarray, inv2eb, ebx2, eb_chk):
    x = np.ascontiguousarray(x, dtype=np.float32).ravel()
    q = np.zeros(x.size, np.int32)
    e = np.zeros(x.size, np.uint8)
    lib().orc_prequant(_p(x, f32p), x.size, float(inv2eb), float(ebx2), float(eb_chk), _p(q, i32p), _p(e, u8p))
    return q, e.astype(bool)


def block_shape(ndim: int):
    b = np.zeros(3, np.uint32)
    lib().orc_block_shape(ndim, _p(b, u32p))
    return tuple(int(v) for v in b)


def lorenzo_block(k: int, ndim: int, block, qb: np.ndarray, inb: np.ndarray | None = None):
    b = np.asarray(block, dtype=np.uint32)
    qb = np.ascontiguousarray(qb, dtype=np.int32).ravel()
    inb = np.ones(qb.size, np.uint8) if inb is None else np.ascontiguousarray(inb, dtype=np.uint8).ravel()
    d = np.zeros(qb.size, np.int64)
    lib().orc_lorenzo_block(k, ndim, _p(b, u32p), _p(qb, i32p), _p(inb, u8p), _p(d, i64p))
    return d


def lorenzo_block_inverse(k: int, ndim: int, block, delta: np.ndarray):
    b = np.asarray(block, dtype=np.uint32)
    v = np.ascontiguousarray(delta, dtype=np.int64).ravel().copy()
    lib().orc_lorenzo_block_inverse(k, ndim, _p(b, u32p), _p(v, i64p))
    return v


def huffman_lengths(counts) -> np.ndarray:
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    ln = np.zeros(c.size, np.uint8)
    _chk(lib().orc_huffman_lengths(_p(c, u64p), c.size, _p(ln, u8p)), "huffman_lengths")
    return ln


def canonical_codes(lengths) -> np.ndarray:
    ln = np.ascontiguousarray(lengths, dtype=np.uint8)
    code = np.zeros(ln.size, np.uint32)
    _chk(lib().orc_canonical_codes(_p(ln, u8p), ln.size, _p(code, u32p)), "canonical_codes")
    return code


def quantize_stage(x: np.ndarray, ndim, dims, inv2eb, ebx2, eb_chk, k=1, R=512):
    x = np.ascontiguousarray(x, dtype=np.float32).ravel()
    d = _dims3(dims)
    blk = block_shape(ndim)
    nb = [int(-(-int(d[a]) // blk[a])) for a in range(3)]
    n_blocks = nb[0] * nb[1] * nb[2]
    bs = blk[0] * blk[1] * blk[2]
    codes = np.zeros(n_blocks * bs, np.uint16)
    anchors = np.zeros(n_blocks, np.int32)
    hist = np.zeros(2 * R, np.uint64)
    no, ne = C.c_uint64(), C.c_uint64()
    _chk(lib().orc_quantize_stage(_p(x, f32p), ndim, _p(d, u64p), float(inv2eb), float(ebx2), float(eb_chk), k, R,
                                  _p(codes, u16p), _p(anchors, i32p), _p(hist, u64p), C.byref(no), C.byref(ne)),
         "quantize_stage")
    return codes, anchors, hist, no.value, ne.value


def encode(codes: np.ndarray, chunk: int, lengths: np.ndarray):
    codes = np.ascontiguousarray(codes, dtype=np.uint16)
    ln = np.ascontiguousarray(lengths, dtype=np.uint8)
    cap = (codes.size * 24 + 31) // 32 + 1
    words = np.zeros(cap, np.uint32)
    nch = -(-codes.size // chunk)
    cb = np.zeros(nch, np.uint32)
    tb = C.c_uint64()
    _chk(lib().orc_encode(_p(codes, u16p), codes.size, chunk, _p(ln, u8p), ln.size, _p(words, u32p), cap,
                          _p(cb, u32p), C.byref(tb)), "encode")
    return words[: (tb.value + 31) // 32].copy(), cb, tb.value


def decode(words: np.ndarray, total_bits: int, lengths: np.ndarray, n: int):
    w = np.ascontiguousarray(words, dtype=np.uint32)
    if w.size == 0:
        w = np.zeros(1, np.uint32)
    ln = np.ascontiguousarray(lengths, dtype=np.uint8)
    out = np.zeros(n, np.uint16)
    _chk(lib().orc_decode(_p(w, u32p), total_bits, _p(ln, u8p), ln.size, n, _p(out, u16p)), "decode")
    return out


# ---------------------------------------------------------------- pipeline
def compress_bound(shape) -> int:
    d = _dims3(shape[::-1])
    return int(lib().orc_compress_bound(len(shape), _p(d, u64p)))


def compress(x: np.ndarray, eb: float, mode: str = "rel", lorenzo_k: int = 1, radius: int = 512) -> np.ndarray:
    """Compress a C-order float32 array (last axis fastest = the format's x)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    shape = x.shape
    ndim = len(shape)
    d = _dims3(shape[::-1])
    cap = int(lib().orc_compress_bound(ndim, _p(d, u64p))) + 4096
    out = np.zeros(cap, np.uint8)
    nb = C.c_uint64()
    st = lib().orc_compress(_p(x, f32p), ndim, _p(d, u64p), 1 if mode == "rel" else 0, float(eb), lorenzo_k,
                            radius, _p(out, u8p), cap, C.byref(nb))
    _chk(st, "compress")
    return out[: nb.value].copy()


def decompress(buf: np.ndarray) -> np.ndarray:
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    ndim, dims, n = C.c_uint32(), np.zeros(3, np.uint64), C.c_uint64()
    _chk(lib().orc_stream_info(_p(buf, u8p), buf.size, C.byref(ndim), _p(dims, u64p), C.byref(n)), "stream_info")
    out = np.zeros(n.value, np.float32)
    _chk(lib().orc_decompress(_p(buf, u8p), buf.size, _p(out, f32p), n.value), "decompress")
    shape = tuple(int(v) for v in dims[: ndim.value][::-1])
    return out.reshape(shape)
