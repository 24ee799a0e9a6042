"""CPU oracle of the compression path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` import this package.  It compiles ``fz_oracle.c`` with gcc into
``oracle/_build`` and wraps the C functions with ctypes and numpy.  Nothing here touches the CUDA
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


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, plain C11); returns its path."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
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
    L.orc_compress_pred.argtypes = [f32p, C.c_uint32, u64p, C.c_uint32, C.c_double, C.c_uint32, C.c_uint32,
                                    u16p, u8p, C.c_uint64, u64p]
    L.orc_compress_chunk.argtypes = [f32p, C.c_uint32, u64p, C.c_uint32, C.c_double, C.c_uint32, C.c_uint32,
                                     u16p, C.c_uint32, u8p, C.c_uint64, u64p]
    L.orc_compress_full.argtypes = [f32p, C.c_uint32, u64p, C.c_uint32, C.c_double, C.c_uint32, C.c_uint32,
                                    u16p, C.c_uint32, C.c_uint32, u8p, C.c_uint64, u64p]
    L.orc_interp_block.argtypes = [C.c_int, C.c_int, u8p, i32p, u8p, i64p]
    L.orc_interp_block.restype = None
    L.orc_ginterp_field.argtypes = [C.c_int, u64p, i64p]
    L.orc_block_costs.argtypes = [i32p, u8p, i32p, u8p, C.c_uint32, u64p]
    L.orc_log2fix.argtypes = [C.c_uint64]
    L.orc_log2fix.restype = C.c_float
    L.orc_f32_to_bf16.argtypes = [C.c_float]
    L.orc_f32_to_bf16.restype = C.c_uint16
    L.orc_bf16_to_f32.argtypes = [C.c_uint16]
    L.orc_bf16_to_f32.restype = C.c_float
    L.orc_block_features.argtypes = [i32p, u8p, i32p, u8p, C.c_uint32, u64p, u16p]
    L.orc_block_features.restype = None
    L.orc_mlp_infer.argtypes = [u16p, u16p, f32p]
    L.orc_mlp_loss_grad.argtypes = [u16p, u16p, u8p, C.c_uint64, C.POINTER(C.c_double)]
    L.orc_mlp_loss_grad.restype = C.c_double
    L.orc_mlp_loss_double.argtypes = [C.POINTER(C.c_double), u16p, u8p, C.c_uint64]
    L.orc_mlp_loss_double.restype = C.c_double
    dp = C.POINTER(C.c_double)
    L.orc_adam_step.argtypes = [dp, dp, dp, dp, C.c_uint64, C.c_uint32, C.c_double, C.c_double, C.c_double,
                                C.c_double]
    L.orc_adam_step.restype = None
    L.orc_field_blocks.argtypes = [f32p, u64p, C.c_uint32, C.c_double, C.c_uint32, u8p, u64p, u16p]


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


PRED_IDS = {"lorenzo1": 0, "lorenzo2": 1, "interp_linear": 2, "interp_cubic": 3, "ginterp": 4, "mlp": 16,
            "exhaustive": 17}


def compress(x: np.ndarray, eb: float, mode: str = "rel", lorenzo_k: int = 1, radius: int = 512,
             predictor=None, weights: np.ndarray | None = None, chunk: int = 0,
             encoder: str = "huffman") -> np.ndarray:
    """Compress a C-order float32 array (last axis fastest = the format's x).
    ``predictor`` (name or id) overrides ``lorenzo_k``; ``weights`` are the
    selector network's bfloat16 bits for predictor "mlp"; ``chunk`` is the
    Huffman chunk in symbols (0: the block size); ``encoder`` "huffman" or
    "shuffle" (bit-shuffle + zero-word encoding)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    shape = x.shape
    ndim = len(shape)
    d = _dims3(shape[::-1])
    cap = int(lib().orc_compress_bound(ndim, _p(d, u64p))) + 4096
    out = np.zeros(cap, np.uint8)
    nb = C.c_uint64()
    pred = lorenzo_k - 1 if predictor is None else (PRED_IDS[predictor] if isinstance(predictor, str) else predictor)
    wp = None
    if weights is not None:
        weights = np.ascontiguousarray(weights, dtype=np.uint16)
        wp = _p(weights, u16p)
    st = lib().orc_compress_full(_p(x, f32p), ndim, _p(d, u64p), 1 if mode == "rel" else 0, float(eb), pred,
                                 radius, wp, int(chunk), {"huffman": 0, "shuffle": 1}[encoder], _p(out, u8p), cap,
                                 C.byref(nb))
    _chk(st, "compress")
    return out[: nb.value].copy()


# ---------------------------------------------------------------- selector
NFEAT, NHID, NPRED = 32, 64, 4
NW = NHID * NFEAT + NHID + NPRED * NHID + NPRED


def interp_block(cubic: bool, inverse: bool, values, inb=None, corner_q=None, corner_in=None):
    v = np.ascontiguousarray(values, dtype=np.int64).ravel().copy()
    inb = np.ones(512, np.uint8) if inb is None else np.ascontiguousarray(inb, dtype=np.uint8).ravel()
    cq = np.zeros(8, np.int32) if corner_q is None else np.ascontiguousarray(corner_q, dtype=np.int32)
    ci = np.zeros(8, np.uint8) if corner_in is None else np.ascontiguousarray(corner_in, dtype=np.uint8)
    lib().orc_interp_block(int(cubic), int(inverse), _p(inb, u8p), _p(cq, i32p), _p(ci, u8p), _p(v, i64p))
    return v


def ginterp_field(values, inverse: bool = False) -> np.ndarray:
    """Full-field multilevel interpolation of a 3D integer array (C order,
    shape (nz, ny, nx)): residuals of q (forward) or q from the residuals
    (inverse); the anchors (all coordinates multiples of 8) pass through."""
    v = np.ascontiguousarray(values, dtype=np.int64)
    if v.ndim != 3:
        raise ValueError("3D array expected")
    v = v.copy()
    d = _dims3(v.shape[::-1])
    _chk(lib().orc_ginterp_field(int(inverse), _p(d, u64p), _p(v, i64p)), "ginterp_field")
    return v


def block_costs(qb, inb=None, corner_q=None, corner_in=None, R=512):
    qb = np.ascontiguousarray(qb, dtype=np.int32).ravel()
    inb = np.ones(512, np.uint8) if inb is None else np.ascontiguousarray(inb, dtype=np.uint8).ravel()
    cq = np.zeros(8, np.int32) if corner_q is None else np.ascontiguousarray(corner_q, dtype=np.int32)
    ci = np.zeros(8, np.uint8) if corner_in is None else np.ascontiguousarray(corner_in, dtype=np.uint8)
    c = np.zeros(NPRED, np.uint64)
    best = lib().orc_block_costs(_p(qb, i32p), _p(inb, u8p), _p(cq, i32p), _p(ci, u8p), R, _p(c, u64p))
    return best, c


def log2fix(s: int) -> float:
    return lib().orc_log2fix(int(s))


def f32_to_bf16(f: float) -> int:
    return int(lib().orc_f32_to_bf16(float(f)))


def bf16_to_f32(h: int) -> float:
    return lib().orc_bf16_to_f32(int(h))


def block_features(qb, inb=None, corner_q=None, corner_in=None, R=512):
    qb = np.ascontiguousarray(qb, dtype=np.int32).ravel()
    inb = np.ones(512, np.uint8) if inb is None else np.ascontiguousarray(inb, dtype=np.uint8).ravel()
    cq = np.zeros(8, np.int32) if corner_q is None else np.ascontiguousarray(corner_q, dtype=np.int32)
    ci = np.zeros(8, np.uint8) if corner_in is None else np.ascontiguousarray(corner_in, dtype=np.uint8)
    stat = np.zeros(NFEAT, np.uint64)
    feat = np.zeros(NFEAT, np.uint16)
    lib().orc_block_features(_p(qb, i32p), _p(inb, u8p), _p(cq, i32p), _p(ci, u8p), R, _p(stat, u64p),
                             _p(feat, u16p))
    return stat, feat


def mlp_infer(weights, feat):
    w = np.ascontiguousarray(weights, dtype=np.uint16)
    f = np.ascontiguousarray(feat, dtype=np.uint16)
    lg = np.zeros(NPRED, np.float32)
    best = lib().orc_mlp_infer(_p(w, u16p), _p(f, u16p), _p(lg, f32p))
    return best, lg


def mlp_loss_grad(weights, feat, labels):
    w = np.ascontiguousarray(weights, dtype=np.uint16)
    f = np.ascontiguousarray(feat, dtype=np.uint16)
    lb = np.ascontiguousarray(labels, dtype=np.uint8)
    g = np.zeros(NW, np.float64)
    loss = lib().orc_mlp_loss_grad(_p(w, u16p), _p(f, u16p), _p(lb, u8p), lb.size,
                                   g.ctypes.data_as(C.POINTER(C.c_double)))
    return loss, g


def mlp_loss_double(W, feat, labels):
    W = np.ascontiguousarray(W, dtype=np.float64)
    f = np.ascontiguousarray(feat, dtype=np.uint16)
    lb = np.ascontiguousarray(labels, dtype=np.uint8)
    return lib().orc_mlp_loss_double(W.ctypes.data_as(C.POINTER(C.c_double)), _p(f, u16p), _p(lb, u8p), lb.size)


def adam_step(w, g, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam step in float64; returns the updated (w, m, v) as new arrays."""
    w, g, m, v = (np.array(a, dtype=np.float64, copy=True).ravel() for a in (w, g, m, v))
    dp = C.POINTER(C.c_double)
    lib().orc_adam_step(w.ctypes.data_as(dp), g.ctypes.data_as(dp), m.ctypes.data_as(dp), v.ctypes.data_as(dp),
                        w.size, int(t), float(lr), float(beta1), float(beta2), float(eps))
    return w, m, v


def field_blocks(x: np.ndarray, eb: float, mode: str = "rel", radius: int = 512):
    """Exhaustive-trial labels, trial costs and bfloat16 features of every
    block of a 3D field (nz, ny, nx)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    d = _dims3(x.shape[::-1])
    nb = int(np.prod([-(-s // 8) for s in x.shape]))
    lab = np.zeros(nb, np.uint8)
    costs = np.zeros((nb, NPRED), np.uint64)
    feat = np.zeros((nb, NFEAT), np.uint16)
    _chk(lib().orc_field_blocks(_p(x, f32p), _p(d, u64p), 1 if mode == "rel" else 0, float(eb), radius,
                                _p(lab, u8p), _p(costs, u64p), _p(feat, u16p)), "field_blocks")
    return lab, costs, feat


def decompress(buf: np.ndarray) -> np.ndarray:
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    ndim, dims, n = C.c_uint32(), np.zeros(3, np.uint64), C.c_uint64()
    _chk(lib().orc_stream_info(_p(buf, u8p), buf.size, C.byref(ndim), _p(dims, u64p), C.byref(n)), "stream_info")
    out = np.zeros(n.value, np.float32)
    _chk(lib().orc_decompress(_p(buf, u8p), buf.size, _p(out, f32p), n.value), "decompress")
    shape = tuple(int(v) for v in dims[: ndim.value][::-1])
    return out.reshape(shape)
