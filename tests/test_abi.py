"""The C-ABI library loads on a machine without a GPU and exports every
entry point declared in include/fz.h; host-only calls behave as documented."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fz.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fz_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def fzlib():
    from paper_2509_20563_gb300 import build
    build.build()
    import paper_2509_20563_gb300 as fz
    return fz.lib()


def test_exports_every_declared_symbol(fzlib):
    names = _declared()
    assert "fz_compress" in names and "fz_decompress" in names
    for n in names:
        assert hasattr(fzlib, n), n


def test_compress_bound(fzlib):
    d = (C.c_uint64 * 3)(100, 7, 3)
    assert fzlib.fz_compress_bound(3, d) == (256 + 4 * 2100 + 15) // 16 * 16
    assert fzlib.fz_compress_bound(0, d) == 0
    d = (C.c_uint64 * 3)(1 << 20, 1 << 12, 1)
    assert fzlib.fz_compress_bound(2, d) == 0  # N >= 2^32


def test_status_strings(fzlib):
    assert fzlib.fz_status_str(0) == b"ok"
    assert fzlib.fz_status_str(5) == b"corrupt stream"


def test_stream_info_reads_oracle_header(fzlib):
    import paper_2509_20563_gb300 as fz
    import synth
    x = synth.smooth_nd((20, 30, 40), 1).numpy()
    buf = oracle.compress(x, 1e-3)
    shape, eb_abs, flags = fz.stream_info(buf[:256].tobytes())
    assert shape == (20, 30, 40) and flags == 0
    assert eb_abs == pytest.approx(1e-3 * (float(x.max()) - float(x.min())), rel=0, abs=0)
    bad = bytearray(buf[:256].tobytes())
    bad[0] ^= 1
    with pytest.raises(fz.FzError):
        fz.stream_info(bytes(bad))


def test_header_struct_size():
    # the documented header layout is exactly 256 bytes with these offsets
    src = open(os.path.join(ROOT, "include", "fz.h")).read()
    assert "uint8_t pad[40];" in src


def test_null_arguments_rejected_without_gpu(fzlib):
    d = (C.c_uint64 * 3)(8, 1, 1)
    nb = C.c_uint64()
    assert fzlib.fz_compress(None, None, 1, d, 1, 1e-3, None, None, 0, C.byref(nb), None, None) == 1
    assert fzlib.fz_decompress(None, None, 0, None, None, 0, None) == 1


def test_batch_bound_and_argument_checks(fzlib):
    ndim = (C.c_uint32 * 3)(3, 2, 1)
    dims = (C.c_uint64 * 9)(10, 10, 10, 33, 65, 7, 100003, 9, 9)
    want = sum((256 + 4 * n + 15) // 16 * 16 for n in (1000, 33 * 65, 100003))
    assert fzlib.fz_compress_batch_bound(3, ndim, dims) == want
    assert fzlib.fz_compress_batch_bound(0, ndim, dims) == 0
    bad = (C.c_uint32 * 3)(3, 4, 1)
    assert fzlib.fz_compress_batch_bound(3, bad, dims) == 0
    # argument errors are reported before any device work
    offs = (C.c_uint64 * 4)()
    assert fzlib.fz_compress_batch(None, 3, None, ndim, dims, 1, None, None, None, 0, offs, None) == 1
    assert fzlib.fz_decompress_batch(None, 0, None, offs, None, None, None) == 1
    assert fzlib.fz_ctx_set_batch_options(None, 1, 1) == 1
