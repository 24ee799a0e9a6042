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


def _hdr_u64(buf, off, val):
    b = bytearray(buf)
    b[off:off + 8] = int(val).to_bytes(8, "little")
    return bytes(b)


def test_stream_check_rejects_wrapping_offsets(fzlib):
    """fz_stream_check (the validation every decompress runs before any
    launch) on a valid oracle stream, then with each section offset pushed
    to a 16-aligned value near 2^64 (where offset + length wraps around and
    an unsigned chain of sums would pass), and with the stream truncated."""
    import paper_2509_20563_gb300 as fz
    import synth
    x = synth.smooth_nd((20, 30, 40), 1).numpy()
    buf = oracle.compress(x, 1e-3).tobytes()
    hdr, n = buf[:256], len(buf)
    assert fz.stream_check(hdr, n) == 0
    assert fz.stream_check(hdr, n - 1) == 5          # total_bytes beyond the stream
    # off_lens 136, off_ids 144, off_anchors 152, off_chunk_bits 160, off_out_idx 168,
    # off_out_val 176, off_exc_idx 184, off_exc_val 192, off_bits 200
    for off in (136, 152, 160, 168, 176, 184, 192, 200):
        for v in ((1 << 64) - 16, (1 << 64) - 4096, 1 << 63, n + 16):
            assert fz.stream_check(_hdr_u64(hdr, off, v), n) == 5, (off, v)
    # counts that make a section longer than the stream
    for off, v in ((112, (1 << 32) - 1), (120, (1 << 32) - 1), (128, 1 << 62)):
        assert fz.stream_check(_hdr_u64(hdr, off, v), n) == 5, (off, v)
    assert fz.stream_check(hdr, 255) == 1
    assert fzlib.fz_stream_check(None, 4096) == 1


def test_stream_check_rejects_positions_beyond_32_bits(fzlib):
    """A Huffman stream of a field whose padded code stream would need
    positions of 2^32 or more (the format's outlier and exception indices are
    32-bit) is rejected; the same extents are fine for a raw stream."""
    import paper_2509_20563_gb300 as fz
    import synth
    x = synth.smooth_nd((20, 30, 40), 1).numpy()
    hdr = oracle.compress(x, 1e-3).tobytes()[:256]

    def consistent(dims):
        # a header whose sections are laid out for `dims` (no outliers or
        # exceptions, one bit per code); the check reads nothing past it
        nb = 1
        for d in dims:
            nb *= -(-d // 8)
        a16 = lambda v: (v + 15) // 16 * 16
        tb = nb * 512
        o_anch = a16(256 + 1024)
        o_cb = a16(o_anch + 4 * nb)
        o_oi = a16(o_cb + 4 * nb)
        o_bits = o_oi
        total = a16(o_bits + 4 * (-(-tb // 32)))
        h = hdr
        for off, v in ((16, dims[0]), (24, dims[1]), (32, dims[2]), (96, nb), (104, nb), (112, 0), (120, 0),
                       (128, tb), (136, 256), (144, 0), (152, o_anch), (160, o_cb), (168, o_oi), (176, o_oi),
                       (184, o_oi), (192, o_oi), (200, o_bits), (208, total)):
            h = _hdr_u64(h, off, v)
        return h, total
    h, total = consistent((20, 30, 40))
    assert fz.stream_check(h, total) == 0
    # 1620 x 1620 x 1630 has fewer than 2^32 values, its 8x8x8 blocks
    # (1624 x 1624 x 1632) more than 2^32 code positions
    assert 1620 * 1620 * 1630 < (1 << 32) < 1624 * 1624 * 1632
    h, total = consistent((1620, 1620, 1630))
    assert fz.stream_check(h, total) == 5
    h, total = consistent((1600, 1600, 1600))
    assert fz.stream_check(h, total) == 0


def test_struct_layout_matches_header(tmp_path):
    """The ctypes mirror of fz_pipeline and the documented fz_header offsets
    agree with what a C compiler makes of include/fz.h."""
    import subprocess
    import paper_2509_20563_gb300 as fz
    src = tmp_path / "layout.c"
    fields_h = ["magic", "version", "flags", "ndim", "eb_mode", "dims", "eb", "eb_abs", "ebx2_bits",
                "inv2eb_bits", "ebchk_bits", "radius", "block", "predictor", "chunk", "n_blocks", "n_chunks",
                "n_out", "n_exc", "total_bits", "off_lens", "off_ids", "off_anchors", "off_chunk_bits",
                "off_out_idx", "off_out_val", "off_exc_idx", "off_exc_val", "off_bits", "total_bytes"]
    fields_p = ["struct_size", "predictor", "radius", "block", "chunk", "encoder", "selector_weights"]
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{ROOT}/include/fz.h"', "int main(void){"]
    lines += [f'printf("h {f} %zu\\n", offsetof(fz_header, {f}));' for f in fields_h]
    lines += [f'printf("p {f} %zu\\n", offsetof(fz_pipeline, {f}));' for f in fields_p]
    lines += ['printf("hs %zu\\nps %zu\\n", sizeof(fz_header), sizeof(fz_pipeline)); return 0;}']
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-o", str(exe), str(src)], check=True)
    out = dict((" ".join(l.split()[:-1]), int(l.split()[-1]))
               for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines())
    assert out["hs"] == 256
    assert out["ps"] == C.sizeof(fz.Pipeline)
    for f in fields_p:
        assert out[f"p {f}"] == getattr(fz.Pipeline, f).offset, f
    # the oracle writes the header by byte offset: the same offsets
    want = {"magic": 0, "version": 4, "flags": 6, "ndim": 8, "eb_mode": 12, "dims": 16, "eb": 40, "eb_abs": 48,
            "ebx2_bits": 56, "inv2eb_bits": 60, "ebchk_bits": 64, "radius": 68, "block": 72, "predictor": 84,
            "chunk": 88, "n_blocks": 96, "n_chunks": 104, "n_out": 112, "n_exc": 120, "total_bits": 128,
            "off_lens": 136, "off_ids": 144, "off_anchors": 152, "off_chunk_bits": 160, "off_out_idx": 168,
            "off_out_val": 176, "off_exc_idx": 184, "off_exc_val": 192, "off_bits": 200, "total_bytes": 208}
    for f, o in want.items():
        assert out[f"h {f}"] == o, f


def test_pipeline_and_spin_limit_argument_checks(fzlib):
    assert fzlib.fz_ctx_set_spin_limit(None, 100) == 1
    assert fzlib.fz_selftest_bounded_wait(None, None) == 1
