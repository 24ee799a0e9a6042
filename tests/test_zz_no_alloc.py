"""fz_decompress_noalloc (fixed scratch, no allocation) gives the same floats
as fz_decompress, bit for bit, on two calls in a row; oversized and
unsupported streams are rejected.  Collected last on purpose: it must also
pass after every other test has used the library."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

fz = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global fz
    from paper_2509_20563_gb300 import build
    build.build()
    import paper_2509_20563_gb300 as m
    m.lib()
    fz = m


def _bits(t):
    return t.cpu().numpy().view(np.uint32)


def _fields():
    nanf = synth.smooth_nd((17, 30, 24), 4).clone()
    nanf[3, 4, 5] = float("nan")
    spiky = synth.blobs3d((40, 37, 70), seed=3).clone()
    spiky[5, 5, ::7] += 50.0  # outliers
    return [
        (synth.blobs3d((64, 64, 64), seed=1), 1e-3, "lorenzo1"),
        (spiky, 1e-4, "lorenzo1"),
        (nanf, 1e-3, "lorenzo2"),
        (synth.smooth_nd((333, 517), 7), 1e-4, "lorenzo1"),
        (synth.smooth_nd((100003,), 3), 1e-3, "lorenzo2"),
        (torch.full((16, 16, 16), 1.5), 1e-3, "lorenzo1"),                               # CONST stream
        (torch.rand(20, 20, 20, generator=torch.Generator().manual_seed(1)), 1e-7, "lorenzo1"),  # RAW stream
    ]


@pytest.mark.parametrize("case", range(7))
def test_noalloc_matches_decompress_twice(case):
    x, eb, pred = _fields()[case]
    xg = x.contiguous().cuda()
    buf = fz.compress(xg, eb, predictor=pred)
    ref = fz.decompress(buf)
    out = torch.empty_like(ref)
    for _ in range(2):
        out.fill_(-1.0)
        fz.decompress_noalloc(buf, out=out)
        assert np.array_equal(_bits(out), _bits(ref))
    # header read from the device stream
    plain = buf.clone()
    assert not hasattr(plain, "fz_header")
    y = fz.decompress_noalloc(plain)
    assert np.array_equal(_bits(y), _bits(ref))


def test_noalloc_limit_and_unsupported():
    lib = fz.lib()
    assert lib.fz_decompress_noalloc(None, 0, None, None, 0, None) == 1
    # one chunk more than the fixed scratch holds: 65 x 32 x 32 blocks of 8^3
    x = synth.smooth_nd((256, 256, 520), 2).cuda()
    buf = fz.compress(x, 1e-3)
    with pytest.raises(fz.FzError) as e:
        fz.decompress_noalloc(buf)
    assert e.value.code == 4
    # exactly at the limit: accepted
    x2 = x[:, :, :512].contiguous()
    buf2 = fz.compress(x2, 1e-3)
    assert np.array_equal(_bits(fz.decompress_noalloc(buf2)), _bits(fz.decompress(buf2)))
    # per-block predictor selection needs a field-sized code buffer
    x3 = synth.stitched3d(64, seed=3, region=32, device="cuda")
    buf3 = fz.compress(x3, 1e-4, predictor="exhaustive")
    with pytest.raises(fz.FzError) as e:
        fz.decompress_noalloc(buf3)
    assert e.value.code == 7


def test_noalloc_plane_chunks_twice():
    """A stream with one-plane (64-symbol) Huffman chunks, decoded by the
    plane-parallel decoder with exceptions written afterwards: the no-alloc
    entry point gives fz_decompress's floats on two calls in a row."""
    x = synth.smooth_nd((40, 37, 70), 5).clone()
    x[3, 4, 5] = float("nan")
    xg = x.contiguous().cuda()
    buf = fz.compress(xg, 1e-3, chunk=64)
    ref = fz.decompress(buf)
    out = torch.empty_like(ref)
    for _ in range(2):
        out.fill_(-1.0)
        fz.decompress_noalloc(buf, out=out)
        assert np.array_equal(_bits(out), _bits(ref))


@pytest.mark.parametrize("chunk", [128, 512])
def test_noalloc_2d_chunks_below_the_block_twice(chunk):
    """A 2D stream whose chunks are block rows, decoded by the sub-chunk
    decoder (outliers at radius 8, an exception): the no-alloc entry point
    gives fz_decompress's floats on two calls in a row."""
    x = synth.smooth_nd((333, 517), 8).clone()
    x[100, 200] = float("inf")
    xg = x.contiguous().cuda()
    buf = fz.compress(xg, 1e-4, radius=8, chunk=chunk)
    ref = fz.decompress(buf)
    out = torch.empty_like(ref)
    for _ in range(2):
        out.fill_(-1.0)
        fz.decompress_noalloc(buf, out=out)
        assert np.array_equal(_bits(out), _bits(ref))
