"""GPU: the bit-shuffle + zero-word encoder of FZMod-Speed (§3.3) against the
oracle -- streams byte for byte, reconstructions bit for bit -- over every
dimensionality, both Lorenzo orders, ragged sizes, outliers, exceptions and
the fallbacks; full size; damaged streams reported without a fault."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
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


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)


def _check(x, eb, mode="rel", predictor="lorenzo1", radius=512):
    k = 2 if predictor == "lorenzo2" else 1
    ref = oracle.compress(x, eb, mode, lorenzo_k=k, radius=radius, encoder="shuffle")
    buf = fz.compress(torch.from_numpy(np.ascontiguousarray(x)).cuda(), eb, mode, predictor=predictor, radius=radius,
                      encoder="shuffle")
    got = buf.cpu().numpy()
    assert got.size == ref.size, (got.size, ref.size)
    if not np.array_equal(got, ref):
        d = np.nonzero(got != ref)[0]
        raise AssertionError(f"stream differs at {d.size} bytes, first at {d[0]}")
    yref = oracle.decompress(ref)
    y = fz.decompress(buf).cpu().numpy()
    assert np.array_equal(_bits(y), _bits(yref))
    y2 = fz.decompress(torch.from_numpy(ref).cuda()).cpu().numpy()
    assert np.array_equal(_bits(y2), _bits(yref))
    return got


SHAPES = [(1,), (37,), (1024,), (5000,), (100003,), (1, 1), (61, 45), (100, 100), (33, 300), (1, 1, 1),
          (8, 8, 8), (17, 9, 33), (40, 37, 70), (16, 64, 130)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("predictor", ["lorenzo1", "lorenzo2"])
def test_shuffle_bit_exact_shapes(shape, predictor):
    x = synth.smooth_nd(shape, seed=sum(shape) + 3).numpy()
    _check(x, 1e-3, "rel", predictor)


@pytest.mark.parametrize("eb,mode,radius", [(1e-2, "rel", 512), (1e-4, "rel", 512), (1e-5, "rel", 512),
                                            (0.05, "abs", 512), (1e-3, "rel", 64), (1e-3, "rel", 2)])
def test_shuffle_bounds_radius_outliers(eb, mode, radius):
    x = synth.blobs3d((40, 48, 56), seed=11).numpy()
    flags = int(np.frombuffer(_check(x, eb, mode, radius=radius)[6:8].tobytes(), np.uint16)[0])
    assert flags in (1, 8)


def test_shuffle_special_values_and_fallbacks():
    x = synth.smooth_nd((30, 40, 20), 5).numpy()
    x[3, 4, 5] = np.nan
    x[10, 10, 10] = np.inf
    x[20, 1, 0] = -np.inf
    _check(x, 1e-3)
    _check(synth.smooth_nd((2000,), 2).numpy().copy(), 1e-3)
    assert _check(np.full((10, 11), 3.25, np.float32), 1e-3).size == 272          # constant
    w = np.random.default_rng(0).standard_normal((50, 60)).astype(np.float32)
    assert _check(w, 1e-7).size == 256 + 4 * w.size                                 # raw


def test_shuffle_full_size_512cubed():
    x = synth.grf3d(512, seed=2, device="cuda")
    buf = fz.compress(x, 1e-4, encoder="shuffle")
    y = fz.decompress(buf)
    ref = oracle.compress(x.cpu().numpy(), 1e-4, encoder="shuffle")
    got = buf.cpu().numpy()
    assert got.size == ref.size and np.array_equal(got, ref)
    assert np.array_equal(y.cpu().numpy().view(np.uint32), oracle.decompress(ref).view(np.uint32))


def test_shuffle_full_size_hacc_and_cesm():
    for x, eb in ((synth.hacc1d(synth.HACC_N, seed=3, device="cuda"), 1e-3), (synth.cesm2d(1800, 3600, seed=4), 1e-4)):
        xd = x.contiguous().cuda()
        buf = fz.compress(xd, eb, encoder="shuffle")
        y = fz.decompress(buf)
        ref = oracle.compress(xd.cpu().numpy(), eb, encoder="shuffle")
        assert np.array_equal(buf.cpu().numpy(), ref)
        assert np.array_equal(y.cpu().numpy().view(np.uint32), oracle.decompress(ref).view(np.uint32))


def test_shuffle_damaged_streams_and_noalloc():
    x = synth.blobs3d((32, 40, 48), seed=2).numpy()
    buf = fz.compress(torch.from_numpy(x).cuda(), 1e-3, encoder="shuffle")
    host = buf.cpu().numpy()
    h = host[:256].tobytes()
    off_maps, off_cb = int.from_bytes(h[136:144], "little"), int.from_bytes(h[160:168], "little")
    # damages that change how many words a tile stores, or set bit planes at
    # or above 2R (a map change that keeps both is a different valid stream)
    for pos, val in ((off_maps + 1, 0xFF), (off_maps + 40, 0x01), (off_maps + 3, 0x80)):
        t = host.copy()
        t[pos] ^= val
        with pytest.raises(fz.FzError) as e:
            fz.decompress(torch.from_numpy(t).cuda(), header=h)
        assert e.value.code == 5
    t = host.copy()
    t[off_cb:off_cb + 8].view(np.uint32)[:] += np.array([32, -32], np.int64).astype(np.uint32)
    with pytest.raises(fz.FzError) as e:
        fz.decompress(torch.from_numpy(t).cuda(), header=h)
    assert e.value.code == 5
    # the no-alloc entry point reads shuffle streams too
    ref = fz.decompress(buf)
    out = torch.empty_like(ref)
    hb = C.create_string_buffer(h, 256)
    for _ in range(2):
        out.fill_(-1)
        assert fz.lib().fz_decompress_noalloc(C.c_void_p(buf.data_ptr()), buf.numel(), hb, C.c_void_p(out.data_ptr()),
                                              out.numel(), None) == 0
        assert torch.equal(out.view(torch.int32), ref.view(torch.int32))


def test_shuffle_rejects_unsupported_pipelines():
    x = torch.from_numpy(synth.blobs3d((24, 24, 24), seed=4).numpy()).cuda()
    for kw in ({"predictor": "interp_cubic"}, {"chunk": 512}):
        with pytest.raises(fz.FzError) as e:
            fz.compress(x, 1e-3, encoder="shuffle", **kw)
        assert e.value.code == 7
