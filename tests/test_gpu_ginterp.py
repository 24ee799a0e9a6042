"""GPU parity of the full-field multilevel interpolation pipeline
(FZMod-Quality: G-Interp predictor + Huffman, §3.3) against the oracle:
byte-identical streams, bit-identical reconstructions (which also equal the
Lorenzo pipeline's: both are lossless on the prequantized field), the
refine passes' tiling (several column tiles, plane runs of 8 and of 32,
ragged edges at every level), many outliers, exceptions, and damaged
streams rejected without a fault."""
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


def _check(x, eb, mode="rel", radius=512, lorenzo_equal=True):
    ref = oracle.compress(x, eb, mode=mode, predictor="ginterp", radius=radius)
    xg = torch.from_numpy(x).cuda()
    buf = fz.compress(xg, eb, mode=mode, predictor="ginterp", radius=radius)
    got = buf.cpu().numpy()
    assert got.size == ref.size
    assert np.array_equal(got, ref)
    y = fz.decompress(buf).cpu().numpy()
    assert np.array_equal(_bits(y), _bits(oracle.decompress(ref)))
    lz = fz.compress(xg, eb, mode=mode, radius=radius)
    raw = [int(np.frombuffer(b[6:8].tobytes(), np.uint16)[0]) & 1 for b in (got, lz[:8].cpu().numpy())]
    if lorenzo_equal and raw[0] == raw[1]:  # a RAW fallback on one side only stores the input itself
        yl = fz.decompress(lz).cpu().numpy()
        assert np.array_equal(_bits(y), _bits(yl))
    return ref


@pytest.mark.parametrize("shape", [(64, 64, 64), (40, 37, 70), (9, 17, 13), (70, 40, 150), (33, 130, 65),
                                   (3, 5, 200), (17, 1, 1), (1, 300, 2)])
def test_streams_and_reconstructions_bit_exact(shape):
    x = synth.smooth_nd(shape, 11).numpy().copy()
    if x.size > 100:
        x.flat[x.size // 3] = np.nan   # exceptions: q 0 feeds the neighbours' predictions
        x.flat[x.size // 2] = -np.inf
    _check(x, 1e-4)


@pytest.mark.parametrize("eb,mode", [(1e-2, "rel"), (1e-3, "rel"), (1e-6, "rel"), (5e-3, "abs")])
def test_bounds_and_modes(eb, mode):
    x = synth.blobs3d((48, 56, 72), seed=4).numpy()
    _check(x, eb, mode=mode)


@pytest.mark.parametrize("radius", [2, 8, 64])
def test_many_outliers(radius):
    """Small radii turn most residuals into outliers (the refine passes look
    each one up in the ascending list)."""
    x = synth.blobs3d((40, 44, 52), seed=6).numpy()
    ref = _check(x, 1e-4, radius=radius)
    n_out = int(np.frombuffer(ref[112:120].tobytes(), np.uint64)[0])
    flags = int(np.frombuffer(ref[6:8].tobytes(), np.uint16)[0])
    assert flags != 0 or n_out > 1000


def test_long_plane_runs():
    """Enough column tiles for runs of 32 planes on the last pass, with a
    ragged last run and ragged tiles in x and y."""
    x = synth.smooth_nd((150, 250, 520), 13).numpy()
    _check(x, 1e-4, lorenzo_equal=False)


def test_full_size_grf_against_oracle():
    """The 512^3 field at REL 1e-4: stream bytes equal the oracle's, the
    reconstruction equals the Lorenzo pipeline's bit for bit, the bound holds,
    and the interpolation stream is smaller than the Lorenzo one."""
    xg = synth.grf3d(512, device="cuda")
    xh = xg.cpu().numpy()
    buf = fz.compress(xg, 1e-4, predictor="ginterp")
    ref = oracle.compress(xh, 1e-4, predictor="ginterp")
    assert buf.numel() == ref.size
    assert np.array_equal(buf.cpu().numpy(), ref)
    del ref
    y = fz.decompress(buf)
    lz = fz.compress(xg, 1e-4)
    yl = fz.decompress(lz)
    assert torch.equal(y.view(torch.int32), yl.view(torch.int32))
    eba = 1e-4 * (float(xg.max()) - float(xg.min()))
    assert float((y.double() - xg.double()).abs().max()) <= eba
    assert buf.numel() < lz.numel()


def test_damaged_streams_are_rejected():
    x = synth.blobs3d((40, 44, 52), seed=6).numpy()
    buf = fz.compress(torch.from_numpy(x).cuda(), 1e-4, predictor="ginterp", radius=8)
    h = buf[:256].cpu().numpy()
    hdr = np.frombuffer(h.tobytes(), np.uint64)
    n_out = int(hdr[112 // 8])
    off_oidx = int(hdr[168 // 8])
    off_bits = int(hdr[200 // 8])
    assert n_out > 2
    # two outlier positions swapped: the list no longer ascends
    b1 = buf.clone()
    a = b1[off_oidx: off_oidx + 4].clone()
    b1[off_oidx: off_oidx + 4] = b1[off_oidx + 4: off_oidx + 8]
    b1[off_oidx + 4: off_oidx + 8] = a
    with pytest.raises(fz.FzError) as e:
        fz.decompress(b1)
    assert e.value.code == 5
    # bitstream bits flipped: a chunk's bit count no longer matches
    b2 = buf.clone()
    b2[off_bits + 40: off_bits + 48] ^= 0x5A
    with pytest.raises(fz.FzError) as e:
        fz.decompress(b2)
    assert e.value.code == 5
    # the context stays usable
    y = fz.decompress(buf).cpu().numpy()
    assert np.array_equal(_bits(y), _bits(oracle.decompress(buf.cpu().numpy())))


def test_unsupported_requests():
    x1 = torch.arange(1000, dtype=torch.float32, device="cuda")
    with pytest.raises(fz.FzError) as e:
        fz.compress(x1, 1e-3, predictor="ginterp")
    assert e.value.code == 7
    x3 = synth.smooth_nd((16, 16, 16), 1).cuda()
    for kw in ({"chunk": 1024}, {"encoder": "shuffle"}):
        with pytest.raises(fz.FzError) as e:
            fz.compress(x3, 1e-3, predictor="ginterp", **kw)
        assert e.value.code == 7
