"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

The stream format is fully determined by the method's readings (rounding,
block order, Huffman tie-break, bit order), so the GPU stream must equal the
oracle's byte for byte and the reconstructions must be bit-identical.  Sizes
span several quantization/encode/decode tiles and ragged tails; the last
tests run the full workload sizes of the benchmark.
"""
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


def _eb_abs(x, eb, mode):
    if mode == "abs":
        return eb
    f = x[np.isfinite(x)]
    if f.size == 0:
        return 0.0
    return eb * (float(f.max()) - float(f.min()))


def _roundtrip_check(x, eb, mode="rel", predictor="lorenzo1", radius=512):
    k = 2 if predictor == "lorenzo2" else 1
    ref = oracle.compress(x, eb, mode, lorenzo_k=k, radius=radius)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    buf = fz.compress(xd, eb, mode, predictor=predictor, radius=radius)
    got = buf.cpu().numpy()
    assert got.size == ref.size, (got.size, ref.size)
    if not np.array_equal(got, ref):
        diff = np.nonzero(got != ref)[0]
        raise AssertionError(f"stream differs at {diff.size} bytes, first at {diff[0]}")
    y = fz.decompress(buf).cpu().numpy()
    yref = oracle.decompress(ref)
    assert y.shape == x.shape
    assert np.array_equal(_bits(y), _bits(yref))
    # the GPU decoder also reads the oracle's stream (cross-decode)
    y2 = fz.decompress(torch.from_numpy(ref).cuda()).cpu().numpy()
    assert np.array_equal(_bits(y2), _bits(yref))
    eba = _eb_abs(x, eb, mode)
    fin = np.isfinite(x)
    assert (np.abs(x[fin].astype(np.float64) - y[fin].astype(np.float64)) <= eba).all()
    assert np.array_equal(_bits(x[~fin]), _bits(y[~fin]))
    return got


SHAPES = [(1,), (37,), (1024,), (5000,), (20000,), (1, 1), (61, 45), (100, 100), (33, 300), (1, 1, 1),
          (8, 8, 8), (17, 9, 33), (40, 37, 70), (16, 64, 130)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("predictor", ["lorenzo1", "lorenzo2"])
def test_stream_bit_exact_shapes(shape, predictor):
    x = synth.smooth_nd(shape, seed=sum(shape)).numpy()
    _roundtrip_check(x, 1e-3, "rel", predictor)


@pytest.mark.parametrize("eb,mode,radius", [(1e-2, "rel", 512), (1e-4, "rel", 512), (1e-5, "rel", 512),
                                            (0.05, "abs", 512), (1e-3, "rel", 64), (1e-3, "rel", 2)])
def test_stream_bit_exact_bounds_and_radius(eb, mode, radius):
    x = synth.blobs3d((40, 48, 56), seed=11).numpy()
    _roundtrip_check(x, eb, mode, radius=radius)


def test_workload_generators_small():
    _roundtrip_check(synth.blobs3d().numpy(), 1e-3)                                  # 64^3, REL 1e-3
    _roundtrip_check(synth.grf3d(64, device="cpu").numpy(), 1e-4)
    _roundtrip_check(synth.hacc1d(1 << 20, device="cpu").numpy(), 1e-4)
    _roundtrip_check(synth.cesm2d(180, 360).numpy(), 1e-3)


def test_special_values():
    x = synth.smooth_nd((30, 40, 20), 5).numpy()
    x[3, 4, 5] = np.nan
    x[10, 10, 10] = np.inf
    x[20, 1, 0] = -np.inf
    x[0, 0, 0] = 3e38
    _roundtrip_check(x, 1e-3)
    # constant field -> CONST stream
    got = _roundtrip_check(np.full((10, 11), 3.25, np.float32), 1e-3)
    assert got.size == 272
    # all NaN with identical bits -> CONST; mixed zeros of both signs -> RAW
    _roundtrip_check(np.full(100, np.nan, np.float32), 1e-3)
    z = np.zeros(64, np.float32)
    z[::2] = -0.0
    _roundtrip_check(z, 1e-3)
    # white noise at a tiny bound -> RAW fallback
    w = np.random.default_rng(0).standard_normal((50, 60)).astype(np.float32)
    got = _roundtrip_check(w, 1e-7)
    assert got.size == 256 + 4 * w.size


@pytest.mark.parametrize("shape", [(40, 37, 70), (100003,), (61, 450)])
def test_prequant_near_the_integer_limit(shape):
    """Values whose scaled magnitude |x / 2eb| lies in [2^22, 2^23) next to
    ordinary ones: the quantizer's two rounding forms must agree with the
    oracle's rint everywhere."""
    s = synth.smooth_nd(shape, seed=12).numpy()
    x = (s * 1000.0).astype(np.float32)
    x.ravel()[::3] += np.float32(3.0e6)  # scaled by 1 / (2 * 0.25): about 6e6
    _roundtrip_check(x, 0.25, "abs")
    _roundtrip_check(x, 0.4, "abs")


@pytest.mark.parametrize("eb", [2.0 ** -15, 2.0 ** -16, 1e-4])
@pytest.mark.parametrize("shape", [(40, 37, 70), (24, 24, 520)])
def test_block_spread_at_the_narrow_state_limit(eb, shape):
    """Blocks whose values sweep the whole value range along x, upwards in
    half of them and downwards in the others, so that a block's quantized
    values differ from its anchor by up to 1 / (2 eb): at REL 2^-15 the
    decoder's 16-bit plane state (REL bounds of at least 2^-15, no
    exceptions) is at its limit; at 2^-16 the spread needs the 32-bit state.
    The long shape gives every decoding warp several work units."""
    z, y, x = np.meshgrid(*(np.arange(n) for n in shape), indexing="ij")
    ramp = (x % 8) / 7.0
    up = ((x // 8 + y // 8 + z // 8) % 2) == 0
    f = (np.where(up, ramp, 1.0 - ramp) * 1000.0 - 200.0).astype(np.float32)
    _roundtrip_check(f, eb, "rel")


@pytest.mark.parametrize("shape", [(40, 48, 72), (24, 40, 520)])
def test_exceptions_and_the_narrow_state(shape):
    """Values near 128 with a range of 1 at REL 1e-4: thousands of exceptions
    whose value was quantized (the float rounding check failed), then a NaN
    at a block origin or an infinity elsewhere (values that were not
    quantized, q = 0).  These streams are below 4096 work units, so the
    32-bit plane state decodes all three; bit-exact against the oracle."""
    s = synth.smooth_nd(shape, seed=21).numpy()
    x = (128.0 + (s - s.min()) / (s.max() - s.min())).astype(np.float32)
    _roundtrip_check(x, 1e-4, "rel")
    y = x.copy()
    y[8, 16, 24] = np.nan
    _roundtrip_check(y, 1e-4, "rel")
    z = x.copy()
    z[9, 17, 30] = np.inf
    _roundtrip_check(z, 1e-4, "rel")


def test_full_exceptions_and_the_narrow_state():
    """A 256 x 512 x 512 field (4096 work units, where a stream with
    exceptions starts to try the 16-bit plane state) near 128 with a range of
    1: rounding-check exceptions only (the 16-bit state decodes), then a NaN
    at a block origin (the offset pass's check picks the 32-bit state).
    Streams byte-identical and reconstructions bit-identical to the
    oracle's."""
    g = synth.grf3d(512, seed=5, device="cuda")[:256].contiguous()
    x = (128.0 + (g - g.min()) / (g.max() - g.min())).float().contiguous()
    for case in range(2):
        xd = x.clone()
        if case == 1:
            xd[8, 16, 24] = float("nan")
        buf = fz.compress(xd, 1e-4)
        y = fz.decompress(buf).cpu().numpy()
        xh = xd.cpu().numpy()
        ref = oracle.compress(xh, 1e-4)
        got = buf.cpu().numpy()
        assert got.size == ref.size and np.array_equal(got, ref), case
        assert int.from_bytes(ref[120:128].tobytes(), "little") > 0  # the stream holds exceptions
        assert np.array_equal(_bits(y), _bits(oracle.decompress(ref))), case


def test_deterministic():
    x = torch.from_numpy(synth.grf3d(64, device="cpu").numpy()).cuda()
    a = fz.compress(x, 1e-4).cpu().numpy()
    b = fz.compress(x, 1e-4).cpu().numpy()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("shape", [(5000,), (61, 45), (17, 9, 33), (64, 64, 64)])
def test_quantize_stage_matches_oracle(shape):
    x = synth.smooth_nd(shape, seed=3).numpy()
    x.ravel()[::101] += 3.0  # outliers
    ndim = len(shape)
    codes, anchors, hist, n_out, n_exc, eb_abs = fz.lorenzo_quantize(torch.from_numpy(x).cuda(), 1e-4, "rel")
    assert eb_abs == _eb_abs(x, 1e-4, "rel")
    ebx2, inv2eb, eb_chk = oracle.constants(eb_abs)
    rc, ra, rh, rno, rne = oracle.quantize_stage(x, ndim, shape[::-1], inv2eb, ebx2, eb_chk, 1, 512)
    assert np.array_equal(codes.cpu().numpy().view(np.uint16), rc)
    assert np.array_equal(anchors.cpu().numpy(), ra)
    assert np.array_equal(hist.cpu().numpy().astype(np.uint64), rh)
    assert (n_out, n_exc) == (rno, rne)
    assert n_out > 0


def _codebook_case(counts):
    h = torch.from_numpy(counts.astype(np.int64)).cuda()
    lens, codes = fz.huffman_codebook(h)
    rl = oracle.huffman_lengths(counts.astype(np.uint64))
    assert np.array_equal(lens.cpu().numpy(), rl)
    rcode = oracle.canonical_codes(rl)
    assert np.array_equal(codes.cpu().numpy().view(np.uint32), rcode)


@pytest.mark.parametrize("seed", range(8))
def test_codebook_matches_oracle(seed):
    rng = np.random.default_rng(seed)
    nsym = int(rng.choice([2, 3, 17, 256, 1000, 1024]))
    c = rng.geometric(rng.uniform(0.001, 0.3), size=nsym).astype(np.int64)
    c[rng.random(nsym) < 0.2] = 0
    if (c > 0).sum() == 0:
        c[0] = 1
    _codebook_case(c)


def test_codebook_edge_cases():
    c = np.zeros(1024, np.int64)
    c[512] = 10 ** 9
    _codebook_case(c)  # single used symbol
    fib = [1, 1]
    while len(fib) < 45:
        fib.append(fib[-1] + fib[-2])
    c = np.zeros(1024, np.int64)
    c[100:145] = fib
    _codebook_case(c)  # forces the 14-bit length limit
    c = np.ones(1024, np.int64)
    _codebook_case(c)  # all equal weights: ties everywhere


def test_corrupt_streams_are_rejected_without_fault():
    x = synth.blobs3d((32, 32, 32), seed=2).numpy()
    buf = fz.compress(torch.from_numpy(x).cuda(), 1e-3)
    host = buf.cpu().numpy()
    hdr = host[:256].tobytes()
    # header corruption
    bad = bytearray(hdr)
    bad[0] ^= 0xFF
    with pytest.raises(fz.FzError) as e:
        fz.decompress(buf, header=bytes(bad))
    assert e.value.code == 5
    # section offsets near 2^64 (offset + length wraps around): rejected on
    # the host before any launch, by every decompress entry point
    for off in (152, 160, 168, 200):
        w = bytearray(hdr)
        w[off:off + 8] = ((1 << 64) - 16).to_bytes(8, "little")
        with pytest.raises(fz.FzError) as e:
            fz.decompress(buf, header=bytes(w))
        assert e.value.code == 5
        out = torch.empty(x.size, dtype=torch.float32, device="cuda")
        hb = C.create_string_buffer(bytes(w), 256)
        assert fz.lib().fz_decompress_noalloc(C.c_void_p(buf.data_ptr()), buf.numel(), hb,
                                              C.c_void_p(out.data_ptr()), out.numel(), None) == 5
    # over-subscribed code-length table
    t = host.copy()
    t[256:256 + 1024] = 1
    with pytest.raises(fz.FzError):
        fz.decompress(torch.from_numpy(t).cuda(), header=hdr)
    # random bit flips in the payload: either a clean error or some output
    rng = np.random.default_rng(1)
    for _ in range(20):
        t = host.copy()
        i = int(rng.integers(1280, t.size))
        t[i] ^= np.uint8(1 << int(rng.integers(0, 8)))
        try:
            fz.decompress(torch.from_numpy(t).cuda(), header=hdr)
        except fz.FzError as err:
            assert err.code == 5
    # truncated stream length
    with pytest.raises(fz.FzError):
        fz.decompress(buf[:1000].clone(), header=hdr)
    torch.cuda.synchronize()


def test_chunk_length_corruption_is_reported():
    """One chunk bit length off by one: the work-unit offsets no longer add up
    to the header's bit total, and the error word reaches the caller (the
    decoder's last CTA writes it to the host)."""
    x = synth.grf3d(64, seed=4, device="cuda")
    buf = fz.compress(x, 1e-4)
    host = buf.cpu().numpy()
    hdr = host[:256].tobytes()
    off_cb = int(np.frombuffer(hdr[160:168], np.uint64)[0])
    t = host.copy()
    cb = t[off_cb:off_cb + 4].view(np.uint32)
    cb[0] += 1
    with pytest.raises(fz.FzError) as e:
        fz.decompress(torch.from_numpy(t).cuda(), header=hdr)
    assert e.value.code == 5
    # the same context decodes a good stream right after
    y = fz.decompress(buf)
    assert float((y.double() - x.double()).abs().max()) <= 1e-4 * (float(x.max()) - float(x.min()))


def test_calls_alternating_between_two_streams():
    """Compress and decompress on two CUDA streams in turn, with host copies
    queued behind them: every stream and reconstruction equals the
    default-stream result bit for bit."""
    x = synth.grf3d(96, seed=6, device="cuda")
    ref = fz.compress(x, 1e-4)
    yref = fz.decompress(ref)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = []
    for i in range(6):
        s = streams[i % 2]
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            xs = x.clone()
            b = fz.compress(xs, 1e-4, stream=s)
            y = fz.decompress(b, stream=s)
            outs.append((b.cpu(), y.cpu()))
    torch.cuda.synchronize()
    for b, y in outs:
        assert torch.equal(b, ref.cpu())
        assert torch.equal(y.view(torch.int32), yref.cpu().view(torch.int32))


def test_bad_arguments():
    x = torch.zeros(100, device="cuda")
    with pytest.raises(fz.FzError) as e:
        fz.compress(x, -1.0)
    assert e.value.code == 1
    with pytest.raises(fz.FzError) as e:
        fz.compress(x, 1e-3, out=torch.empty(100, dtype=torch.uint8, device="cuda"))
    assert e.value.code == 4
    with pytest.raises(fz.FzError) as e:
        fz.compress(x, 1e-3, predictor="interp_cubic", radius=512)
    assert e.value.code == 7


# ---------------------------------------------------------------- full workload sizes
def _full_check(x, eb, predictor="lorenzo1", weights=None, chunk=0):
    """Full workload size: GPU stream == oracle stream byte for byte, the
    GPU reconstruction == the oracle's reconstruction bit for bit (the
    decoder's multi-unit path: every warp claims several work units here),
    and the bound on every value."""
    xd = x.cuda() if not x.is_cuda else x
    wd = torch.from_numpy(weights.view(np.int16)).cuda() if weights is not None else None
    buf = fz.compress(xd, eb, predictor=predictor, selector_weights=wd, chunk=chunk)
    y = fz.decompress(buf)
    f = xd[torch.isfinite(xd)]
    eba = eb * (float(f.max()) - float(f.min()))
    assert float((y.double() - xd.double()).abs().max()) <= eba
    xh = xd.cpu().numpy()
    ref = oracle.compress(xh, eb, predictor=predictor, weights=weights, chunk=chunk)
    got = buf.cpu().numpy()
    assert got.size == ref.size and np.array_equal(got, ref)
    del buf
    yref = oracle.decompress(ref)
    assert np.array_equal(y.cpu().numpy().view(np.uint32), yref.view(np.uint32))
    return got.size


def test_full_512cubed_grf_rel1e4():
    x = synth.grf3d(512, seed=2, device="cuda")
    n = _full_check(x, 1e-4)
    assert n < x.numel() * 4


def test_full_hacc_1d_rel():
    """All three bounds of the particle workload, plus REL 1e-6 (the paper's
    Table 3 blanks that entry for this dataset; every bound must succeed
    here)."""
    x = synth.hacc1d(synth.HACC_N, seed=3, device="cuda")
    for eb in (1e-2, 1e-3, 1e-4, 1e-6):
        _full_check(x, eb)


def test_bounded_wait_times_out_and_context_survives():
    """The look-back's bounded wait, on a predecessor that never publishes,
    gives up after the context's spin limit with FZ_ETIMEOUT; the same
    context then compresses and decompresses normally."""
    fz.set_spin_limit(100000)  # about 50 microseconds
    try:
        assert fz.selftest_bounded_wait() == 6
        assert fz.selftest_bounded_wait() == 6
    finally:
        fz.set_spin_limit(0)
    _roundtrip_check(synth.blobs3d((48, 40, 56), seed=3).numpy(), 1e-3)


def test_pipeline_block_and_chunk_arguments():
    """The pipeline's block shape and chunk size: the defaults, written out,
    give the default stream; other values are rejected before any launch."""
    x = torch.from_numpy(synth.blobs3d((24, 24, 24), seed=4).numpy()).cuda()
    ref = fz.compress(x, 1e-3).cpu()
    assert torch.equal(fz.compress(x, 1e-3, block=(8, 8, 8), chunk=512).cpu(), ref)
    for kw, code in (({"block": (4, 4, 4)}, 7), ({"block": (8, 8, 0)}, 1), ({"chunk": 300}, 7),
                     ({"chunk": 256}, 7), ({"chunk": 8192}, 7)):
        with pytest.raises(fz.FzError) as e:
            fz.compress(x, 1e-3, **kw)
        assert e.value.code == code, kw


def test_full_cesm_2d_rel():
    x = synth.cesm2d(1800, 3600, seed=4)
    for eb in (1e-2, 1e-3, 1e-4):
        _full_check(x, eb)


# ---------------------------------------------------------------- Huffman chunk sizes
@pytest.mark.parametrize("shape,chunks", [((40, 37, 70), (64, 1024, 2048, 4096)), ((17, 9, 33), (64, 4096)),
                                          ((16, 64, 130), (64, 2048)), ((61, 450), (2048, 4096)),
                                          ((100003,), (2048, 4096)), ((5000,), (4096,))])
@pytest.mark.parametrize("predictor", ["lorenzo1", "lorenzo2"])
def test_chunk_sizes_bit_exact(shape, chunks, predictor):
    """Every chunk size of the format: the GPU stream equals the oracle's
    byte for byte, and the GPU decoder (the plane-parallel one for 64-symbol
    chunks, the block decoder for multiples of the block) reconstructs the
    oracle's floats bit for bit; exceptions (NaN, infinity) included."""
    x = synth.smooth_nd(shape, seed=sum(shape) + 1).numpy().copy()
    flat = x.reshape(-1)
    flat[7] = np.nan
    flat[flat.size // 2] = np.inf
    k = 2 if predictor == "lorenzo2" else 1
    xd = torch.from_numpy(x).cuda()
    for C in chunks:
        ref = oracle.compress(x, 1e-3, lorenzo_k=k, chunk=C)
        buf = fz.compress(xd, 1e-3, predictor=predictor, chunk=C)
        got = buf.cpu().numpy()
        assert got.size == ref.size and np.array_equal(got, ref), C
        yref = oracle.decompress(ref)
        y = fz.decompress(buf).cpu().numpy()
        assert np.array_equal(_bits(y), _bits(yref)), C
        y2 = fz.decompress(torch.from_numpy(ref).cuda()).cpu().numpy()
        assert np.array_equal(_bits(y2), _bits(yref)), C


@pytest.mark.parametrize("shape", [(61, 450), (100, 65), (33, 300), (256, 1100)])
def test_chunks_below_the_block_2d(shape):
    """2D first-order Lorenzo streams with chunks of 4, 8 or 16 block rows:
    byte-identical streams, and reconstructions bit-identical to the
    oracle's by the two-pass sub-chunk decoder (its lanes hand each other
    the column state of the rows above their chunk), with exceptions (NaN,
    infinities) and, at radius 4, outliers in most chunks; second-order
    Lorenzo streams reject these chunks before any launch."""
    x = synth.smooth_nd(shape, seed=sum(shape) + 3).numpy().copy()
    flat = x.reshape(-1)
    flat[7] = np.nan
    flat[flat.size // 2] = np.inf
    flat[flat.size // 3] = -np.inf
    xd = torch.from_numpy(x).cuda()
    for C in (128, 256, 512):
        for radius in (512, 4):
            ref = oracle.compress(x, 1e-3, radius=radius, chunk=C)
            buf = fz.compress(xd, 1e-3, radius=radius, chunk=C)
            got = buf.cpu().numpy()
            assert got.size == ref.size and np.array_equal(got, ref), (C, radius)
            yref = oracle.decompress(ref)
            y = fz.decompress(buf).cpu().numpy()
            assert np.array_equal(_bits(y), _bits(yref)), (C, radius)
    with pytest.raises(fz.FzError) as e:
        fz.compress(xd, 1e-3, predictor="lorenzo2", chunk=256)
    assert e.value.code == 7


def test_chunks_below_the_block_2d_corruption():
    """One bit moved between the stored lengths of two neighbouring
    sub-block chunks (total unchanged) is reported as a corrupt stream."""
    x = synth.smooth_nd((61, 450), seed=9).numpy()
    ref = oracle.compress(x, 1e-3, chunk=256)
    h = ref[:256].tobytes()
    off_cb = int.from_bytes(h[160:168], "little")
    t = ref.copy()
    cb = t[off_cb:off_cb + 64].view(np.uint32)
    cb[5] += 1
    cb[6] -= 1
    with pytest.raises(fz.FzError) as e:
        fz.decompress(torch.from_numpy(t).cuda())
    assert e.value.code == 5


@pytest.mark.parametrize("chunk", [128, 256])
def test_full_cesm_2d_chunks_below_the_block(chunk):
    _full_check(synth.cesm2d(1800, 3600, seed=4), 1e-4, chunk=chunk)


def test_chunk64_outliers_and_corruption():
    """64-symbol chunks with many outliers (radius 2) and with the lengths of
    two neighbouring chunks exchanged one bit (total unchanged): the first
    decodes bit-exactly, the second is reported as corrupt."""
    x = synth.blobs3d((40, 48, 56), seed=11).numpy()
    ref = oracle.compress(x, 1e-4, radius=2, chunk=64)
    buf = fz.compress(torch.from_numpy(x).cuda(), 1e-4, radius=2, chunk=64)
    assert np.array_equal(buf.cpu().numpy(), ref)
    assert np.array_equal(_bits(fz.decompress(buf).cpu().numpy()), _bits(oracle.decompress(ref)))
    h = ref[:256].tobytes()
    off_cb = int.from_bytes(h[160:168], "little")
    t = ref.copy()
    cb = t[off_cb:off_cb + 64].view(np.uint32)
    cb[5] += 1
    cb[6] -= 1
    with pytest.raises(fz.FzError) as e:
        fz.decompress(torch.from_numpy(t).cuda())
    assert e.value.code == 5


def test_full_512cubed_grf_chunk64():
    """The headline field with one-plane chunks, at full size, against the
    oracle: stream byte for byte, reconstruction bit for bit."""
    x = synth.grf3d(512, seed=2, device="cuda")
    xd = x.contiguous()
    buf = fz.compress(xd, 1e-4, chunk=64)
    y = fz.decompress(buf)
    xh = xd.cpu().numpy()
    ref = oracle.compress(xh, 1e-4, chunk=64)
    got = buf.cpu().numpy()
    assert got.size == ref.size and np.array_equal(got, ref)
    assert np.array_equal(y.cpu().numpy().view(np.uint32), oracle.decompress(ref).view(np.uint32))
