"""Batched compression: every stream of a batched call is byte-identical to
the single-field call (and to the oracle), batched decompression matches
single-field decompression bit for bit, and the cached graph replays
correctly with new data of the same shapes."""
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


def _fields(seed=5):
    fs = synth.batch_fields(seed=seed, n3=5, n2=5, scale=0.125, device="cpu")
    nanf = synth.smooth_nd((17, 30, 24), 4).clone()
    nanf[3, 4, 5] = float("nan")
    nanf[9, 0, 23] = float("inf")
    extra = [
        synth.smooth_nd((100003,), 3),                 # 1D, ragged last block
        torch.full((16, 16, 16), 1.5),                 # constant field
        torch.rand(20, 20, 20, generator=torch.Generator().manual_seed(seed)),  # raw fallback at a tiny bound
        nanf,                                          # exceptions
        synth.smooth_nd((5,), 6),                      # tiny 1D
        synth.smooth_nd((33, 65), 7),                  # 2D, ragged blocks
    ]
    fs = fs[:4] + extra[:3] + fs[4:8] + extra[3:] + fs[8:]
    ebs = [1e-7 if f.shape == (20, 20, 20) else 1e-3 for f in fs]
    return [f.contiguous() for f in fs], ebs


def _chunk_of(stream_bytes):
    """The Huffman chunk a stream's header records (0 for raw and constant streams)."""
    return int(np.frombuffer(np.ascontiguousarray(stream_bytes[88:92]).tobytes(), np.uint32)[0])


def _check_batch(xs, ebs, mode="rel", predictor="lorenzo1", with_oracle=True, chunk=0, ctx=None):
    xg = [x.cuda() for x in xs]
    buf, offs = fz.compress_batch(xg, ebs, mode=mode, predictor=predictor, chunk=chunk, ctx=ctx)
    assert len(offs) == len(xs) + 1
    hb = buf[: offs[-1]].cpu().numpy()
    singles = []
    for j, (x, eb) in enumerate(zip(xs, ebs)):
        C = _chunk_of(hb[offs[j]: offs[j] + 256])  # the batch's chunk for this field (tuned or given)
        if chunk:
            assert C in (0, chunk), (j, C)
        one = fz.compress(xg[j], eb, mode=mode, predictor=predictor, chunk=C)
        s = one.cpu().numpy()
        assert offs[j] % 16 == 0
        assert offs[j + 1] - offs[j] == (s.size + 15) // 16 * 16, j
        assert np.array_equal(hb[offs[j]: offs[j] + s.size], s), j
        if with_oracle:
            ref = oracle.compress(x.numpy(), eb, mode=mode, lorenzo_k=2 if predictor == "lorenzo2" else 1, chunk=C)
            assert np.array_equal(s, ref), j
        singles.append(one)
    ys = fz.decompress_batch(buf, offs)
    for j, (x, eb) in enumerate(zip(xs, ebs)):
        y1 = fz.decompress(singles[j])
        assert ys[j].shape == x.shape
        assert np.array_equal(ys[j].cpu().numpy().view(np.uint32), y1.cpu().numpy().view(np.uint32)), j
        xn = x.numpy().astype(np.float64)
        f = np.isfinite(xn)
        if f.any() and mode == "rel":
            eba = eb * (xn[f].max() - xn[f].min())
        else:
            eba = eb
        assert (np.abs(xn[f] - ys[j].cpu().numpy()[f]) <= eba).all(), j
    return buf, offs


def test_batch_matches_single_calls_and_oracle():
    xs, ebs = _fields()
    _check_batch(xs, ebs)


def test_batch_graph_replay_with_new_data():
    xs, ebs = _fields()
    _check_batch(xs, ebs, with_oracle=False)
    # same shapes, new values and bounds: the cached graph runs with the new table
    xs2 = [(x * 1.7 + 0.25).contiguous() for x in xs]
    ebs2 = [e * 2 for e in ebs]
    _check_batch(xs2, ebs2)
    _check_batch(xs2, ebs2, with_oracle=False)
    prof = fz.profile()
    assert prof.batch_graphs >= 1 and prof.batch_graphs == prof.batch_plans


@pytest.mark.parametrize("mode,predictor", [("abs", "lorenzo2"), ("rel", "lorenzo2"), ("abs", "lorenzo1")])
def test_batch_modes(mode, predictor):
    xs, ebs = _fields(seed=8)
    if mode == "abs":
        ebs = [1e-3 if e > 1e-6 else 1e-9 for e in ebs]
    _check_batch(xs, ebs, mode=mode, predictor=predictor)


def test_batch_options_do_not_change_bytes():
    """Launch shapes (tuned or not, graph or eager) never change the bytes
    when the chunk is fixed; the chunk itself is the one tuned parameter that
    does (and every stream records it)."""
    xs, ebs = _fields(seed=9)
    xg = [x.cuda() for x in xs]
    ref, ro = fz.compress_batch(xg, ebs, chunk=1024)
    ref = ref[: ro[-1]].cpu().numpy()
    try:
        for tune, graphs in [(False, False), (False, True), (True, False)]:
            fz.set_batch_options(autotune=tune, graphs=graphs)
            for _ in range(2):
                buf, offs = fz.compress_batch(xg, ebs, chunk=1024)
                assert offs == ro
                assert np.array_equal(buf[: offs[-1]].cpu().numpy(), ref)
    finally:
        fz.set_batch_options(True, True)


def test_batch_padding_is_written():
    """Streams are packed at 16-byte offsets; the bytes between a stream's end
    and the next offset (a RAW stream of N floats, N not a multiple of 4, ends
    unaligned) are zero, whatever the output buffer held before."""
    xs, ebs = _fields(seed=5)
    xg = [x.cuda() for x in xs]
    outs = []
    for fill in (0x00, 0xA5):
        nd = fz._batch_shapes(xg)
        bound = int(fz.lib().fz_compress_batch_bound(len(xg), nd[0], nd[1]))
        o = torch.full((bound,), fill, dtype=torch.uint8, device="cuda")
        buf, offs = fz.compress_batch(xg, ebs, chunk=1024, out=o)
        outs.append(buf[: offs[-1]].cpu().numpy().copy())
    assert np.array_equal(outs[0], outs[1])


def test_batch_output_too_small():
    xs, ebs = _fields(seed=10)
    xg = [x.cuda() for x in xs]
    _, offs = fz.compress_batch(xg, ebs)
    small = torch.zeros(offs[-1] - 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(fz.FzError) as e:
        fz.compress_batch(xg, ebs, out=small)
    assert e.value.code == 4
    # the context stays usable
    buf, offs2 = fz.compress_batch(xg, ebs)
    assert offs2 == offs


def test_batch_full_size_workload():
    """The 64-field workload (32 cubes of side 32-256, 32 lat/lon fields of
    side 512-4096) at REL 1e-4: every stream equals the single-field call and
    every reconstruction is within the bound."""
    xs = synth.batch_fields(seed=5, device="cuda")
    assert len(xs) == 64
    buf, offs = fz.compress_batch(xs, 1e-4)
    ys = fz.decompress_batch(buf, offs)
    for j, x in enumerate(xs):
        C = _chunk_of(buf[offs[j]: offs[j] + 256].cpu().numpy())
        one = fz.compress(x, 1e-4, chunk=C)
        assert torch.equal(buf[offs[j]: offs[j] + one.numel()], one), j
        eba = 1e-4 * (float(x.max()) - float(x.min()))
        assert float((ys[j].double() - x.double()).abs().max()) <= eba, j
        del one


@pytest.mark.parametrize("chunk", [2048, 4096])
def test_batch_explicit_chunk(chunk):
    """A chunk given for the whole batch: every Huffman stream records it and
    equals the single call and the oracle with that chunk; the batched
    decoder reads the multi-block chunks bit-exactly."""
    xs, ebs = _fields(seed=8)
    _check_batch(xs, ebs, chunk=chunk)


def test_batch_autotuner_picks_a_chunk():
    """The autotuner's chunk choice (per kind of field) is one of the block
    size, its double or its quadruple, is reported by the profile, and is the
    chunk every stream of that kind records."""
    ctx = fz.Context(0)
    try:
        xs, ebs = _fields(seed=9)
        _check_batch(xs, ebs, with_oracle=False, ctx=ctx)
        prof = fz.profile(ctx=ctx)
        c3, c12 = int(prof.batch_chunk[0]), int(prof.batch_chunk[1])
        assert c3 in (512, 1024, 2048) and c12 in (1024, 2048, 4096)
    finally:
        ctx.close()
