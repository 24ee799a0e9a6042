"""Pins of the oracle's full-field multilevel interpolation (FZMod-Quality's
G-Interp predictor, §3.3; §3.1-§3.2): hand-worked residuals, the exactness
of the interpolation stencils on polynomials, equality with the block-local
variant where the two availability rules coincide, inverse of forward, and
whole-pipeline reconstructions identical to the Lorenzo pipeline's (both are
lossless on the prequantized field)."""
import pathlib

import numpy as np
import pytest

import oracle
import synth

GOLD = pathlib.Path(__file__).parent / "golden"


def _read_golden(name):
    q, d, cur = [], [], None
    for line in (GOLD / name).read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("q:") or line.startswith("delta:"):
            cur = q if line.startswith("q:") else d
            line = line.split(":", 1)[1]
        if line:
            cur.append([int(t) for t in line.split()])
    return np.array(q, np.int64), np.array(d, np.int64)


def test_line_golden():
    q, d = _read_golden("ginterp_line17.txt")
    q = q.reshape(1, 1, 17)
    assert np.array_equal(oracle.ginterp_field(q)[0, 0], d.ravel())
    assert np.array_equal(oracle.ginterp_field(d.reshape(1, 1, 17), inverse=True), q)


def test_pass_order_golden():
    q, d = _read_golden("ginterp_grid5x5.txt")
    q = q.reshape(1, 5, 5)
    assert np.array_equal(oracle.ginterp_field(q)[0], d)
    assert np.array_equal(oracle.ginterp_field(d.reshape(1, 5, 5), inverse=True), q)


def _level_axis(x, y, z):
    """Level s and axis of a non-anchor point, from its coordinates alone:
    s is the largest power of two (<= 4) dividing all three, the axis the
    last one that s divides an odd number of times."""
    v = x | y | z
    s = 1 if v & 1 else (2 if v & 2 else 4)
    c = (x, y, z)
    a = max(b for b in range(3) if (c[b] // s) & 1)
    return s, a


def _stencil_class(shape_zyx):
    """Per point: 0 anchor, 3 cubic (p-3s and p+3s in the domain), 2 linear
    (p+s in the domain), 1 fallback."""
    nz, ny, nx = shape_zyx
    d = (nx, ny, nz)
    cls = np.zeros(shape_zyx, np.int8)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if x % 8 == 0 and y % 8 == 0 and z % 8 == 0:
                    continue
                s, a = _level_axis(x, y, z)
                c = (x, y, z)[a]
                if c >= 3 * s and c + 3 * s < d[a]:
                    cls[z, y, x] = 3
                elif c + s < d[a]:
                    cls[z, y, x] = 2
                else:
                    cls[z, y, x] = 1
    return cls


@pytest.mark.parametrize("shape", [(9, 13, 30), (17, 17, 17), (4, 21, 11)])
def test_cubic_polynomials_are_annihilated_where_the_cubic_form_applies(shape):
    """The 4-point midpoint rule is exact for polynomials of degree <= 3 (the
    numerator is exactly 16 q), so on a field that is cubic along every axis
    line the residual is 0 wherever the cubic form applies; the linear form
    leaves q - (q[-s] + q[+s] + 1) >> 1, nonzero for a generic cubic."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    q = (3 * x ** 3 - 5 * x ** 2 + 2 * y ** 3 + 7 * y - z ** 3 + 4 * z ** 2 + x * y * z + 11).astype(np.int64)
    res = oracle.ginterp_field(q)
    cls = _stencil_class(shape)
    assert (res[cls == 3] == 0).all()
    anchors = cls == 0
    assert np.array_equal(res[anchors], q[anchors])
    # where the cubic form does not apply, the residual is not generally 0
    assert (res[(cls == 1) | (cls == 2)] != 0).mean() > 0.5


@pytest.mark.parametrize("shape", [(9, 13, 30), (8, 8, 8), (3, 19, 26)])
def test_affine_fields(shape):
    """Both interpolation forms reproduce an affine function exactly (a
    constant: the rounding adds nothing either); the fallback q[-s] leaves
    the slope along its axis times s."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    g = (4, -6, 10)  # slopes along x, y, z (even: the linear form's midpoint is an integer)
    q = (g[0] * x + g[1] * y + g[2] * z + 1000).astype(np.int64)
    res = oracle.ginterp_field(q)
    cls = _stencil_class(shape)
    assert (res[(cls == 2) | (cls == 3)] == 0).all()
    for (zz, yy, xx) in zip(*np.nonzero(cls == 1)):
        s, a = _level_axis(int(xx), int(yy), int(zz))
        assert res[zz, yy, xx] == g[a] * s
    const = oracle.ginterp_field(np.full(shape, -77, np.int64))
    assert (const[cls != 0] == 0).all()


def test_single_block_equals_the_block_local_variant():
    """On a field of exactly one 8x8x8 block the two availability rules are
    the same (in the domain = in the block; the only in-domain corner is the
    origin), so the full-field residuals equal the block-local cubic ones."""
    rng = np.random.default_rng(3)
    q = rng.integers(-5000, 5000, size=(8, 8, 8)).astype(np.int64)
    full = oracle.ginterp_field(q)
    cq = np.zeros(8, np.int32)
    cq[0] = q[0, 0, 0]
    cin = np.zeros(8, np.uint8)
    cin[0] = 1
    local = oracle.interp_block(True, False, q.ravel(), corner_q=cq, corner_in=cin)
    assert np.array_equal(full.ravel(), local)


def test_bigger_fields_differ_from_the_block_local_variant():
    """Across blocks the full-field stencil reaches the neighbouring block:
    on a smooth field it predicts better than the block-local one."""
    f = synth.smooth_nd((24, 24, 24), 2).numpy().astype(np.float64)
    q = np.rint(f * 2000).astype(np.int64)
    full = np.abs(oracle.ginterp_field(q)).sum()
    loc = 0
    for bz in range(3):
        for by in range(3):
            for bx in range(3):
                blk = q[8 * bz:8 * bz + 8, 8 * by:8 * by + 8, 8 * bx:8 * bx + 8]
                cq = np.zeros(8, np.int32)
                cin = np.zeros(8, np.uint8)
                for c in range(8):
                    Z, Y, X = 8 * (bz + (c >> 2)), 8 * (by + ((c >> 1) & 1)), 8 * (bx + (c & 1))
                    if Z < 24 and Y < 24 and X < 24:
                        cq[c], cin[c] = q[Z, Y, X], 1
                loc += np.abs(oracle.interp_block(True, False, blk.ravel(), corner_q=cq, corner_in=cin)).sum()
    assert full < loc


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 2), (1, 1, 17), (5, 5, 1), (9, 9, 9), (17, 3, 2),
                                   (20, 33, 12), (2, 40, 3)])
def test_inverse_of_forward(shape):
    rng = np.random.default_rng(sum(shape))
    q = rng.integers(-(1 << 22), 1 << 22, size=shape).astype(np.int64)
    assert np.array_equal(oracle.ginterp_field(oracle.ginterp_field(q), inverse=True), q)


@pytest.mark.parametrize("shape,eb,mode", [((20, 30, 41), 1e-3, "rel"), ((33, 8, 17), 1e-4, "rel"),
                                           ((16, 16, 16), 1e-2, "abs"), ((9, 2, 400), 1e-3, "rel")])
def test_pipeline_reconstruction_equals_lorenzo(shape, eb, mode):
    """Both predictors are lossless on the prequantized field, so the two
    pipelines reconstruct the same floats, bit for bit (exceptions too)."""
    x = synth.smooth_nd(shape, 5).numpy()
    x = x.copy()
    x.flat[7] = np.nan
    x.flat[len(x.flat) // 2] = np.inf
    a = oracle.compress(x, eb, mode=mode, predictor="ginterp")
    b = oracle.compress(x, eb, mode=mode, predictor="lorenzo1")
    ya, yb = oracle.decompress(a), oracle.decompress(b)
    assert np.array_equal(ya.view(np.uint32), yb.view(np.uint32))
    hdr = np.frombuffer(a[:256].tobytes(), np.uint32)
    assert hdr[84 // 4] == 4  # the predictor field (byte 84) records G-Interp


def test_pipeline_rejects_other_dimensionalities():
    with pytest.raises(oracle.OracleError) as e:
        oracle.compress(np.zeros(100, np.float32) + np.arange(100, dtype=np.float32), 1e-3, predictor="ginterp")
    assert e.value.code == 7
