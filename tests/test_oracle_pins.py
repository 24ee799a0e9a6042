"""Pins of the CPU oracle against what the method and the mathematics fix.

None of these re-type the oracle's own formulas: each check is an invariant, a
closed form, a brute force on tiny inputs, a published worked example
(tests/golden) or an independent textbook algorithm.
"""
import heapq
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def f32(v):
    return np.float32(v)


# ---------------------------------------------------------------- value range (§3.2, §4.2)
@pytest.mark.parametrize("seed", range(8))
def test_value_range_over_finite_values(seed):
    """The REL range is the minimum and maximum over the finite values: numpy's
    nanmin/nanmax after masking the infinities; the same-bits flag is an exact
    comparison of the bit patterns."""
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal(4097) * 10 ** rng.uniform(-3, 3)).astype(np.float32)
    k = int(rng.integers(0, 40))
    idx = rng.choice(x.size, size=k, replace=False)
    x[idx] = rng.choice(np.array([np.nan, np.inf, -np.inf, 0.0, -0.0], np.float32), size=k)
    anyf, lo, hi, same = oracle.value_range(x)
    fin = x[np.isfinite(x)]
    assert anyf == (fin.size > 0)
    assert lo == fin.min() and hi == fin.max()
    assert not same


def test_value_range_special_cases():
    # no finite value at all
    anyf, _, _, same = oracle.value_range(np.array([np.nan, np.inf, -np.inf], np.float32))
    assert not anyf and not same
    # a constant field: every bit pattern equal
    anyf, lo, hi, same = oracle.value_range(np.full(1000, 2.5, np.float32))
    assert anyf and lo == hi == 2.5 and same
    # +0 and -0 compare equal but differ in bits: a zero range, not bit-constant
    anyf, lo, hi, same = oracle.value_range(np.array([0.0, -0.0], np.float32))
    assert anyf and lo == hi == 0.0 and not same
    # all NaN with one payload: bit-constant without a finite value
    anyf, _, _, same = oracle.value_range(np.full(7, np.nan, np.float32))
    assert not anyf and same


# ---------------------------------------------------------------- constants
@pytest.mark.parametrize("eb_abs", [1e-3, 0.0256, 3.7e-7, 1.0, 12345.678, 2.0 ** -20, 1e30])
def test_constants_directed_rounding(eb_abs):
    ebx2, inv2eb, eb_chk = oracle.constants(eb_abs)
    # ebx2 is the largest float32 <= 2*eb_abs*(1-2^-12) (exact rational check)
    target = 2 * Fraction(eb_abs) * (1 - Fraction(1, 4096))
    assert Fraction(float(ebx2)) <= target
    assert Fraction(float(np.nextafter(ebx2, np.float32(np.inf)))) > target
    # eb_chk likewise for eb_abs*(1-2^-23), and strictly below eb_abs
    t2 = Fraction(eb_abs) * (1 - Fraction(1, 2 ** 23))
    assert Fraction(float(eb_chk)) <= t2 < Fraction(float(np.nextafter(eb_chk, np.float32(np.inf))))
    # inv2eb is within one float32 ulp of 1/ebx2 (double then float rounding)
    inv = 1 / Fraction(float(ebx2))
    lo = Fraction(float(np.nextafter(inv2eb, np.float32(0))))
    hi = Fraction(float(np.nextafter(inv2eb, np.float32(np.inf))))
    assert lo < inv < hi


# ---------------------------------------------------------------- prequant
def test_prequant_nearest_bin_bruteforce():
    rng = np.random.default_rng(7)
    x = (rng.standard_normal(4000) * rng.choice([1e-3, 1, 1e3], 4000)).astype(np.float32)
    eb_abs = 1e-2
    ebx2, inv2eb, eb_chk = oracle.constants(eb_abs)
    q, exc = oracle.prequant(x, inv2eb, ebx2, eb_chk)
    e2 = Fraction(float(ebx2))
    for xi, qi, ei in zip(x[:600], q[:600], exc[:600]):
        X = Fraction(float(xi))
        if ei:
            continue
        # q is a nearest integer to x/ebx2 up to the float rounding of x*inv2eb:
        # its bin is never worse than a neighbour's by more than one bin width
        d = abs(X - qi * e2)
        assert d <= abs(X - (qi + 1) * e2) + e2 / 1000 or d <= abs(X - (qi - 1) * e2) + e2 / 1000
        assert d <= e2 / 2 * (1 + Fraction(1, 1000))


def test_prequant_exact_multiples():
    ebx2, inv2eb, eb_chk = oracle.constants(0.5)
    ks = np.array([0, 1, -1, 7, -300, 4096, -65536], np.int64)
    x = (ks.astype(np.float64) * float(ebx2)).astype(np.float32)
    q, exc = oracle.prequant(x, inv2eb, ebx2, eb_chk)
    assert not exc.any()
    assert np.array_equal(q, ks.astype(np.int32))


def test_prequant_exceptions():
    ebx2, inv2eb, eb_chk = oracle.constants(1e-3)
    x = np.array([np.nan, np.inf, -np.inf, 1e30, -1e30, 0.0, 1.0], np.float32)
    q, exc = oracle.prequant(x, inv2eb, ebx2, eb_chk)
    assert exc.tolist() == [True, True, True, True, True, False, False]
    assert q[:5].tolist() == [0] * 5


# ---------------------------------------------------------------- Lorenzo
def _factored_lorenzo(q, k, ndim):
    """(1 - S_a)^k along every axis with zero padding, by array shifts."""
    v = q.astype(np.int64)
    for ax in range(ndim):
        for _ in range(k):
            sh = np.zeros_like(v)
            sl_dst = [slice(None)] * v.ndim
            sl_src = [slice(None)] * v.ndim
            sl_dst[v.ndim - 1 - ax] = slice(1, None)
            sl_src[v.ndim - 1 - ax] = slice(None, -1)
            sh[tuple(sl_dst)] = v[tuple(sl_src)]
            v = v - sh
    return v


@pytest.mark.parametrize("ndim", [1, 2, 3])
@pytest.mark.parametrize("k", [1, 2])
def test_lorenzo_direct_sum_equals_factored_form(ndim, k):
    blk = oracle.block_shape(ndim)
    shape = tuple(blk[:ndim][::-1])
    rng = np.random.default_rng(ndim * 10 + k)
    q = rng.integers(-1000, 1000, size=shape).astype(np.int32)
    d = oracle.lorenzo_block(k, ndim, blk, q)
    assert np.array_equal(d, _factored_lorenzo(q, k, ndim).ravel())


def test_lorenzo_closed_forms_3d():
    blk = (8, 8, 8)
    z, y, x = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    interior = (x > 0) & (y > 0) & (z > 0)
    # order 1: a field independent of one axis has zero interior residual
    d = oracle.lorenzo_block(1, 3, blk, (3 * y + 5 * z * z).astype(np.int32)).reshape(8, 8, 8)
    assert not d[interior].any()
    # order 1: q = x*y*z leaves exactly 1 in the interior
    d = oracle.lorenzo_block(1, 3, blk, (x * y * z).astype(np.int32)).reshape(8, 8, 8)
    assert (d[interior] == 1).all()
    # order 2 annihilates fields linear in x (times anything in y, z)
    interior2 = (x > 1) & (y > 1) & (z > 1)
    d = oracle.lorenzo_block(2, 3, blk, ((2 * x + 1) * (y * y + z)).astype(np.int32)).reshape(8, 8, 8)
    assert not d[interior2].any()
    # the origin residual is the value itself (the anchor)
    q = np.full((8, 8, 8), 77, np.int32)
    for k in (1, 2):
        assert oracle.lorenzo_block(k, 3, blk, q)[0] == 77


@pytest.mark.parametrize("ndim", [1, 2, 3])
@pytest.mark.parametrize("k", [1, 2])
def test_lorenzo_inverse_roundtrip(ndim, k):
    blk = oracle.block_shape(ndim)
    n = blk[0] * blk[1] * blk[2]
    rng = np.random.default_rng(100 + ndim + k)
    q = rng.integers(-(2 ** 22), 2 ** 22, size=n).astype(np.int32)
    d = oracle.lorenzo_block(k, ndim, blk, q)
    assert np.array_equal(oracle.lorenzo_block_inverse(k, ndim, blk, d), q.astype(np.int64))


# ---------------------------------------------------------------- Huffman
def _heap_huffman_cost(counts):
    """Independent textbook Huffman (binary heap); returns the optimal cost."""
    h = [c for c in counts if c > 0]
    if len(h) == 1:
        return h[0]
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a = heapq.heappop(h)
        b = heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def _heap_huffman_maxlen(counts):
    """Longest codeword of an (unlimited) heap Huffman code."""
    h = [(c, i, 0) for i, c in enumerate(counts) if c > 0]
    if len(h) == 1:
        return 1
    heapq.heapify(h)
    nid = len(counts)
    while len(h) > 1:
        a = heapq.heappop(h)
        b = heapq.heappop(h)
        heapq.heappush(h, (a[0] + b[0], nid, max(a[2], b[2]) + 1))
        nid += 1
    return h[0][2]


def _prefix_free(codes, lens):
    words = sorted(format(int(c), f"0{int(l)}b") for c, l in zip(codes, lens) if l)
    return all(not words[i + 1].startswith(words[i]) for i in range(len(words) - 1))


def test_huffman_textbook_example():
    rows = _golden("huffman_textbook.txt")
    counts = np.array([int(r[1]) for r in rows], np.uint64)
    want = [int(r[2]) for r in rows]
    ln = oracle.huffman_lengths(counts)
    assert ln.tolist() == want
    assert int((counts * ln).sum()) == 224


def test_canonical_codes_rfc1951_example():
    rows = _golden("rfc1951_canonical.txt")
    lens = np.array([int(r[1]) for r in rows], np.uint8)
    codes = oracle.canonical_codes(lens)
    assert [format(int(c), f"0{int(l)}b") for c, l in zip(codes, lens)] == [r[2] for r in rows]


def _golden_cases(name):
    """Cases of a golden file: a line 'case <id> [nsym=<n>]' opens a case,
    data rows follow."""
    cases, cur = [], None
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("case "):
                parts = line.split()
                opts = dict(p.split("=") for p in parts[2:])
                cur = {"id": parts[1], "nsym": int(opts.get("nsym", 0)), "rows": []}
                cases.append(cur)
            else:
                cur["rows"].append(line.split())
    return cases


@pytest.mark.parametrize("case", _golden_cases("huffman_ties.txt"), ids=lambda c: c["id"])
def test_huffman_ties_hand_derived(case):
    """Ties between a leaf and a package of equal weight, and between equal
    counts of different symbols, decide which optimal code is chosen: the
    lengths and codewords worked by hand in tests/golden/huffman_ties.txt
    from the stated rule (leaf first on equal weight; leaves by (count,
    symbol))."""
    rows = case["rows"]
    nsym = case["nsym"] or (max(int(r[0]) for r in rows) + 1)
    counts = np.zeros(nsym, np.uint64)
    for r in rows:
        counts[int(r[0])] = int(r[1])
    ln = oracle.huffman_lengths(counts)
    codes = oracle.canonical_codes(ln)
    for r in rows:
        s = int(r[0])
        assert int(ln[s]) == int(r[2]), (case["id"], s, int(ln[s]))
        assert format(int(codes[s]), f"0{int(ln[s])}b") == r[3], (case["id"], s)
    assert int(ln.sum()) == sum(int(r[2]) for r in rows)  # unused symbols get no code


@pytest.mark.parametrize("seed", range(12))
def test_huffman_optimal_kraft_prefix_free(seed):
    rng = np.random.default_rng(seed)
    nsym = int(rng.integers(2, 1025))
    counts = rng.geometric(rng.uniform(0.001, 0.5), size=nsym).astype(np.uint64)
    counts[rng.random(nsym) < 0.3] = 0
    if (counts > 0).sum() < 2:
        counts[:2] = [3, 5]
    ln = oracle.huffman_lengths(counts)
    used = counts > 0
    assert (ln[used] > 0).all() and (ln[~used] == 0).all()
    assert sum(Fraction(1, 2 ** int(l)) for l in ln[used]) == 1  # Kraft equality
    assert ln.max() <= 14
    opt = _heap_huffman_cost([int(c) for c in counts])
    if _heap_huffman_maxlen([int(c) for c in counts]) <= 14:
        assert int((counts * ln).sum()) == opt  # optimal whenever the limit is not needed
    else:
        assert int((counts * ln).sum()) >= opt
    codes = oracle.canonical_codes(ln)
    assert _prefix_free(codes, ln)


@pytest.mark.parametrize("seed", range(30))
def test_huffman_exhaustive_small(seed):
    rng = np.random.default_rng(1000 + seed)
    m = int(rng.integers(2, 7))
    counts = rng.integers(1, 50, size=m).astype(np.uint64)
    ln = oracle.huffman_lengths(counts)
    best = None
    for lv in itertools.product(range(1, m), repeat=m):
        if sum(Fraction(1, 2 ** l) for l in lv) <= 1:
            c = sum(int(a) * b for a, b in zip(counts, lv))
            best = c if best is None else min(best, c)
    assert int((counts * ln).sum()) == best


def _dp_limited_optimum(counts, lmax=14):
    """Independent exact optimum over prefix codes with depth <= lmax: fill
    depths top-down with the heaviest symbols first (optimal lengths are
    monotone in weight); avail = free nodes at the current depth."""
    import functools
    w = sorted((int(c) for c in counts if c > 0), reverse=True)
    n = len(w)
    if n == 1:
        return w[0]
    pre = [0]
    for v in w:
        pre.append(pre[-1] + v)

    @functools.lru_cache(maxsize=None)
    def best(i, d, avail):
        if i == n:
            return 0
        if d > lmax or avail == 0:
            return float("inf")
        avail = min(avail, n - i)
        out = float("inf")
        for k in range(0, avail + 1):
            rest = best(i + k, d + 1, min(2 * (avail - k), n - i - k)) if i + k < n else 0
            out = min(out, (pre[i + k] - pre[i]) * d + rest)
        return out

    return best(0, 1, 2)


@pytest.mark.parametrize("seed", range(6))
def test_length_limited_code_is_optimal_dp(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(16, 23))
    fib = [1, 1]
    while len(fib) < n:
        fib.append(fib[-1] + fib[-2])
    counts = np.array(fib, np.uint64) * np.uint64(rng.integers(1, 4))
    counts = counts[rng.permutation(n)]
    ln = oracle.huffman_lengths(counts)
    assert ln.max() <= 14 and _heap_huffman_maxlen([int(c) for c in counts]) > 14  # the limit binds
    assert sum(Fraction(1, 2 ** int(l)) for l in ln) <= 1
    assert int((counts * ln).sum()) == _dp_limited_optimum(counts)


def test_huffman_single_symbol_and_length_limit():
    c = np.zeros(1024, np.uint64)
    c[512] = 1000
    ln = oracle.huffman_lengths(c)
    assert ln[512] == 1 and ln.sum() == 1
    # Fibonacci counts force a depth-(n-1) tree without the limit
    fib = [1, 1]
    while len(fib) < 40:
        fib.append(fib[-1] + fib[-2])
    c = np.zeros(1024, np.uint64)
    c[:40] = fib
    ln = oracle.huffman_lengths(c)
    assert ln.max() <= 14
    assert sum(Fraction(1, 2 ** int(l)) for l in ln[:40]) <= 1
    assert _prefix_free(oracle.canonical_codes(ln), ln)


# ---------------------------------------------------------------- encode / decode
def test_bit_order_msb_first():
    # lengths 1,2,2 -> canonical codes 0, 10, 11
    lens = np.array([1, 2, 2], np.uint8)
    assert oracle.canonical_codes(lens).tolist() == [0, 2, 3]
    codes = np.array([1, 2, 0, 1] * 8 + [2], np.uint16)  # 10 11 0 10 ... 11
    words, cb, tb = oracle.encode(codes, 1024, lens)
    bits = "".join({0: "0", 1: "10", 2: "11"}[int(c)] for c in codes)
    assert tb == len(bits) and cb.tolist() == [len(bits)]
    want = bits + "0" * (-len(bits) % 32)
    assert [int(want[i:i + 32], 2) for i in range(0, len(want), 32)] == words.tolist()


@pytest.mark.parametrize("chunk", [1, 7, 512, 1024])
def test_encode_decode_roundtrip(chunk):
    rng = np.random.default_rng(chunk)
    counts = rng.integers(0, 200, 1024).astype(np.uint64)
    counts[512] = 5000
    ln = oracle.huffman_lengths(counts)
    used = np.nonzero(counts)[0]
    codes = rng.choice(used, size=3001).astype(np.uint16)
    words, cb, tb = oracle.encode(codes, chunk, ln)
    assert tb == int(sum(int(ln[c]) for c in codes)) == int(cb.sum())
    assert np.array_equal(oracle.decode(words, tb, ln, codes.size), codes)


# ---------------------------------------------------------------- stage-level pins
@pytest.mark.parametrize("shape", [(37,), (1025,), (33, 70), (9, 17, 13), (8, 8, 8)])
def test_codes_hist_outliers_bruteforce(shape):
    x = synth.smooth_nd(shape, seed=len(shape)).numpy()
    x.ravel()[::97] += 5.0  # force some outliers
    ndim = len(shape)
    eb_abs = 1e-3
    ebx2, inv2eb, eb_chk = oracle.constants(eb_abs)
    R = 512
    codes, anchors, hist, n_out, n_exc = oracle.quantize_stage(x, ndim, shape[::-1], inv2eb, ebx2, eb_chk, 1, R)
    assert int(hist.sum()) == codes.size
    assert np.array_equal(hist, np.bincount(codes, minlength=2 * R).astype(np.uint64))
    # brute force: residuals by the factored form on each zero-padded block
    q, exc = oracle.prequant(x, inv2eb, ebx2, eb_chk)
    q = q.reshape(shape)
    blk = oracle.block_shape(ndim)[:ndim][::-1]
    nb = [-(-s // b) for s, b in zip(shape, blk)]
    want_out = 0
    bi = 0
    bs = int(np.prod(blk))
    # iterate blocks in the format's block order (x fastest)
    bs_shape = blk
    for bz in range(nb[0] if ndim == 3 else 1):
        for by in range(nb[-2] if ndim >= 2 else 1):
            for bx in range(nb[-1]):
                idx = (bz, by, bx)[3 - ndim:]
                sl = tuple(slice(i * b, min((i + 1) * b, s)) for i, b, s in zip(idx, blk, shape))
                part = q[sl]
                sub = np.zeros(bs_shape, np.int64)
                sub[tuple(slice(0, p) for p in part.shape)] = part
                d = _factored_lorenzo(sub, 1, ndim).ravel()
                inside = np.zeros(bs_shape, bool)
                inside[tuple(slice(0, p) for p in part.shape)] = True
                inside = inside.ravel()
                cb = codes[bi * bs:(bi + 1) * bs]
                assert anchors[bi] == d[0] and cb[0] == R
                dd = d[1:][inside[1:]]
                want = np.where(np.abs(dd) < R, dd + R, 0)
                assert np.array_equal(cb[1:][inside[1:]], want)
                assert (cb[~inside] == R).all()
                want_out += int((np.abs(dd) >= R).sum())
                bi += 1
    assert bi == int(np.prod(nb))
    assert n_out == want_out and n_exc == int(exc.sum())


# ---------------------------------------------------------------- whole stream
def _bound_ok(x, y, eb_abs):
    x64, y64 = x.astype(np.float64), y.astype(np.float64)
    fin = np.isfinite(x64)
    assert np.array_equal(x.view(np.uint32)[~fin], y.view(np.uint32)[~fin])
    assert (np.abs(x64[fin] - y64[fin]) <= eb_abs).all()


def _hdr_eb_abs(buf):
    return float(np.frombuffer(buf[48:56].tobytes(), np.float64)[0])


@pytest.mark.parametrize("shape,eb,mode", [((4096,), 1e-3, "rel"), ((1,), 1e-2, "rel"), ((3000,), 0.01, "abs"),
                                           ((61, 45), 1e-4, "rel"), ((100, 100), 1e-2, "rel"),
                                           ((17, 9, 33), 1e-3, "rel"), ((24, 24, 24), 1e-5, "rel"),
                                           ((5, 3, 2), 0.1, "abs")])
@pytest.mark.parametrize("k", [1, 2])
def test_roundtrip_error_bound(shape, eb, mode, k):
    x = synth.smooth_nd(shape, seed=sum(shape)).numpy()
    buf = oracle.compress(x, eb, mode, lorenzo_k=k)
    y = oracle.decompress(buf)
    assert y.shape == x.shape
    flags = int(np.frombuffer(buf[6:8].tobytes(), np.uint16)[0])
    if mode == "rel":
        fin = x[np.isfinite(x)]
        eb_abs = eb * (float(fin.max()) - float(fin.min()))
    else:
        eb_abs = eb
    if flags == 0:
        assert _hdr_eb_abs(buf) == eb_abs
    _bound_ok(x.ravel(), y.ravel(), eb_abs)


def test_roundtrip_workload_generators():
    for x, eb in [(synth.blobs3d().numpy(), 1e-3), (synth.hacc1d(1 << 18, device="cpu").numpy(), 1e-4),
                  (synth.cesm2d(90, 180).numpy(), 1e-3), (synth.grf3d(32, device="cpu").numpy(), 1e-3)]:
        buf = oracle.compress(x, eb)
        assert int(np.frombuffer(buf[6:8].tobytes(), np.uint16)[0]) == 0  # compressed, not raw
        y = oracle.decompress(buf)
        _bound_ok(x.ravel(), y.ravel(), eb * (float(x.max()) - float(x.min())))
        assert buf.size < x.nbytes / 2


def test_special_values_and_fallbacks():
    # constant field -> constant stream (header + one float, 16-byte padded)
    x = np.full((10, 11), 3.25, np.float32)
    buf = oracle.compress(x, 1e-3)
    assert buf.size == 272 and int(np.frombuffer(buf[6:8].tobytes(), np.uint16)[0]) == 2
    assert np.array_equal(oracle.decompress(buf), x)
    # NaN / Inf are kept bit for bit as exceptions
    x = synth.smooth_nd((40, 50), 3).numpy()
    x[3, 4] = np.nan
    x[10, 10] = np.inf
    x[20, 1] = -np.inf
    buf = oracle.compress(x, 1e-3)
    y = oracle.decompress(buf)
    fin = np.isfinite(x)
    _bound_ok(x.ravel(), y.ravel(), 1e-3 * (float(x[fin].max()) - float(x[fin].min())))
    # white noise at a tiny bound -> outliers exceed N/8 -> raw stream
    x = np.random.default_rng(0).standard_normal(5000).astype(np.float32)
    buf = oracle.compress(x, 1e-7)
    assert int(np.frombuffer(buf[6:8].tobytes(), np.uint16)[0]) == 1 and buf.size == 256 + 4 * x.size
    assert np.array_equal(oracle.decompress(buf).view(np.uint32), x.view(np.uint32))
    # all NaN -> constant stream when all bits are equal
    x = np.full(100, np.nan, np.float32)
    buf = oracle.compress(x, 1e-3)
    assert buf.size == 272


@pytest.mark.parametrize("eb", [1e-2, 1e-4, 1e-6])
def test_hacc_like_all_bounds_succeed(eb):
    x = synth.hacc1d(1 << 18, device="cpu").numpy()
    buf = oracle.compress(x, eb)
    y = oracle.decompress(buf)
    _bound_ok(x, y, eb * (float(x.max()) - float(x.min())))


def test_corrupt_streams_rejected():
    x = synth.blobs3d((16, 16, 16)).numpy()
    buf = oracle.compress(x, 1e-3)
    with pytest.raises(oracle.OracleError):
        oracle.decompress(buf[:200])
    bad = buf.copy()
    bad[0] ^= 0xFF
    with pytest.raises(oracle.OracleError):
        oracle.decompress(bad)
    bad = buf.copy()
    bad[256 + 512] = 1  # code length table now over-subscribed or inconsistent
    bad[256 + 513] = 1
    with pytest.raises(oracle.OracleError):
        oracle.decompress(bad)
    rng = np.random.default_rng(5)
    bits_off = int(np.frombuffer(buf[200:208].tobytes(), np.uint64)[0])
    for _ in range(20):
        bad = buf.copy()
        i = int(rng.integers(bits_off, buf.size))
        bad[i] ^= 1 << int(rng.integers(0, 8))
        try:
            y = oracle.decompress(bad)
            assert y.shape == x.shape
        except oracle.OracleError:
            pass


# ---------------------------------------------------------------- Huffman chunk size (§3.2 chunked encoder)
def _sections(buf):
    h = buf[:256].tobytes()
    u64 = lambda o: int.from_bytes(h[o:o + 8], "little")
    u32 = lambda o: int.from_bytes(h[o:o + 4], "little")
    return {"chunk": u32(88), "n_blocks": u64(96), "n_chunks": u64(104), "total_bits": u64(128),
            "off_cb": u64(160), "off_bits": u64(200), "total": u64(208)}


@pytest.mark.parametrize("shape,chunks", [((40, 37, 70), (64, 1024, 2048, 4096)), ((9, 8, 17), (64, 4096)),
                                          ((61, 450), (128, 256, 512, 2048, 4096)), ((100, 65), (128, 512)),
                                          ((100003,), (2048, 4096))])
def test_chunk_size_only_regroups_chunk_bits(shape, chunks):
    """Chunk j covers code-stream symbols [jC, min((j+1)C, Npad)): the
    bitstream is the same for every C, chunk j's stored length is the sum of
    the code lengths of its symbols (brute force from the stage codes and
    the codebook), the lengths add up to the total, and the reconstruction
    does not change."""
    x = synth.smooth_nd(shape, seed=len(shape) + 7).numpy()
    eb = 1e-3
    base = oracle.compress(x, eb)
    sb = _sections(base)
    ndim = len(shape)
    ebx2, inv2eb, ebchk = oracle.constants(eb * (float(x.max()) - float(x.min())))
    codes, _, hist, _, _ = oracle.quantize_stage(x, ndim, shape[::-1], inv2eb, ebx2, ebchk)
    lens = oracle.huffman_lengths(hist).astype(np.int64)
    bits_per = lens[codes.astype(np.int64)]
    y0 = oracle.decompress(base)
    for C in chunks:
        buf = oracle.compress(x, eb, chunk=C)
        s = _sections(buf)
        assert s["chunk"] == C and s["n_chunks"] == -(-codes.size // C)
        nw = (s["total_bits"] + 31) // 32
        assert s["total_bits"] == sb["total_bits"]
        assert np.array_equal(buf[s["off_bits"]:s["off_bits"] + 4 * nw], base[sb["off_bits"]:sb["off_bits"] + 4 * nw])
        cb = buf[s["off_cb"]:s["off_cb"] + 4 * s["n_chunks"]].view(np.uint32).astype(np.int64)
        want = np.add.reduceat(bits_per, np.arange(0, codes.size, C))
        assert np.array_equal(cb, want)
        assert int(cb.sum()) == s["total_bits"]
        assert np.array_equal(oracle.decompress(buf).view(np.uint32), y0.view(np.uint32))


def test_chunk_size_rejects_bad_values_and_bad_lengths():
    x = synth.smooth_nd((20, 24, 28), seed=3).numpy()
    for C in (32, 100, 256, 768, 8192):
        with pytest.raises(oracle.OracleError) as e:
            oracle.compress(x, 1e-3, chunk=C)
        assert e.value.code == oracle.EUNSUPPORTED
    with pytest.raises(oracle.OracleError):
        oracle.compress(synth.smooth_nd((5000,), 1).numpy(), 1e-3, chunk=64)  # 64 is for 3D blocks only
    # chunks below the block: 2D first-order Lorenzo only
    x2 = synth.smooth_nd((61, 450), seed=4).numpy()
    for arr, C, k in ((synth.smooth_nd((5000,), 1).numpy(), 256, 1), (x2, 256, 2), (x2, 64, 1), (x2, 1000, 1)):
        with pytest.raises(oracle.OracleError) as e:
            oracle.compress(arr, 1e-3, lorenzo_k=k, chunk=C)
        assert e.value.code == oracle.EUNSUPPORTED
    buf = oracle.compress(x, 1e-3, chunk=64)
    s = _sections(buf)
    cb = buf[s["off_cb"]:s["off_cb"] + 4 * s["n_chunks"]].view(np.uint32)
    # moving one bit from a chunk to its neighbour keeps the total but breaks both chunks
    t = buf.copy()
    tc = t[s["off_cb"]:s["off_cb"] + 4 * s["n_chunks"]].view(np.uint32)
    tc[3] += 1
    tc[4] -= 1
    with pytest.raises(oracle.OracleError) as e:
        oracle.decompress(t)
    assert e.value.code == oracle.ECORRUPT


# ---------------------------------------------------------------- bit-shuffle + zero-word encoder (FZMod-Speed, §3.3)
def _numpy_shuffle(codes, R):
    """The encoder's definition through numpy's bit unpacking: zig-zag the
    residuals, view 64 codes as 32 little-endian rows of 32 bits, transpose
    each 32x32 bit matrix (np.unpackbits / np.packbits), keep the nonzero
    column words in column order."""
    d = codes.astype(np.int64) - R
    v = np.where(d >= 0, 2 * d, -2 * d - 1).astype(np.uint32)
    rows = (v[0::2] | (v[1::2] << 16)).astype("<u4").reshape(-1, 32)           # runs x 32 rows
    bits = np.unpackbits(rows.view(np.uint8).reshape(-1, 32, 4), axis=2, bitorder="little")  # runs x 32 x 32
    cols = np.ascontiguousarray(bits.transpose(0, 2, 1))                         # runs x col b x row r
    words = np.packbits(cols, axis=2, bitorder="little").reshape(-1, 32, 4).view("<u4")[..., 0]  # runs x 32
    nz = words != 0
    maps = (nz.astype(np.uint64) << np.arange(32, dtype=np.uint64)).sum(1).astype(np.uint32)
    return maps, words[nz].astype(np.uint32), nz


@pytest.mark.parametrize("shape", [(40, 37, 70), (9, 8, 17), (61, 450), (100003,)])
@pytest.mark.parametrize("eb", [1e-2, 1e-4])
def test_shuffle_encoder_matches_numpy_transpose(shape, eb):
    x = synth.smooth_nd(shape, seed=len(shape) + 11).numpy()
    buf = oracle.compress(x, eb, encoder="shuffle")
    h = buf[:256].tobytes()
    u64 = lambda o: int.from_bytes(h[o:o + 8], "little")
    if int.from_bytes(h[6:8], "little") != 8:
        pytest.skip("raw fallback")
    ndim = len(shape)
    ebx2, inv2eb, ebchk = oracle.constants(eb * (float(x.max()) - float(x.min())))
    codes, _, _, _, _ = oracle.quantize_stage(x, ndim, shape[::-1], inv2eb, ebx2, ebchk)
    maps, words, nz = _numpy_shuffle(codes, 512)
    off_maps, off_cb, off_bits, tbits = u64(136), u64(160), u64(200), u64(128)
    assert int.from_bytes(h[88:92], "little") == 1024
    assert np.array_equal(buf[off_maps:off_maps + 4 * maps.size].view(np.uint32), maps)
    assert tbits == 32 * words.size
    assert np.array_equal(buf[off_bits:off_bits + 4 * words.size].view(np.uint32), words)
    # chunk j (1024 codes = 16 runs) stores 32 bits per word it keeps
    per_run = nz.sum(1)
    n_tiles = -(-codes.size // 1024)
    want = np.add.reduceat(per_run, np.arange(0, per_run.size, 16)) * 32
    assert np.array_equal(buf[off_cb:off_cb + 4 * n_tiles].view(np.uint32), want)
    # zig-zag values stay below 2R: no column word above bit 9 of either half
    assert not (maps & 0xFC00FC00).any()
    y = oracle.decompress(buf)
    eba = eb * (float(x.max()) - float(x.min()))
    assert (np.abs(y.astype(np.float64) - x) <= eba).all()
    # the same codes as the Huffman stream: identical reconstruction
    assert np.array_equal(y.view(np.uint32), oracle.decompress(oracle.compress(x, eb)).view(np.uint32))


def test_shuffle_special_cases_and_corruption():
    """A field whose residuals are all zero stores no word; bad arguments and
    damaged maps or tile lengths are rejected."""
    x = np.tile(np.arange(64, dtype=np.float32), (8, 8, 1))  # affine in x: Lorenzo-1 residual 1 -> few bits
    buf = oracle.compress(np.zeros((16, 16, 16), np.float32) + 2.0, 1e-3, mode="abs", encoder="shuffle")
    h = buf[:256].tobytes()
    assert int.from_bytes(h[128:136], "little") == 0  # no word at all
    assert (np.abs(oracle.decompress(buf).astype(np.float64) - 2.0) <= 1e-3).all()
    with pytest.raises(oracle.OracleError) as e:
        oracle.compress(x, 1e-3, encoder="shuffle", predictor="interp_linear")
    assert e.value.code == oracle.EUNSUPPORTED
    with pytest.raises(oracle.OracleError) as e:
        oracle.compress(x, 1e-3, encoder="shuffle", chunk=2048)
    assert e.value.code == oracle.EUNSUPPORTED
    buf = oracle.compress(synth.smooth_nd((24, 20, 40), 2).numpy(), 1e-3, encoder="shuffle")
    h = buf[:256].tobytes()
    off_maps, off_cb = int.from_bytes(h[136:144], "little"), int.from_bytes(h[160:168], "little")
    t = buf.copy()
    t[off_maps] ^= 1  # a column word appears or disappears: the tile length no longer matches
    with pytest.raises(oracle.OracleError):
        oracle.decompress(t)
    t = buf.copy()
    t[off_cb:off_cb + 8].view(np.uint32)[:] += np.array([32, -32], np.int64).astype(np.uint32)
    with pytest.raises(oracle.OracleError):
        oracle.decompress(t)


def test_zigzag_closed_forms():
    """Zig-zag order of the residuals (0, -1, 1, -2, 2, ...) through the
    encoder: a run of identical codes c gives one value repeated, whose
    column words are all-ones exactly at the set bits of zigzag(c - R)."""
    R = 512
    for d, v in ((0, 0), (-1, 1), (1, 2), (-2, 3), (2, 4), (-512, 1023), (511, 1022)):
        maps, words, _ = _numpy_shuffle(np.full(64, R + d, np.uint16), R)
        want = [b for b in range(10) if (v >> b) & 1] + [16 + b for b in range(10) if (v >> b) & 1]
        assert [b for b in range(32) if (int(maps[0]) >> b) & 1] == want, d
        assert (words == 0xFFFFFFFF).all()
