"""Pins of the oracle's per-block predictor selection: interpolation
predictors, trial costs, block features, the selector network's exact
inference and its training gradients."""
import numpy as np
import pytest
import torch

import oracle
import synth


def _block_coords():
    z, y, x = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    return x.ravel(), y.ravel(), z.ravel()


def _corners(fn):
    cq = np.zeros(8, np.int32)
    for c in range(8):
        cq[c] = fn(8 * (c & 1), 8 * ((c >> 1) & 1), 8 * (c >> 2))
    return cq


def _level_axis(x, y, z):
    """Level s and pass axis of a non-origin block point (the traversal
    order: levels 4, 2, 1; passes x, y, z)."""
    c = (x, y, z)
    for s in (4, 2, 1):
        if all(v % s == 0 for v in c):
            ax = max(a for a in range(3) if (c[a] // s) % 2 == 1)
            return s, ax
    raise AssertionError


def _avail(c, ax, off):
    p = list(c)
    p[ax] += off
    if all(0 <= v < 8 for v in p):
        return True
    return all(v in (0, 8) for v in p)


def test_interp_linear_exact_on_affine_fields():
    fn = lambda x, y, z: 3 * x - 2 * y + 5 * z + 7
    x, y, z = _block_coords()
    q = fn(x, y, z)
    d = oracle.interp_block(False, False, q, corner_q=_corners(fn), corner_in=np.ones(8, np.uint8))
    assert d[0] == q[0]  # the origin keeps q (the anchor)
    checked = 0
    for i in range(1, 512):
        s, ax = _level_axis(x[i], y[i], z[i])
        c = (x[i], y[i], z[i])
        if _avail(c, ax, -s) and _avail(c, ax, s):
            assert d[i] == 0, (c, d[i])
            checked += 1
    assert checked > 200


def test_interp_cubic_exact_on_cubic_polynomials():
    for ax in range(3):
        fn = lambda x, y, z, ax=ax: (x, y, z)[ax] ** 3 - 4 * (x, y, z)[ax] ** 2 + 11
        x, y, z = _block_coords()
        q = fn(x, y, z)
        d = oracle.interp_block(True, False, q, corner_q=_corners(fn), corner_in=np.ones(8, np.uint8))
        hits = 0
        for i in range(1, 512):
            s, a = _level_axis(x[i], y[i], z[i])
            c = (x[i], y[i], z[i])
            if a == ax and all(_avail(c, a, o) for o in (-3 * s, -s, s, 3 * s)):
                assert d[i] == 0
                hits += 1
        assert hits > 0


@pytest.mark.parametrize("cubic", [False, True])
@pytest.mark.parametrize("seed", range(4))
def test_interp_inverse_roundtrip(cubic, seed):
    rng = np.random.default_rng(seed)
    q = rng.integers(-(2 ** 22), 2 ** 22, 512).astype(np.int32)
    inb = np.ones((8, 8, 8), np.uint8)
    if seed % 2:  # a ragged block at the domain edge
        inb[5:, :, :] = 0
        inb[:, :, 6:] = 0
    inb = inb.ravel()
    cin = rng.integers(0, 2, 8).astype(np.uint8)
    cin[0] = 1
    cq = rng.integers(-1000, 1000, 8).astype(np.int32)
    qm = np.where(inb > 0, q, 0)
    d = oracle.interp_block(cubic, False, qm, inb, cq, cin)
    r = oracle.interp_block(cubic, True, d, inb, cq, cin)
    assert np.array_equal(r[inb > 0], qm[inb > 0].astype(np.int64))


def test_trial_costs_and_labels():
    # constant block: Lorenzo-1 and both interpolations leave zeros -> 511
    # one-bit codes and the first id wins; Lorenzo-2's zero padding leaves
    # nonzero residuals next to the block faces
    best, c = oracle.block_costs(np.full(512, 40, np.int32), corner_q=np.full(8, 40, np.int32),
                                 corner_in=np.ones(8, np.uint8))
    assert best == 0 and c[0] == c[2] == c[3] == 511 and c[1] > 511
    # a single huge spike: outliers cost 96 bits
    q = np.zeros(512, np.int32)
    q[511] = 10 ** 6
    _, c = oracle.block_costs(q)
    assert c[0] == 510 + 96
    # the label of every block of a field is the argmin of its costs (ties -> lowest)
    x = synth.stitched3d(64, seed=3, region=32, device="cpu").numpy()
    lab, costs, _ = oracle.field_blocks(x, 1e-4)
    assert np.array_equal(lab, np.argmin(costs, axis=1))


def test_log2fix_definition():
    cases = {0: 0.0, 1: 1.0, 2: 1.5, 3: 2.0, 6: 2.75, 15: 4.0, 16: 4.0625, 31: 5.0, 47: 5.5,
             (1 << 20) - 1: 20.0, (1 << 40) + (1 << 36) - 1: 40.0625}
    for s_, v in cases.items():
        assert oracle.log2fix(s_) == v, (s_, oracle.log2fix(s_), v)


def test_bf16_round_to_nearest_even():
    assert oracle.f32_to_bf16(1.0) == 0x3F80
    assert oracle.f32_to_bf16(1.0 + 2 ** -8) == 0x3F80       # tie -> even
    assert oracle.f32_to_bf16(1.0 + 3 * 2 ** -8) == 0x3F82   # tie -> even
    rng = np.random.default_rng(0)
    v = (rng.standard_normal(2000) * 10.0 ** rng.uniform(-3, 3, 2000)).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    got = np.array([oracle.f32_to_bf16(float(a)) for a in v], np.uint16)
    assert np.array_equal(got, ref)


def test_features_closed_forms():
    st, ft = oracle.block_features(np.full(512, 9, np.int32), corner_q=np.full(8, 9, np.int32),
                                   corner_in=np.ones(8, np.uint8))
    # every statistic vanishes except Lorenzo-2's (zero padding at the faces)
    assert st[[0, 1, 4, 5, 6, 7]].sum() == 0 and st[2] > 0
    assert st[8:26].sum() == 0 and st[29] == 512 and st[30] == 9 and st[31] == 0
    assert st[26:29].tolist() == [1, 1, 1]
    x, y, z = _block_coords()
    st, _ = oracle.block_features(x.astype(np.int32))  # ramp along x, no corners
    assert st[8] == 7 * 64 and st[9] == 0 and st[10] == 0
    assert st[11] == 0 and st[14] == 0 and st[20:23].sum() == 0
    assert st[23] == 64 * (3 + 2 + 1 + 0 + 1 + 2 + 3 + 4) and st[24] == 7
    assert st[31] == 2 * 6 * 64 and st[26:29].tolist() == [0, 0, 0]
    # features are bf16(log2fix(stat))
    for v, f in zip(st, _):
        assert f == oracle.f32_to_bf16(oracle.log2fix(int(v)))


def _rand_weights(rng):
    w = (rng.standard_normal(oracle.NW) * 0.3).astype(np.float32)
    return torch.from_numpy(w).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)


def _bf(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).view(torch.bfloat16).float().double().numpy()


def test_mlp_inference_matches_double_forward():
    rng = np.random.default_rng(3)
    w = _rand_weights(rng)
    W = _bf(w)
    n1, n2 = oracle.NHID * oracle.NFEAT, oracle.NHID
    agree = 0
    for _ in range(200):
        f32 = rng.uniform(0, 20, oracle.NFEAT).astype(np.float32)
        f = torch.from_numpy(f32).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
        best, lg = oracle.mlp_infer(w, f)
        fd = _bf(f)
        h = np.maximum(W[:n1].reshape(64, 32) @ fd + W[n1:n1 + n2], 0)
        lgd = W[n1 + n2:n1 + n2 + 256].reshape(4, 64) @ h + W[-4:]
        srt = np.sort(lgd)
        if srt[-1] - srt[-2] > 1e-2 * max(1.0, abs(srt[-1])):
            assert best == int(np.argmax(lgd))
            agree += 1
        assert np.allclose(lg, lgd, rtol=2e-2, atol=2e-2 * np.abs(lgd).max())
    assert agree > 150


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(11)
    w = _rand_weights(rng)
    nb = 64
    f32 = rng.uniform(0, 10, (nb, oracle.NFEAT)).astype(np.float32)
    feat = torch.from_numpy(f32).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    lab = rng.integers(0, 4, nb).astype(np.uint8)
    loss, g = oracle.mlp_loss_grad(w, feat, lab)
    W = _bf(w)
    assert abs(oracle.mlp_loss_double(W, feat, lab) - loss) < 1e-12
    idx = rng.choice(oracle.NW, 60, replace=False)
    for i in idx:
        e = 1e-6
        Wp, Wm = W.copy(), W.copy()
        Wp[i] += e
        Wm[i] -= e
        fd = (oracle.mlp_loss_double(Wp, feat, lab) - oracle.mlp_loss_double(Wm, feat, lab)) / (2 * e)
        assert abs(fd - g[i]) <= 1e-6 + 1e-4 * abs(fd), (i, fd, g[i])


def test_selector_streams_roundtrip_and_ids():
    x = synth.stitched3d(64, seed=5, region=32, device="cpu").numpy()
    eb = 1e-4
    eb_abs = eb * (float(x.max()) - float(x.min()))
    lab, _, _ = oracle.field_blocks(x, eb)
    for pred in ("interp_linear", "interp_cubic", "exhaustive"):
        buf = oracle.compress(x, eb, predictor=pred)
        y = oracle.decompress(buf)
        assert (np.abs(x.astype(np.float64) - y) <= eb_abs).all()
    buf = oracle.compress(x, eb, predictor="exhaustive")
    off_ids = int(np.frombuffer(buf[144:152].tobytes(), np.uint64)[0])
    ids = np.unpackbits(buf[off_ids:off_ids + (lab.size + 3) // 4][:, None], axis=1, bitorder="little")
    ids = (ids.reshape(-1, 4, 2) * np.array([1, 2])).sum(-1).ravel()[: lab.size]
    assert np.array_equal(ids, lab)
    # random weights: any choice keeps the bound
    w = _rand_weights(np.random.default_rng(0))
    y = oracle.decompress(oracle.compress(x, eb, predictor="mlp", weights=w))
    assert (np.abs(x.astype(np.float64) - y) <= eb_abs).all()


# ---------------------------------------------------------------- hand-worked goldens
GOLD = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def _interp_cases():
    rows = []
    with open(GOLD + "/interp_rounding.txt") as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.mark.parametrize("row", _interp_cases(), ids=lambda r: r[0])
def test_interp_rounding_hand_worked(row):
    """Odd neighbour sums (linear form) and cubic numerators at or next to a
    multiple of 16 plus 8, where the rounding constant and the floor of the
    arithmetic shift decide the prediction: residuals worked by hand in
    tests/golden/interp_rounding.txt."""
    name, pred, px, py, pz, want = row[:6]
    q = np.zeros(512, np.int64)
    cq = np.zeros(8, np.int32)
    for a in row[6:]:
        kind, rest = a.split(":")
        key, val = rest.split("=")
        if kind == "q":
            x, y, z = (int(v) for v in key.split(","))
            q[(z * 8 + y) * 8 + x] = int(val)
        else:
            cq[int(key)] = int(val)
    d = oracle.interp_block(pred == "cubic", False, q, np.ones(512, np.uint8), cq, np.ones(8, np.uint8))
    i = (int(pz) * 8 + int(py)) * 8 + int(px)
    assert int(d[i]) == int(want), (name, int(d[i]))
    # and the inverse restores q exactly
    r = oracle.interp_block(pred == "cubic", True, d, np.ones(512, np.uint8), cq, np.ones(8, np.uint8))
    assert np.array_equal(r, q)


def _round_binary(r, mant_bits):
    """Exact rational r rounded to the binary format with `mant_bits` stored
    mantissa bits and the binary32 exponent range (subnormals kept), to
    nearest, ties to even; returns a Fraction."""
    from fractions import Fraction
    if r == 0:
        return Fraction(0)
    neg = r < 0
    a = -r if neg else r
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    quantum = Fraction(2) ** (max(e, -126) - mant_bits)
    m = a / quantum
    qi, rem = divmod(m.numerator, m.denominator)
    if 2 * rem > m.denominator or (2 * rem == m.denominator and qi % 2 == 1):
        qi += 1
    v = qi * quantum
    return -v if neg else v


def _exact_logits(w16, f16):
    """The selector's inference as a chain of binary32 fused multiply-adds,
    each one the exact product plus accumulator rounded once (IEEE-754
    fusedMultiplyAdd), with the hidden layer rounded to bfloat16."""
    from fractions import Fraction
    val = lambda h: Fraction(float(np.array([int(h) << 16], np.uint32).view(np.float32)[0]))
    W = [val(v) for v in w16]
    F = [val(v) for v in f16]
    nf, nh = oracle.NFEAT, oracle.NHID
    h = []
    for j in range(nh):
        acc = W[nf * nh + j]
        for k in range(nf):
            acc = _round_binary(acc + W[j * nf + k] * F[k], 23)
        acc = acc if acc > 0 else Fraction(0)
        h.append(_round_binary(acc, 7))
    out = []
    for i in range(oracle.NPRED):
        acc = W[nf * nh + nh + oracle.NPRED * nh + i]
        for j in range(nh):
            acc = _round_binary(acc + W[nf * nh + nh + i * nh + j] * h[j], 23)
        out.append(np.float32(float(acc)))
    return np.array(out, np.float32)


def test_mlp_subnormal_chain_hand_worked():
    """The hand-worked case of tests/golden/mlp_subnormal_chain.txt: a
    product below the subnormal grid makes a fused chain, an unfused one and
    a reversed one give different logits and different argmax."""
    w = np.zeros(oracle.NW, np.uint16)
    want, want_best = {}, None
    with open(GOLD + "/mlp_subnormal_chain.txt") as f:
        for line in f:
            p = line.split()
            if not p or p[0].startswith("#"):
                continue
            if p[0] == "weight":
                w[int(p[1])] = int(p[2], 16)
            elif p[0] == "logit":
                want[int(p[1])] = int(p[2], 16)
            elif p[0] == "argmax":
                want_best = int(p[1])
    rng = np.random.default_rng(1)
    for _ in range(3):  # the logits do not depend on the features (W1 = 0)
        f = rng.integers(0, 0x4280, oracle.NFEAT).astype(np.uint16)
        best, lg = oracle.mlp_infer(w, f)
        assert [int(v) for v in lg.view(np.uint32)] == [want[i] for i in range(4)]
        assert best == want_best
    assert np.array_equal(_exact_logits(w, f).view(np.uint32), lg.view(np.uint32))


def test_mlp_inference_is_an_exact_fma_chain():
    """Random bfloat16 weights and features: the oracle's logits equal, bit
    for bit, the chain of exactly rounded binary32 fused multiply-adds in
    index order (which fixes the order of the sums and the rounding of the
    hidden layer)."""
    rng = np.random.default_rng(7)
    for trial in range(6):
        w32 = (rng.standard_normal(oracle.NW) * 0.3).astype(np.float32)
        w = torch.from_numpy(w32).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
        f32 = rng.uniform(0, 24, oracle.NFEAT).astype(np.float32)
        f = torch.from_numpy(f32).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
        best, lg = oracle.mlp_infer(w, f)
        ex = _exact_logits(w, f)
        assert np.array_equal(ex.view(np.uint32), lg.view(np.uint32)), (trial, ex, lg)
        assert best == int(np.argmax(ex))


# ---------------------------------------------------------------- optimizer (Adam, Kingma and Ba 2015, Alg. 1)
def test_adam_hand_worked_steps():
    """Three steps on one parameter, worked in exact decimal arithmetic in
    tests/golden/adam_steps.txt."""
    w, m, v = np.ones(1), np.zeros(1), np.zeros(1)
    with open(GOLD + "/adam_steps.txt") as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for t, g, em, ev, ew in rows:
        w, m, v = oracle.adam_step(w, [float(g)], m, v, int(t), 0.1, 0.9, 0.999, 1e-8)
        assert m[0] == pytest.approx(float(em), rel=1e-14)
        assert v[0] == pytest.approx(float(ev), rel=1e-13)
        assert w[0] == pytest.approx(float(ew), rel=1e-14)


def test_adam_closed_forms():
    """With a constant gradient g the bias-corrected moments are exactly g and
    g^2 at every step, so every step moves w by lr g / (|g| + eps); a zero
    gradient never moves w; the step is invariant to scaling g (up to eps)."""
    rng = np.random.default_rng(4)
    n = 257
    g = rng.standard_normal(n) * np.exp(rng.uniform(-8, 3, n))
    w0 = rng.standard_normal(n)
    lr, eps = 1e-2, 1e-8
    w, m, v = w0.copy(), np.zeros(n), np.zeros(n)
    for t in range(1, 41):
        wp = w
        w, m, v = oracle.adam_step(w, g, m, v, t, lr, 0.9, 0.999, eps)
        assert np.allclose(m / (1 - 0.9 ** t), g, rtol=1e-12, atol=0)
        assert np.allclose(v / (1 - 0.999 ** t), g * g, rtol=1e-11, atol=0)
        assert np.allclose(wp - w, lr * g / (np.abs(g) + eps), rtol=1e-9, atol=1e-15)
    wz, mz, vz = oracle.adam_step(w0, np.zeros(n), np.zeros(n), np.zeros(n), 1, lr)
    assert np.array_equal(wz, w0) and not mz.any() and not vz.any()
    # scale invariance: g and 1000 g give the same step when |g| >> eps
    big = np.abs(g) > 1e-3
    w1, _, _ = oracle.adam_step(w0, g, np.zeros(n), np.zeros(n), 1, lr, eps=0.0)
    w2, _, _ = oracle.adam_step(w0, 1000 * g, np.zeros(n), np.zeros(n), 1, lr, eps=0.0)
    assert np.allclose(w1[big], w2[big], rtol=1e-14, atol=1e-15)
