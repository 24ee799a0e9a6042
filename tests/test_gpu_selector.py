"""GPU parity of the per-block predictor selection against the oracle, the
selector network's gradients against the oracle's double-precision ones,
and the trained network's compression ratio against plain Lorenzo and the
exhaustive trial."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

fz = None
sel = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global fz, sel
    from paper_2509_20563_gb300 import build
    build.build()
    import paper_2509_20563_gb300 as m
    import paper_2509_20563_gb300.selector as s
    m.lib()
    fz, sel = m, s


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)


def _rand_weights(seed):
    w = (np.random.default_rng(seed).standard_normal(oracle.NW) * 0.3).astype(np.float32)
    return torch.from_numpy(w).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)


@pytest.mark.parametrize("shape", [(64, 64, 64), (40, 37, 70), (9, 17, 13)])
def test_block_report_matches_oracle(shape):
    x = synth.stitched3d(64, seed=7, region=32, device="cpu")[: shape[0], : shape[1], : shape[2]].contiguous()
    lab, cst, fea = fz.block_report(x.cuda(), 1e-4)
    rl, rc, rf = oracle.field_blocks(x.numpy(), 1e-4)
    assert np.array_equal(lab.cpu().numpy(), rl)
    assert np.array_equal(cst.cpu().numpy().astype(np.uint64), rc)
    assert np.array_equal(fea.cpu().numpy().view(np.uint16), rf)


@pytest.mark.parametrize("pred", ["interp_linear", "interp_cubic", "exhaustive", "mlp"])
@pytest.mark.parametrize("shape", [(64, 64, 64), (40, 37, 70)])
def test_selector_streams_bit_exact(pred, shape):
    x = synth.stitched3d(64, seed=9, region=32, device="cpu")[: shape[0], : shape[1], : shape[2]].numpy().copy()
    x[3, 4, 5] = np.nan  # an exception inside a block
    w = _rand_weights(5) if pred == "mlp" else None
    ref = oracle.compress(x, 1e-4, predictor=pred, weights=w)
    wd = torch.from_numpy(w.view(np.int16)).cuda() if w is not None else None
    buf = fz.compress(torch.from_numpy(x).cuda(), 1e-4, predictor=pred, selector_weights=wd)
    got = buf.cpu().numpy()
    assert got.size == ref.size
    assert np.array_equal(got, ref)
    y = fz.decompress(buf).cpu().numpy()
    yref = oracle.decompress(ref)
    assert np.array_equal(_bits(y), _bits(yref))
    f = np.isfinite(x)
    eba = 1e-4 * (float(x[f].max()) - float(x[f].min()))
    assert (np.abs(x[f].astype(np.float64) - y[f]) <= eba).all()


def test_selector_subnormal_chain_matches_oracle():
    """Weights whose logits differ between a fused and an unfused (or
    reversed) multiply-add chain (worked by hand in
    tests/golden/mlp_subnormal_chain.txt): the GPU must pick predictor 1 in
    every block, as the oracle does."""
    import os
    w = np.zeros(oracle.NW, np.uint16)
    with open(os.path.join(os.path.dirname(__file__), "golden", "mlp_subnormal_chain.txt")) as f:
        for line in f:
            p = line.split()
            if p and p[0] == "weight":
                w[int(p[1])] = int(p[2], 16)
    # a smooth field, so that predictor 1 everywhere stays far from the raw
    # fallback and the stream carries its per-block ids
    x = synth.blobs3d((40, 37, 70), seed=3).numpy()
    ref = oracle.compress(x, 1e-3, predictor="mlp", weights=w)
    buf = fz.compress(torch.from_numpy(x).cuda(), 1e-3, predictor="mlp",
                      selector_weights=torch.from_numpy(w.view(np.int16)).cuda())
    got = buf.cpu().numpy()
    assert got.size == ref.size and np.array_equal(got, ref)
    assert int(np.frombuffer(got[6:8].tobytes(), np.uint16)[0]) == 4  # ids present
    off_ids = int(np.frombuffer(got[144:152].tobytes(), np.uint64)[0])
    nb = 5 * 5 * 9
    ids = np.unpackbits(got[off_ids:off_ids + (nb + 3) // 4][:, None], axis=1, bitorder="little")
    ids = (ids.reshape(-1, 4, 2) * np.array([1, 2])).sum(-1).ravel()[:nb]
    assert (ids == 1).all()


def test_mlp_gradient_matches_oracle():
    rng = np.random.default_rng(2)
    wb = _rand_weights(3)
    n = 1000
    f32 = rng.uniform(0, 25, (n, oracle.NFEAT)).astype(np.float32)
    feat = torch.from_numpy(f32).to(torch.bfloat16).view(torch.int16)
    lab = torch.from_numpy(rng.integers(0, 4, n).astype(np.uint8))
    loss_ref, g_ref = oracle.mlp_loss_grad(wb, feat.numpy().view(np.uint16), lab.numpy())
    w_master = torch.from_numpy(wb.view(np.int16)).view(torch.bfloat16).float().cuda().contiguous()
    g, loss = fz.mlp_grad(w_master, feat.cuda().contiguous(), lab.cuda().contiguous())
    g = g.cpu().double().numpy()
    assert abs(loss - loss_ref) <= 1e-4 * abs(loss_ref)
    o1 = oracle.NHID * oracle.NFEAT
    parts = [(0, o1), (o1, o1 + 64), (o1 + 64, o1 + 64 + 256), (o1 + 320, oracle.NW)]
    for a, b in parts:
        d = np.linalg.norm(g[a:b] - g_ref[a:b]) / max(np.linalg.norm(g_ref[a:b]), 1e-30)
        cos = float(g[a:b] @ g_ref[a:b] / (np.linalg.norm(g[a:b]) * np.linalg.norm(g_ref[a:b]) + 1e-300))
        assert d <= 1e-3 and cos > 0.9999, (a, b, d, cos)
    # deterministic: the same call gives the same bits
    fc, lc = feat.cuda().contiguous(), lab.cuda().contiguous()
    g2 = fz.mlp_grad(w_master, fc, lc)[0].cpu().numpy()
    g3 = fz.mlp_grad(w_master, fc, lc)[0].cpu().numpy()
    assert np.array_equal(g2.view(np.uint32), g3.view(np.uint32))


def test_adam_step_matches_oracle():
    """fz_mlp_adam (float32 on the GPU) against the oracle's float64 Adam
    step (Kingma and Ba 2015, Algorithm 1) over five steps with random
    gradients.  Tolerance: each float32 operation errs by at most 2^-24
    relative; the moments take three operations per step and stay below the
    largest |g| (and g^2), and the step mhat / (sqrt(vhat) + eps) has about
    ten operations, so |dm| <= 1e-6 max|g|, |dv| <= 1e-6 max g^2 and
    |dw| <= 2^-22 |w| + 1e-5 lr per step.  The bfloat16 copy is the
    round-to-nearest-even of the float32 master, bit for bit."""
    rng = np.random.default_rng(21)
    n = oracle.NW
    w0 = (rng.standard_normal(n) * 0.3).astype(np.float32)
    wd = torch.from_numpy(w0).cuda()
    md = torch.zeros(n, device="cuda")
    vd = torch.zeros(n, device="cuda")
    wb = torch.empty(n, dtype=torch.int16, device="cuda")
    w, m, v = w0.astype(np.float64), np.zeros(n), np.zeros(n)
    lr, b1, b2, eps = 3e-3, 0.9, 0.999, 1e-8
    gmax = 0.0
    for t in range(1, 6):
        g = (rng.standard_normal(n) * np.exp(rng.uniform(-6, 1, n))).astype(np.float32)
        gmax = max(gmax, float(np.abs(g).max()))
        fz.mlp_adam(wd, torch.from_numpy(g).cuda(), md, vd, t, lr, b1, b2, eps, w_bf16=wb)
        # the oracle gets exactly the float32 hyper-parameters the kernel sees
        w, m, v = oracle.adam_step(w, g.astype(np.float64), m, v, t, float(np.float32(lr)),
                                   float(np.float32(b1)), float(np.float32(b2)), float(np.float32(eps)))
        torch.cuda.synchronize()
        wg, mg, vg = wd.cpu().double().numpy(), md.cpu().double().numpy(), vd.cpu().double().numpy()
        assert np.abs(mg - m).max() <= 1e-6 * gmax, t
        assert np.abs(vg - v).max() <= 1e-6 * gmax * gmax, t
        assert (np.abs(wg - w) <= 2.0 ** -22 * np.abs(w) + 1e-5 * lr * t).all(), t
        want = torch.from_numpy(wd.cpu().numpy()).to(torch.bfloat16).view(torch.int16)
        assert torch.equal(wb.cpu(), want)


def _cr(x, pred, w=None):
    buf = fz.compress(x, 1e-4, predictor=pred, selector_weights=w)
    y = fz.decompress(buf)
    eba = 1e-4 * (float(x.max()) - float(x.min()))
    assert float((y.double() - x.double()).abs().max()) <= eba
    return x.numel() * 4 / buf.numel()


def test_trained_selector_beats_plain_and_tracks_exhaustive():
    """Trained on the GPU with the library's own kernels on exhaustive-trial
    labels of 16 seeded stitched fields; evaluated on an unseen field."""
    torch.manual_seed(0)
    fields = [synth.stitched3d(256, seed=100 + i, region=64, device="cuda") for i in range(16)]
    feat, lab = sel.collect(fields, 1e-4)
    del fields
    w, wb, hist = sel.train(feat, lab, epochs=12, batch=4096, lr=3e-3, seed=0)
    assert hist[-1] < hist[0]
    x = synth.stitched3d(512, seed=200, region=64, device="cuda")
    cr_plain = _cr(x, "lorenzo1")
    cr_exh = _cr(x, "exhaustive")
    cr_mlp = _cr(x, "mlp", wb)
    print(f"CR plain {cr_plain:.4f} exhaustive {cr_exh:.4f} mlp {cr_mlp:.4f}")
    assert cr_mlp > cr_plain
    assert cr_mlp >= 0.98 * cr_exh
    # the full 512^3 streams of both selections, with the trained weights,
    # byte for byte against the oracle, and their reconstructions bit for bit
    xh = x.cpu().numpy()
    wh = wb.cpu().numpy().view(np.uint16)
    for pred, w in (("exhaustive", None), ("mlp", wh)):
        wd = torch.from_numpy(w.view(np.int16)).cuda() if w is not None else None
        buf = fz.compress(x, 1e-4, predictor=pred, selector_weights=wd)
        y = fz.decompress(buf).cpu().numpy()
        got = buf.cpu().numpy()
        del buf
        ref = oracle.compress(xh, 1e-4, predictor=pred, weights=w)
        assert got.size == ref.size and np.array_equal(got, ref), pred
        assert np.array_equal(_bits(y), _bits(oracle.decompress(ref))), pred
