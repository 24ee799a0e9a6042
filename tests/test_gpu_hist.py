"""GPU: the histogram module (§3.2) as a stage -- the warp-private method and
the top-k method give exactly numpy's bincount on every kind of code
distribution, and the quantizer's fused histogram on real codes."""
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


def _codes(kind, n, nsym, seed):
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        c = rng.integers(0, nsym, n)
    elif kind == "lorenzo":    # two-sided geometric around the centre
        c = nsym // 2 + np.round(rng.laplace(0, 6, n)).astype(np.int64)
    elif kind == "peaked":     # one code nearly always (a good predictor)
        c = np.where(rng.random(n) < 0.99, nsym // 2, rng.integers(0, nsym, n))
    elif kind == "constant":
        c = np.full(n, 3)
    else:                      # exactly 16 distinct codes, then 17
        c = rng.integers(0, 17, n) * (nsym // 17)
    return np.clip(c, 0, nsym - 1).astype(np.uint16)


@pytest.mark.parametrize("method", ["private", "topk"])
@pytest.mark.parametrize("kind", ["uniform", "lorenzo", "peaked", "constant", "seventeen"])
@pytest.mark.parametrize("n,nsym", [(1, 1024), (7, 1024), (1000, 4), (123457, 1024), (3 << 20, 1024), (200003, 128)])
def test_histogram_exact(method, kind, n, nsym):
    c = _codes(kind, n, nsym, seed=n + nsym)
    h = fz.histogram(torch.from_numpy(c.view(np.int16)).cuda(), nsym, method).cpu().numpy()
    assert np.array_equal(h, np.bincount(c, minlength=nsym)[:nsym])


def test_histogram_matches_quantizer_on_real_codes():
    """Lorenzo codes of a 3D field and interpolation codes of a smooth one:
    both methods equal the quantizer's own histogram (which the GPU parity
    tests tie to the oracle) and the oracle's stage histogram."""
    x = synth.blobs3d((64, 72, 80), seed=4)
    for pred in ("lorenzo1", "interp_cubic"):
        codes, _, hist, _, _, _ = fz.lorenzo_quantize(x.cuda(), 1e-4, predictor=pred)
        for method in ("private", "topk"):
            h = fz.histogram(codes, 1024, method)
            assert torch.equal(h, hist), (pred, method)
    xh = x.numpy()
    e2, inv, chk = oracle.constants(1e-4 * (float(xh.max()) - float(xh.min())))
    _, _, oh, _, _ = oracle.quantize_stage(xh, 3, xh.shape[::-1], inv, e2, chk)
    codes, _, _, _, _, _ = fz.lorenzo_quantize(x.cuda(), 1e-4)
    assert np.array_equal(fz.histogram(codes, 1024, "topk").cpu().numpy().astype(np.uint64), oh)


def test_histogram_rejects_codes_outside_the_alphabet():
    c = np.array([1, 2, 300, 4, 5, 6, 7, 8], np.uint16)
    for method in ("private", "topk"):
        with pytest.raises(fz.FzError) as e:
            fz.histogram(torch.from_numpy(c.view(np.int16)).cuda(), 256, method)
        assert e.value.code == 1
