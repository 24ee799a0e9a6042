"""GPU: the reconstruction statistics kernel against float64 numpy, and the
rate-distortion sweep of §4.2 against the oracle and the error bound."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

fz = None
report = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global fz, report
    from paper_2509_20563_gb300 import build
    build.build()
    import paper_2509_20563_gb300 as m
    import paper_2509_20563_gb300.report as r
    m.lib()
    fz, report = m, r


@pytest.mark.parametrize("n", [1, 5, 1023, 4096 * 150 + 7, 3 << 20])
def test_error_stats_match_float64(n):
    rng = np.random.default_rng(n)
    x = (rng.standard_normal(n) * 10).astype(np.float32)
    y = (x + rng.uniform(-1e-3, 1e-3, n)).astype(np.float32)
    if n > 10:
        x[3], y[3] = np.nan, np.nan                                     # same bits: not a mismatch
        x[5] = np.inf
        y[5] = 0.0                                                      # a mismatch
    st = fz.error_stats(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    f = np.isfinite(x)
    d = y[f].astype(np.float64) - x[f].astype(np.float64)
    assert st["n_finite"] == int(f.sum())
    assert st["n_nonfinite_mismatch"] == (1 if n > 10 else 0)
    assert st["max_abs_err"] == float(np.abs(d).max())
    assert st["sse"] == pytest.approx(float((d * d).sum()), rel=1e-12)
    assert st["x_min"] == float(x[f].min()) and st["x_max"] == float(x[f].max())
    mse = float((d * d).sum()) / f.sum()
    rng_x = float(x[f].max()) - float(x[f].min())
    if mse > 0 and rng_x > 0:
        want = 20 * math.log10(rng_x) - 10 * math.log10(mse)
        assert st["psnr_db"] == pytest.approx(want, rel=1e-10)
    else:
        assert math.isinf(st["psnr_db"])
    # deterministic: the same call gives the same bits
    st2 = fz.error_stats(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    assert st2 == st


def test_rate_distortion_sweep_against_oracle_and_bound():
    """A small field at REL 1e-2 .. 1e-6: the bit rate equals the oracle
    stream's (the streams are identical), the PSNR equals the one computed in
    float64 from the oracle's reconstruction, it is at least -20 log10(eb)
    (the bound), and both rise as the bound tightens."""
    x = synth.blobs3d((48, 40, 56), seed=9)
    xd = x.contiguous().cuda()
    ebs = [1e-2, 1e-3, 1e-4, 1e-5, 1e-6]
    rows = report.rate_distortion({"blobs": xd}, ebs, [25.0, 100.0], reps=2)
    xh = x.numpy()
    rng = float(xh.max()) - float(xh.min())
    prev = None
    for row, eb in zip(rows, ebs):
        ref = oracle.compress(xh, eb)
        assert row["stream_bytes"] == ref.size
        assert row["bit_rate"] == pytest.approx(8.0 * ref.size / xh.size, abs=1e-4)
        yr = oracle.decompress(ref).astype(np.float64)
        mse = float(((yr - xh.astype(np.float64)) ** 2).mean())
        if mse == 0:  # a raw stream at the tightest bound: exact
            assert math.isinf(row["psnr_db"])
            continue
        psnr = 20 * math.log10(rng) - 10 * math.log10(mse)
        assert row["psnr_db"] == pytest.approx(psnr, abs=2e-3)
        assert row["psnr_db"] >= -20 * math.log10(eb)
        assert row["max_err_over_eb"] <= 1.0
        if prev:
            assert row["bit_rate"] > prev["bit_rate"] and row["psnr_db"] > prev["psnr_db"]
        prev = row
        assert set(row["speedup_eq1"]) == {"25GB/s", "100GB/s"}
