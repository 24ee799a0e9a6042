"""Eq. 1 (overall speedup) and the rate-distortion quantities of §4.2:
pinned by the paper's own worked example and by closed forms."""
import math

import pytest

from paper_2509_20563_gb300 import report


def test_overall_speedup_worked_example():
    """§4.2: over a 100 GB/s link a compressor with CR 2 needs more than
    200 GB/s of throughput to give any speedup -- at exactly 200 GB/s the
    speedup is 1."""
    assert report.overall_speedup(100.0, 2.0, 200.0) == pytest.approx(1.0, rel=1e-15)
    assert report.overall_speedup(100.0, 2.0, 199.0) < 1.0 < report.overall_speedup(100.0, 2.0, 201.0)


def test_overall_speedup_limits():
    """An infinitely fast compressor gains exactly its ratio; one that does
    not compress (CR 1) can only lose; the speedup is the ratio of the raw
    transfer time to compression plus the compressed transfer."""
    assert report.overall_speedup(25.0, 7.5, 1e30) == pytest.approx(7.5, rel=1e-12)
    assert report.overall_speedup(25.0, 1.0, 1000.0) < 1.0
    bw, cr, t = 88.0, 3.5, 900.0
    raw = 1.0 / bw
    assert report.overall_speedup(bw, cr, t) == pytest.approx(raw / (1.0 / t + 1.0 / (bw * cr)), rel=1e-14)


def test_bit_rate_is_32_over_cr():
    for n, s in ((1000, 250), (134217728, 152149360), (7, 272)):
        assert report.bit_rate(n, s) == pytest.approx(32.0 / (4.0 * n / s), rel=1e-15)


def test_psnr_lower_bound_from_the_error_bound():
    """A reconstruction within eb_abs = eb_rel * range of every value has
    MSE <= eb_abs^2, so PSNR >= -20 log10(eb_rel): the bound the GPU sweep is
    checked against."""
    for eb in (1e-2, 1e-4, 1e-6):
        rng = 3.7
        mse_max = (eb * rng) ** 2
        assert 20 * math.log10(rng) - 10 * math.log10(mse_max) == pytest.approx(-20 * math.log10(eb), rel=1e-12)
