"""Evaluation report of FZModules §4.2 on this library: overall speedup
(Eq. 1) and rate-distortion (bit rate against PSNR).

Eq. 1 combines the compression ratio CR, the compression throughput T and
the bandwidth BW of the medium the data crosses:

    speedup = 1 / (((BW * CR)^-1 + T^-1) * BW)

so that compressing pays off (speedup > 1) only when the time to compress
plus the time to move the smaller stream beats moving the raw data.  The
rate-distortion sweep reports, per workload and error bound, the bit rate
(stream bits per input value), the PSNR of the reconstruction (from
fz_error_stats, a kernel of the library), the compression ratio and both
throughputs.  Compression, decompression and the statistics all run in the
library's kernels; torch only holds the buffers and the CUDA events.
"""
from __future__ import annotations

import statistics

import torch

from . import compress, compress_bound, decompress, error_stats


def overall_speedup(bw_gbs: float, cr: float, compress_gbs: float) -> float:
    """Eq. 1: the end-to-end speedup of compressing at compress_gbs (GB/s of
    input) to ratio cr before a transfer at bw_gbs, against sending the raw
    data."""
    return 1.0 / ((1.0 / (bw_gbs * cr) + 1.0 / compress_gbs) * bw_gbs)


def bit_rate(n_values: int, stream_bytes: int) -> float:
    """Average stream bits per input value (32 / CR for float32 input)."""
    return 8.0 * stream_bytes / n_values


def rate_distortion(fields, ebs, bws_gbs, reps: int = 3, mode: str = "rel", flush_bytes: int = 256 << 20):
    """One row per (field, bound): bit rate, PSNR, max error over the bound,
    CR, compression and decompression GB/s (CUDA events on the current
    stream, L2 flushed before each timed call) and Eq. 1's speedup at each
    bandwidth in bws_gbs.  `fields` maps a name to a contiguous float32 CUDA
    tensor."""
    rows = []
    for name, x in fields.items():
        dev = x.device
        stream = torch.cuda.current_stream(dev)
        scratch = torch.empty(flush_bytes // 4, dtype=torch.float32, device=dev)
        ob = torch.empty(compress_bound(x.shape), dtype=torch.uint8, device=dev)
        y = torch.empty_like(x)
        fin = x[torch.isfinite(x)]
        rng = float(fin.max()) - float(fin.min())
        n = x.numel()
        for eb in ebs:
            buf = compress(x, eb, mode, out=ob)
            decompress(buf, out=y)
            st = error_stats(x, y)
            tc, td = [], []
            for _ in range(reps):
                scratch.fill_(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                buf = compress(x, eb, mode, out=ob)
                e1.record(stream)
                scratch.fill_(1)
                e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e2.record(stream)
                decompress(buf, out=y)
                e3.record(stream)
                torch.cuda.synchronize(dev)
                tc.append(e0.elapsed_time(e1))
                td.append(e2.elapsed_time(e3))
            S = buf.numel()
            cr = 4.0 * n / S
            cgbs = 4.0 * n / (statistics.median(tc) * 1e-3) / 1e9
            dgbs = 4.0 * n / (statistics.median(td) * 1e-3) / 1e9
            eb_abs = eb * rng if mode == "rel" else eb
            rows.append({"field": name, "eb_mode": mode, "eb": eb, "stream_bytes": S, "cr": round(cr, 4),
                         "bit_rate": round(bit_rate(n, S), 4), "psnr_db": round(st["psnr_db"], 3),
                         "max_err_over_eb": round(st["max_abs_err"] / eb_abs, 6),
                         "compress_gbs": round(cgbs, 2), "decompress_gbs": round(dgbs, 2),
                         "speedup_eq1": {f"{bw:g}GB/s": round(overall_speedup(bw, cr, cgbs), 4) for bw in bws_gbs}})
        del scratch, ob, y
    return rows
