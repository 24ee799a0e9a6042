#!/usr/bin/env python
"""Benchmark of the compression hot path on GB300.

One step = fz_compress + fz_decompress of a 512^3 float32 Gaussian random
field (Kolmogorov spectrum, seed 2 + rank) at a value-range-relative bound of
1e-4 with first-order Lorenzo and code radius 512 -- the paper's Nyx-shaped
workload (Table 2) with synthetic data.  The field (512 MiB) is larger than
L2, so no flush is needed between timed steps.

Printed (rank 0, one JSON line): round-trip throughput on the input basis
(input bytes / (compress + decompress device time)), per-direction GB/s and
fractions of the HBM roofline, compression ratio, the dominant kernel's
roofline entry (CUDA-event stage timing inside the library), an end-to-end
number through the C ABI with host buffers and copies (with the host link's
measured copy bandwidth beside it), the CPU oracle timed on a bounded slab of
the same field (one thread, and one process per host core), the SM clocks
sampled during the timed region, and -- in the same run -- every other
plain-pipeline workload (the per-mode spectrum reading of the 512^3 field,
the 1D particle and 2D lat/lon fields at three bounds), the 64-field batch
and the learned selector.

``--impl reference`` times the CPU oracle instead (rank 0 only), each step a
bounded slab of the same workload.

Multi-GPU (torchrun): every rank compresses its own field (weak scaling, no
collective on the data path); the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "3D FP32 512^3 Gaussian random field (k^-5/3), REL 1e-4, Lorenzo-1, radius 512"

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of each
# large kernel on exactly this workload (512^3, REL 1e-4), from one ncu
# capture, with the SHA-256 of the kernel's source files at the time of the
# capture and the commit it was taken at.  Reported as roofline.traffic for
# the dominant kernel only while its sources still hash the same (else
# null): a changed kernel needs a new capture.
KERNEL_SOURCES = {
    "range": ["fz_range.cu", "fz_internal.cuh"],
    "quant": ["fz_quant.cu", "fz_internal.cuh"],
    "encode": ["fz_encode.cu", "fz_internal.cuh"],
    "decode": ["fz_decode.cu", "fz_decode_common.cuh", "fz_internal.cuh"],
}
# kernel -> (dram__bytes_read.sum + dram__bytes_write.sum of one launch at 512^3, digest of the kernel's
# sources when captured, commit): one-pass ncu capture of the bench's own first decoder launch
NCU_DRAM_BYTES_512 = {"decode": (250551808 + 478513408, "eef5ad757df9bcfb", "dc0e2dd")}
METRIC = "compress/decompress GB/s vs HBM peak at REL 1e-4; CR learned vs plain"
PROFILE_EVERY = 8  # timed steps per step that records the library's stage events
E2E_WORKERS = 4  # host threads (each with its own context and stream) of the end-to-end leg


def source_digest(kernel: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2509_20563_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """(bytes, commit) of the ncu capture of this kernel if its sources are
    unchanged since, else (None, reason)."""
    rec = NCU_DRAM_BYTES_512.get(kernel)
    if not rec:
        return None, "no capture"
    b, dig, commit = rec
    if dig != source_digest(kernel):
        return None, f"kernel changed since the capture at {commit}"
    return b, commit


def _bind_near_gpu(dev_index: int):
    """Moves this thread to the CPUs of the NUMA node the GPU is attached to
    (from the PCI device's sysfs entry), so that pinned host memory allocated
    next is local to the GPU's host link.  Returns (node or None, previous
    CPU set or None); does nothing where the node or its CPUs are unknown."""
    try:
        pr = torch.cuda.get_device_properties(dev_index)
        addr = f"{pr.pci_domain_id:04x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
        with open(f"/sys/bus/pci/devices/{addr}/numa_node") as f:
            node = int(f.read().strip())
        if node < 0:
            return None, None
        cpus = set()
        with open(f"/sys/devices/system/node/node{node}/cpulist") as f:
            for part in f.read().strip().split(","):
                lo, _, hi = part.partition("-")
                cpus.update(range(int(lo), int(hi or lo) + 1))
        prev = os.sched_getaffinity(0)
        use = cpus & prev
        if not use:
            return None, None
        os.sched_setaffinity(0, use)
        return node, prev
    except Exception:  # an optional placement: never a reason to fail the bench
        return None, None


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time (replicas: every rank times its own work)."""
    if world <= 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def aggregate_gbs(steps: int, world: int, bytes_per_step_per_rank: int, max_ms: float) -> float:
    """Whole-job throughput: the bytes all ranks processed over the slowest rank's time."""
    return steps * world * bytes_per_step_per_rank / (max_ms * 1e-3) / 1e9


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.uuid = None
        try:
            self.uuid = str(torch.cuda.get_device_properties(device).uuid)
        except Exception:
            pass
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"fz_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and self.uuid not in parts[0] and parts[0] not in self.uuid:
                continue
            rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def _oracle_slab_worker(args):
    """One process of the all-core CPU baseline: the oracle, single-threaded
    as written, on its own slab; starts with the others at a barrier."""
    x, eb, barrier = args
    import oracle
    oracle.lib()
    barrier.wait()
    t0 = time.time()
    oracle.decompress(oracle.compress(x, eb))
    return t0, time.time()


def cpu_baseline(field_gpu: torch.Tensor, slab_z: int, eb: float):
    """The CPU oracle, as it stands, on a z-slab of the same field: (a) in
    this process on one thread, (b) as one process per host core on
    disjoint slabs of the field (plain oracle in each; no threading added)."""
    import multiprocessing as mp
    import oracle
    x = field_gpu[:slab_z].contiguous().cpu().numpy()
    t0 = time.perf_counter()
    buf = oracle.compress(x, eb)
    t1 = time.perf_counter()
    oracle.decompress(buf)
    t2 = time.perf_counter()
    gbs = x.nbytes / (t2 - t0) / 1e9
    res = {"value": round(gbs, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
           "sample": f"{x.shape[2]}x{x.shape[1]}x{x.shape[0]} slab of the field ({x.nbytes >> 20} MiB), "
                     f"compress {t1 - t0:.2f} s + decompress {t2 - t1:.2f} s, single thread",
           "compress_gbs": round(x.nbytes / (t1 - t0) / 1e9, 4),
           "decompress_gbs": round(x.nbytes / (t2 - t1) / 1e9, 4), "cpu_model": cpu_model()}
    try:
        cores = len(os.sched_getaffinity(0))
        nz = field_gpu.shape[0]
        per = max(8, min(slab_z, nz // cores))
        slabs = [field_gpu[z:z + per].contiguous().cpu().numpy() for z in range(0, min(nz, per * cores), per)]
        ctxm = mp.get_context("spawn")  # never fork a process that holds a CUDA context
        with ctxm.Manager() as mgr:
            barrier = mgr.Barrier(len(slabs))
            with ctxm.Pool(len(slabs)) as pool:
                spans = pool.map(_oracle_slab_worker, [(s, eb, barrier) for s in slabs])
        wall = max(b for _, b in spans) - min(a for a, _ in spans)
        nbytes = sum(s.nbytes for s in slabs)
        res["all_cores"] = {"value": round(nbytes / wall / 1e9, 4), "unit": "GB/s", "cores": len(slabs),
                            "kind": "oracle", "sample": f"{len(slabs)} processes, each a {per}-plane slab "
                                                        f"({slabs[0].nbytes >> 20} MiB) compressed and "
                                                        f"decompressed, {wall:.2f} s wall"}
    except Exception as e:  # the extra leg never fails the bench
        res["all_cores"] = {"error": str(e)[:200]}
    return res


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.build()
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    field = synth.grf3d(args.size, seed=2, device=dev)
    slab = max(1, args.ref_slab)
    x = field[:slab].contiguous().cpu().numpy()
    for _ in range(args.warmup):
        oracle.decompress(oracle.compress(x, args.eb))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.decompress(oracle.compress(x, args.eb))
    dt = time.perf_counter() - t0
    v = args.steps * x.nbytes / dt / 1e9
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample": f"{args.size}x{args.size}x{slab} slab per step"},
           "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                            "sample": f"{args.size}x{args.size}x{slab} slab ({x.nbytes >> 20} MiB) per step"},
           "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_fz(args, rank, world, local_rank):
    import paper_2509_20563_gb300 as fz
    from paper_2509_20563_gb300 import build as fzbuild
    fzbuild.build()
    L = fz.lib()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    N = args.size ** 3
    x = synth.grf3d(args.size, seed=2 + rank, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = C.c_void_p(stream.cuda_stream)
    ctx = fz.Context(local_rank)
    bound = fz.compress_bound(x.shape)
    buf = torch.empty(bound, dtype=torch.uint8, device=dev)
    y = torch.empty_like(x)
    dims = fz._dims(x.shape)
    pipe = fz._pipeline("lorenzo1", 512)
    nbytes = C.c_uint64()
    hdr = C.create_string_buffer(256)

    # the call arguments are built once, as a caller in a loop would
    fz_compress, fz_decompress = L.fz_compress, L.fz_decompress
    xp, bufp, yp = C.c_void_p(x.data_ptr()), C.c_void_p(buf.data_ptr()), C.c_void_p(y.data_ptr())
    c_args = (ctx.handle, xp, 3, dims, 1, args.eb, C.byref(pipe), bufp, bound, C.byref(nbytes), hdr, sp)

    def compress():
        st = fz_compress(*c_args)
        if st:
            raise fz.FzError(st, "fz_compress")

    def decompress():
        st = fz_decompress(ctx.handle, bufp, nbytes.value, hdr, yp, N, sp)
        if st:
            raise fz.FzError(st, "fz_decompress")

    # correctness of this very configuration before timing
    compress()
    decompress()
    rng = float(x.max()) - float(x.min())
    eb_abs = args.eb * rng
    max_err = float((y.double() - x.double()).abs().max())
    assert max_err <= eb_abs, (max_err, eb_abs)
    S = nbytes.value
    fh = fz.stream_info(hdr.raw)
    for _ in range(args.warmup):
        compress()
        decompress()
    prof = fz.Profile()
    stages_c, stages_d = {}, {}
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    launches0 = _launches(L, ctx)
    # every PROFILE_EVERY-th timed step records the library's stage events (a
    # CUDA event between every two kernels on the launching stream): the
    # stage times and the dominant kernel's duration come from those steps,
    # inside the timed region; the other steps run without the events
    for i in range(args.steps):
        prof_step = i % PROFILE_EVERY == 0
        assert L.fz_ctx_set_profiling(ctx.handle, 1 if prof_step else 0) == 0
        ev[i][0].record(stream)
        compress()
        ev[i][1].record(stream)
        decompress()
        ev[i][2].record(stream)
        if prof_step:
            assert L.fz_ctx_get_profile(ctx.handle, C.byref(prof)) == 0
            for k in range(prof.n_compress):
                stages_c.setdefault(prof.compress_names[k].value.decode(), []).append(prof.compress_ms[k])
            for k in range(prof.n_decompress):
                stages_d.setdefault(prof.decompress_names[k].value.decode(), []).append(prof.decompress_ms[k])
    assert L.fz_ctx_set_profiling(ctx.handle, 0) == 0
    torch.cuda.synchronize(dev)
    launches = _launches(L, ctx) - launches0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    tc = [a.elapsed_time(b) for a, b, _ in ev]
    td = [b.elapsed_time(c) for _, b, c in ev]
    tot_ms = sum(tc) + sum(td)
    tot_ms = max_over_ranks(tot_ms, world, dev)
    peak, peak_kind = _peaks()
    mc, md = statistics.mean(tc), statistics.mean(td)
    comp_gbs = 4 * N / (mc * 1e-3) / 1e9
    dec_gbs = 4 * N / (md * 1e-3) / 1e9
    comp_forced = 12 * N + S       # range read + quant read + codes write + codes read + stream
    dec_forced = S + 4 * N
    # per-kernel algorithmic bytes per launch
    n_blocks = N // 512
    hd = np.frombuffer(hdr.raw, dtype=np.uint8)
    n_out = int(np.frombuffer(hdr.raw[112:120], np.uint64)[0])
    n_exc = int(np.frombuffer(hdr.raw[120:128], np.uint64)[0])
    total_bits = int(np.frombuffer(hdr.raw[128:136], np.uint64)[0])
    alg = {"range": 4 * N, "quant": 4 * N + 2 * N + 4 * n_blocks + 8 * (n_out + n_exc),
           "encode": 2 * N + total_bits // 8 + 4 * n_blocks,
           "decode": S + 4 * N}
    kern = {k: statistics.mean(v) for k, v in {**stages_c, **stages_d}.items() if k in alg}
    dom = max(kern, key=kern.get)
    ach = alg[dom] / (kern[dom] * 1e-3) / 1e9
    value = aggregate_gbs(args.steps, world, 4 * N, tot_ms)
    if args.traffic is not None:
        traffic, traffic_note = args.traffic, "--traffic"
    elif args.size == 512 and args.eb == 1e-4:
        traffic, traffic_note = ncu_traffic(dom)
    else:
        traffic, traffic_note = None, "no capture of this workload"
    res = {"metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(tot_ms / args.steps, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "dims": [args.size] * 3, "eb_mode": "rel", "eb": args.eb,
                      "predictor": "lorenzo1", "radius": 512, "l2": "input 512 MiB > L2, no flush",
                      "parallelism": f"replicas x{world}"},
           "compress_gbs": round(comp_gbs, 2), "decompress_gbs": round(dec_gbs, 2),
           "compress_roofline_frac": round(comp_forced / (mc * 1e-3) / 1e9 / peak, 4),
           "decompress_roofline_frac": round(dec_forced / (md * 1e-3) / 1e9 / peak, 4),
           "roofline_basis": "forced HBM bytes: compress 12N+S, decompress S+4N; peak = MEASURED_PEAKS hbm_gbs "
                             f"({peak_kind})",
           "cr": round(4 * N / S, 4), "stream_bytes": S, "n_outliers": n_out, "n_exceptions": n_exc,
           "max_err_over_eb": round(max_err / eb_abs, 6),
           "stages_ms": {**{f"c.{k}": round(statistics.mean(v), 4) for k, v in stages_c.items()},
                         **{f"d.{k}": round(statistics.mean(v), 4) for k, v in stages_d.items()}},
           "roofline": {"kernel": dom, "bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(ach / peak, 4), "traffic": traffic, "traffic_source": traffic_note,
                        "algorithmic_bytes": alg[dom], "peak_kind": peak_kind,
                        "duration_source": f"the library's stage events (CUDA events on the launching stream) "
                                           f"on 1 of every {PROFILE_EVERY} timed steps",
                        "source_digest": source_digest(dom)},
           "gpu_launches": int(launches), "clocks": clk}
    # end to end through the C ABI with host buffers: H2D input, compress, D2H stream,
    # H2D stream, decompress, D2H reconstruction -- copies inside the timed region.
    # Each library call waits for its own stream, so the steps run on
    # E2E_WORKERS host threads, each with its own context (workspace), stream
    # and buffers, the way a caller with several workers would: one worker's
    # copies overlap the others' kernels and copies.
    if args.e2e_steps > 0:
        # pinned host buffers on the GPU's own NUMA node (the thread runs there
        # while they are allocated and copied): a far node halves the link
        numa, saved_cpus = _bind_near_gpu(local_rank)
        hx = torch.empty(x.shape, dtype=torch.float32, pin_memory=True)
        hx.copy_(x)
        slots = []
        for k in range(E2E_WORKERS):
            sl = {"s": torch.cuda.Stream(dev), "xd": torch.empty_like(x), "buf": torch.empty_like(buf),
                  "bd": torch.empty_like(buf), "y": torch.empty_like(x),
                  "hs": torch.empty(bound, dtype=torch.uint8, pin_memory=True),
                  "hy": torch.empty(x.shape, dtype=torch.float32, pin_memory=True),
                  "ctx": ctx if k == 0 else fz.Context(local_rank), "nbytes": C.c_uint64(),
                  "hdr": C.create_string_buffer(256)}
            sl["sp"] = C.c_void_p(sl["s"].cuda_stream)
            slots.append(sl)

        def e2e_step(sl):
            with torch.cuda.stream(sl["s"]):
                sl["xd"].copy_(hx, non_blocking=True)
            st = fz_compress(sl["ctx"].handle, C.c_void_p(sl["xd"].data_ptr()), 3, dims, 1, args.eb, C.byref(pipe),
                             C.c_void_p(sl["buf"].data_ptr()), bound, C.byref(sl["nbytes"]), sl["hdr"], sl["sp"])
            assert st == 0
            nb = sl["nbytes"].value
            with torch.cuda.stream(sl["s"]):
                sl["hs"][:nb].copy_(sl["buf"][:nb], non_blocking=True)
                sl["bd"][:nb].copy_(sl["hs"][:nb], non_blocking=True)
            st = fz_decompress(sl["ctx"].handle, C.c_void_p(sl["bd"].data_ptr()), nb, sl["hdr"],
                               C.c_void_p(sl["y"].data_ptr()), N, sl["sp"])
            assert st == 0
            with torch.cuda.stream(sl["s"]):
                sl["hy"].copy_(sl["y"], non_blocking=True)
            return nb

        def worker(sl, n_steps, errs):
            try:
                torch.cuda.set_device(dev)
                for _ in range(n_steps):
                    e2e_step(sl)
            except BaseException as exc:  # reported by the main thread
                errs.append(exc)

        for sl in slots:  # warm-up, one worker after the other (first launches set up the library)
            e2e_step(sl)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            torch.distributed.barrier()
        e0.record(stream)
        for sl in slots:
            sl["s"].wait_stream(stream)
        errs = []
        share = [args.e2e_steps // E2E_WORKERS + (1 if k < args.e2e_steps % E2E_WORKERS else 0)
                 for k in range(E2E_WORKERS)]
        threads = [threading.Thread(target=worker, args=(sl, n, errs)) for sl, n in zip(slots, share)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        if errs:
            raise errs[0]
        for sl in slots:
            stream.wait_stream(sl["s"])
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ems = e0.elapsed_time(e1)
        ems = max_over_ranks(ems, world, dev)
        nb = slots[0]["nbytes"].value
        ok = all(torch.equal(sl["y"], y) for sl in slots)  # every step reconstructs the same field
        assert ok
        res["e2e"] = {"value": round(aggregate_gbs(args.e2e_steps, world, 4 * N, ems), 2), "unit": "GB/s",
                      "h2d_bytes_per_step": 4 * N + nb, "d2h_bytes_per_step": nb + 4 * N,
                      "steps": args.e2e_steps, "streams": E2E_WORKERS, "host_threads": E2E_WORKERS,
                      "contexts": E2E_WORKERS, "host_numa_node": numa}
        link = host_link(dev, hx, x)
        # roofline of the end-to-end step: its host-link bytes at the measured
        # link rate (both directions at once), against the measured step time
        t_link = (4 * N + nb + nb + 4 * N) / (link["bidirectional_gbs"] * 1e9)
        res["e2e"]["host_link"] = link
        res["e2e"]["link_frac"] = round(t_link / (ems / args.e2e_steps * 1e-3), 4)
        for sl in slots[1:]:
            sl["ctx"].close()
        if saved_cpus is not None:
            os.sched_setaffinity(0, saved_cpus)
    if rank == 0 and world == 1 and not args.no_configs:
        res["configs"] = bench_configs(fz, dev, stream, args)
    if rank == 0 and world == 1 and not args.no_speed:
        res["speed_pipeline"] = bench_speed(fz, dev, stream, x, args)
    if rank == 0 and world == 1 and not args.no_quality:
        res["quality_pipeline"] = bench_quality(fz, dev, stream, x, args)
    if rank == 0 and world == 1 and not args.no_hist:
        res["histogram"] = bench_histogram(fz, dev, stream, x)
    if rank == 0 and world == 1 and not args.no_rd:
        res["rate_distortion"] = bench_rate_distortion(fz, dev, x, res.get("e2e", {}).get("host_link"))
    if rank == 0 and world == 1 and not args.no_batch:
        res["batch"] = bench_batch(fz, dev, stream, args)
    if rank == 0 and world == 1 and not args.no_learned:
        res["learned"] = bench_learned(fz, dev, args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(x, args.cpu_slab, args.eb)
    if rank == 0:
        print(json.dumps(res), flush=True)
    ctx.close()


def host_link(dev, hpinned: torch.Tensor, dbuf: torch.Tensor):
    """Pinned host <-> device copy bandwidth over the same buffers the
    end-to-end step uses: host to device alone, device to host alone, and
    both directions at once on two streams (GB/s, CUDA events, best of 5)."""
    nbytes = dbuf.numel() * dbuf.element_size()
    d2 = torch.empty_like(dbuf)
    h2 = torch.empty(hpinned.shape, dtype=hpinned.dtype, pin_memory=True)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def best(fn, streams):
        out = []
        for _ in range(5):
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(streams[0])
            for st in streams[1:]:
                st.wait_event(e0)
            fn()
            for st in streams[1:]:
                ev = torch.cuda.Event()
                ev.record(st)
                streams[0].wait_event(ev)
            e1.record(streams[0])
            torch.cuda.synchronize(dev)
            out.append(e0.elapsed_time(e1))
        return min(out)

    def h2d():
        with torch.cuda.stream(s1):
            d2.copy_(hpinned, non_blocking=True)

    def d2h():
        with torch.cuda.stream(s1):
            h2.copy_(dbuf, non_blocking=True)

    def both():
        with torch.cuda.stream(s1):
            d2.copy_(hpinned, non_blocking=True)
        with torch.cuda.stream(s2):
            h2.copy_(dbuf, non_blocking=True)

    t1 = best(h2d, [s1])
    t2 = best(d2h, [s1])
    t3 = best(both, [s1, s2])
    return {"h2d_gbs": round(nbytes / (t1 * 1e-3) / 1e9, 2), "d2h_gbs": round(nbytes / (t2 * 1e-3) / 1e9, 2),
            "bidirectional_gbs": round(2 * nbytes / (t3 * 1e-3) / 1e9, 2), "bytes_per_copy": nbytes}


def _flush_l2(scratch: torch.Tensor):
    scratch.fill_(1)


def bench_configs(fz, dev, stream, args):
    """Every other plain-pipeline workload: compress and decompress
    throughput (CUDA events on the launching stream, L2 flushed before each
    timed call by writing 256 MiB), roofline fractions on forced bytes
    (compress 12N + S, decompress S + 4N), compression ratio and the largest
    error over the bound.  An entry (eb, C) of a workload's bounds uses
    Huffman chunks of C symbols instead of the block."""
    peak, _ = _peaks()
    scratch = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    specs = [("grf512_mode_spectrum", "3D FP32 512^3 Gaussian random field, per-mode amplitude |k|^-5/6 "
              "(power k^-5/3 per mode), seed 2", lambda: synth.grf3d(512, seed=2, slope=-1.0 / 3.0, device=dev),
              [1e-4])]
    specs.append(("hacc1d", "1D FP32 280,953,867 clustered particle coordinates in [0,256), seed 3",
                  lambda: synth.hacc1d(synth.HACC_N, seed=3, device=dev), [1e-2, 1e-3, 1e-4]))
    specs.append(("cesm2d", "2D FP32 1800x3600 lat/lon spherical-harmonic field (l <= 64) + noise, seed 4",
                  lambda: synth.cesm2d(1800, 3600, seed=4).to(dev), [1e-2, 1e-3, 1e-4, (1e-4, 256), (1e-4, 128)]))
    out = []
    for key, desc, make, ebs in specs:
        x = make().contiguous()
        N = x.numel()
        rng = float(x.max()) - float(x.min())
        ob = torch.empty(fz.compress_bound(x.shape), dtype=torch.uint8, device=dev)
        y = torch.empty_like(x)
        for spec in ebs:
            eb, chunk = spec if isinstance(spec, tuple) else (spec, 0)
            buf = fz.compress(x, eb, out=ob, chunk=chunk)
            fz.decompress(buf, out=y)
            err = float((y.double() - x.double()).abs().max()) / (eb * rng)
            S = buf.numel()
            tc, td = [], []
            for i in range(3 + args.config_reps):
                _flush_l2(scratch)
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record(stream)
                buf = fz.compress(x, eb, out=ob, chunk=chunk)
                e1.record(stream)
                _flush_l2(scratch)
                e2.record(stream)
                fz.decompress(buf, out=y)
                e3 = torch.cuda.Event(enable_timing=True)
                e3.record(stream)
                torch.cuda.synchronize(dev)
                if i >= 3:
                    tc.append(e0.elapsed_time(e1))
                    td.append(e2.elapsed_time(e3))
            mc, md = statistics.median(tc), statistics.median(td)
            out.append({"config": key, "workload": desc, "values": N, "eb_mode": "rel", "eb": eb,
                        "chunk": chunk or "block",
                        "compress_gbs": round(4 * N / (mc * 1e-3) / 1e9, 2),
                        "decompress_gbs": round(4 * N / (md * 1e-3) / 1e9, 2),
                        "compress_roofline_frac": round((12 * N + S) / (mc * 1e-3) / 1e9 / peak, 4),
                        "decompress_roofline_frac": round((S + 4 * N) / (md * 1e-3) / 1e9 / peak, 4),
                        "cr": round(4 * N / S, 4), "max_err_over_eb": round(err, 6),
                        "compress_ms": round(mc, 4), "decompress_ms": round(md, 4),
                        "timed_calls": args.config_reps, "l2": "flushed before each timed call"})
        del x, ob, y
        torch.cuda.empty_cache()
    return out


def bench_rate_distortion(fz, dev, x512, link):
    """§4.2's evaluation on the stand-in workloads: bit rate against PSNR at
    REL 1e-2 .. 1e-6, and Eq. 1's overall speedup over the host link measured
    in this run (host to device) and over 25 and 100 GB/s links."""
    import paper_2509_20563_gb300.report as report
    bws = [25.0, 100.0]
    if link and link.get("h2d_gbs"):
        bws.insert(0, float(link["h2d_gbs"]))
    fields = {"grf512": x512, "hacc1d": synth.hacc1d(synth.HACC_N, seed=3, device=dev),
              "cesm2d": synth.cesm2d(1800, 3600, seed=4).to(dev).contiguous()}
    rows = report.rate_distortion(fields, [1e-2, 1e-3, 1e-4, 1e-5, 1e-6], bws, reps=3)
    del fields
    torch.cuda.empty_cache()
    return {"bandwidths_gbs": bws, "rows": rows,
            "note": "Eq. 1 speedup = 1 / (((BW CR)^-1 + T_compress^-1) BW); PSNR from fz_error_stats"}


def bench_speed(fz, dev, stream, x512, args):
    """FZMod-Speed (§3.3): the same quantization codes through the bit-shuffle
    + zero-word encoder instead of Huffman, on the three stand-in workloads;
    compress and decompress GB/s (L2 flushed before each timed call, median
    of the timed calls), roofline fractions on the same forced bytes as the
    Huffman path (compress 12N + S, decompress S + 4N) and the CR beside the
    Huffman stream's."""
    peak, _ = _peaks()
    scratch = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    specs = [("grf512", lambda: x512, 1e-4),
             ("hacc1d", lambda: synth.hacc1d(synth.HACC_N, seed=3, device=dev), 1e-3),
             ("cesm2d", lambda: synth.cesm2d(1800, 3600, seed=4).to(dev).contiguous(), 1e-4)]
    out = []
    for key, make, eb in specs:
        x = make()
        N = x.numel()
        ob = torch.empty(fz.compress_bound(x.shape), dtype=torch.uint8, device=dev)
        y = torch.empty_like(x)
        S_h = fz.compress(x, eb, out=ob).numel()
        buf = fz.compress(x, eb, out=ob, encoder="shuffle")
        fz.decompress(buf, out=y)
        err = float((y.double() - x.double()).abs().max()) / (eb * (float(x.max()) - float(x.min())))
        tc, td = [], []
        for i in range(3 + args.config_reps):
            _flush_l2(scratch)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            buf = fz.compress(x, eb, out=ob, encoder="shuffle")
            e1.record(stream)
            _flush_l2(scratch)
            e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e2.record(stream)
            fz.decompress(buf, out=y)
            e3.record(stream)
            torch.cuda.synchronize(dev)
            if i >= 3:
                tc.append(e0.elapsed_time(e1))
                td.append(e2.elapsed_time(e3))
        S = buf.numel()
        mc, md = statistics.median(tc), statistics.median(td)
        out.append({"workload": key, "eb": eb, "values": N, "cr_shuffle": round(4 * N / S, 4),
                    "cr_huffman": round(4 * N / S_h, 4), "max_err_over_eb": round(err, 6),
                    "compress_gbs": round(4 * N / (mc * 1e-3) / 1e9, 2),
                    "decompress_gbs": round(4 * N / (md * 1e-3) / 1e9, 2),
                    "compress_roofline_frac": round((12 * N + S) / (mc * 1e-3) / 1e9 / peak, 4),
                    "decompress_roofline_frac": round((S + 4 * N) / (md * 1e-3) / 1e9 / peak, 4)})
        if key != "grf512":
            del x
        del ob, y
    del scratch
    torch.cuda.empty_cache()
    return out


def bench_quality(fz, dev, stream, x512, args):
    """FZMod-Quality (§3.3): the full-field multilevel interpolation predictor
    with the Huffman encoder, on the 512^3 Gaussian random field and on the
    smooth stitched 512^3 field, REL 1e-4 and 1e-3; compress and decompress
    GB/s (L2 flushed before each timed call, median of the timed calls),
    roofline fractions on the forced bytes of the Lorenzo path (compress
    12N + S, decompress S + 4N) and the CR beside the Lorenzo stream's."""
    peak, _ = _peaks()
    scratch = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    stitched = synth.stitched3d(512, device=dev)
    specs = [("grf512", x512, 1e-4), ("grf512", x512, 1e-3), ("stitched512", stitched, 1e-4),
             ("stitched512", stitched, 1e-3)]
    out = []
    for key, x, eb in specs:
        N = x.numel()
        ob = torch.empty(fz.compress_bound(x.shape), dtype=torch.uint8, device=dev)
        y = torch.empty_like(x)
        S_l = fz.compress(x, eb, out=ob).numel()
        buf = fz.compress(x, eb, out=ob, predictor="ginterp")
        fz.decompress(buf, out=y)
        err = float((y.double() - x.double()).abs().max()) / (eb * (float(x.max()) - float(x.min())))
        tc, td = [], []
        for i in range(3 + args.config_reps):
            _flush_l2(scratch)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            buf = fz.compress(x, eb, out=ob, predictor="ginterp")
            e1.record(stream)
            _flush_l2(scratch)
            e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e2.record(stream)
            fz.decompress(buf, out=y)
            e3.record(stream)
            torch.cuda.synchronize(dev)
            if i >= 3:
                tc.append(e0.elapsed_time(e1))
                td.append(e2.elapsed_time(e3))
        S = buf.numel()
        mc, md = statistics.median(tc), statistics.median(td)
        out.append({"workload": key, "eb": eb, "values": N, "cr_ginterp": round(4 * N / S, 4),
                    "cr_lorenzo1": round(4 * N / S_l, 4), "max_err_over_eb": round(err, 6),
                    "compress_gbs": round(4 * N / (mc * 1e-3) / 1e9, 2),
                    "decompress_gbs": round(4 * N / (md * 1e-3) / 1e9, 2),
                    "compress_roofline_frac": round((12 * N + S) / (mc * 1e-3) / 1e9 / peak, 4),
                    "decompress_roofline_frac": round((S + 4 * N) / (md * 1e-3) / 1e9 / peak, 4)})
        del ob, y
    del scratch, stitched
    torch.cuda.empty_cache()
    return out


def bench_histogram(fz, dev, stream, x512):
    """The histogram stage (§3.2) on its own, both methods: Lorenzo-1 codes of
    the 512^3 field (REL 1e-4), block-interpolation (cubic) codes of the
    stitched 512^3 field (REL 1e-4) and full-field interpolation codes of the
    same field at REL 1e-2 (whose codes repeat a few values most); 2N code
    bytes read per call, CUDA events on the launching stream, median of 20
    calls."""
    peak, _ = _peaks()
    out = []
    xs = synth.stitched3d(512, seed=200, region=64, device=dev)
    for name, x, pred, eb in (("grf512_lorenzo1", x512, "lorenzo1", 1e-4),
                              ("stitched512_interp_cubic", xs, "interp_cubic", 1e-4),
                              ("stitched512_ginterp_rel1e-2", xs, "ginterp", 1e-2)):
        codes, _, hist, _, _, _ = fz.lorenzo_quantize(x, eb, predictor=pred)
        srt = torch.sort(hist.double(), descending=True).values
        tot = hist.sum().item()
        row = {"codes": name, "n": int(codes.numel()), "top1_share": round(srt[0].item() / tot, 4),
               "top4_share": round(srt[:4].sum().item() / tot, 4)}
        for method in ("private", "topk"):
            h = fz.histogram(codes, 1024, method)
            assert torch.equal(h, hist)
            ts = []
            for _ in range(20):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fz.histogram(codes, 1024, method)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            gbs = 2 * codes.numel() / (ms * 1e-3) / 1e9
            row[method] = {"ms": round(ms, 4), "gbs": round(gbs, 1), "roofline_frac": round(gbs / peak, 4)}
        out.append(row)
        del codes
    del xs
    torch.cuda.empty_cache()
    return out


def bench_batch(fz, dev, stream, args):
    """64 fields of uneven size (32 cubes of side 32-256, 32 lat/lon fields of
    side 512-4096) at REL 1e-4: one batched call (graph replay after the
    first, autotuned call) against one fz_compress call per field; both
    timed with CUDA events on the launching stream."""
    xs = synth.batch_fields(seed=5, device=dev)
    n_vals = sum(x.numel() for x in xs)
    ctx = fz.Context(dev.index or 0)
    buf, offs = fz.compress_batch(xs, args.eb, ctx=ctx)      # autotune + capture
    tune_c = list(fz.profile(ctx=ctx).batch_tune)
    for _ in range(2):
        buf, offs = fz.compress_batch(xs, args.eb, out=buf, ctx=ctx)
    ys = fz.decompress_batch(buf, offs, ctx=ctx)
    for _ in range(2):
        fz.decompress_batch(buf, offs, outs=ys, ctx=ctx)
    S = offs[-1]
    reps = 5

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    t_bc = timed(lambda: fz.compress_batch(xs, args.eb, out=buf, ctx=ctx))
    t_bd = timed(lambda: fz.decompress_batch(buf, offs, outs=ys, ctx=ctx))
    # the per-field calls use the chunk the batch chose for each field
    hb = buf[: offs[-1]].cpu().numpy()
    chunks = [int(np.frombuffer(hb[offs[j] + 88: offs[j] + 92].tobytes(), np.uint32)[0]) for j in range(len(xs))]
    outs = [torch.empty(fz.compress_bound(x.shape), dtype=torch.uint8, device=dev) for x in xs]
    singles = [fz.compress(x, args.eb, out=o, chunk=c) for x, o, c in zip(xs, outs, chunks)]
    t_sc = timed(lambda: [fz.compress(x, args.eb, out=o, chunk=c) for x, o, c in zip(xs, outs, chunks)])
    recon = [torch.empty_like(x) for x in xs]
    t_sd = timed(lambda: [fz.decompress(b, out=r) for b, r in zip(singles, recon)])
    peak, _ = _peaks()
    forced_c = 12 * n_vals + S
    forced_d = 4 * n_vals + S
    prof = fz.profile(ctx=ctx)
    ctx.close()
    gb = lambda t: round(4 * n_vals / (t * 1e-3) / 1e9, 2)
    return {"workload": "64 fields: 32 cubes side U{32..256} + 32 lat/lon fields sides U{512..4096}, REL 1e-4",
            "values": n_vals, "stream_bytes": S, "cr": round(4 * n_vals / S, 4),
            "batch_compress_ms": round(t_bc, 4), "per_field_compress_ms": round(t_sc, 4),
            "batch_decompress_ms": round(t_bd, 4), "per_field_decompress_ms": round(t_sd, 4),
            "batch_compress_gbs": gb(t_bc), "per_field_compress_gbs": gb(t_sc),
            "batch_decompress_gbs": gb(t_bd), "per_field_decompress_gbs": gb(t_sd),
            "batch_compress_roofline_frac": round(forced_c / (t_bc * 1e-3) / 1e9 / peak, 4),
            "batch_decompress_roofline_frac": round(forced_d / (t_bd * 1e-3) / 1e9 / peak, 4),
            "speedup_compress": round(t_sc / t_bc, 3), "speedup_decompress": round(t_sd / t_bd, 3),
            "graphs": int(prof.batch_graphs), "plans": int(prof.batch_plans),
            "autotuned_compress": {"range_segment_log2": tune_c[0], "quant_ctas_per_sm": tune_c[1],
                                   "encode_ctas_per_sm": tune_c[2]},
            "autotuned_decode_ctas_per_sm": int(prof.batch_tune[3]),
            "autotuned_chunk": {"3d": int(prof.batch_chunk[0]), "1d_2d": int(prof.batch_chunk[1])}}


def bench_learned(fz, dev, args):
    """Selector network trained on the GPU (exhaustive-trial labels of 16
    stitched 256^3 fields, seeds 100-115), then compression ratio and
    throughput of plain Lorenzo-1, the exhaustive per-block trial and the
    network on the unseen stitched 512^3 field (seed 200) at REL 1e-4."""
    import paper_2509_20563_gb300.selector as sel
    t0 = time.perf_counter()
    fields = [synth.stitched3d(256, seed=100 + i, region=64, device=dev) for i in range(16)]
    feat, lab = sel.collect(fields, args.eb)
    del fields
    w, wb, hist = sel.train(feat, lab, epochs=12, batch=4096, lr=3e-3, seed=0)
    t_train = time.perf_counter() - t0
    x = synth.stitched3d(512, seed=200, region=64, device=dev)
    out = {"workload": "stitched 512^3 (smooth / oscillatory / noisy 64^3 regions), REL 1e-4, 8^3 blocks",
           "train_seconds": round(t_train, 2), "train_blocks": int(lab.numel()), "final_loss": round(hist[-1], 4)}
    N = x.numel()
    for name, kw in [("plain", {"predictor": "lorenzo1"}), ("exhaustive", {"predictor": "exhaustive"}),
                     ("mlp", {"predictor": "mlp", "selector_weights": wb})]:
        buf = fz.compress(x, args.eb, **kw)
        y = fz.decompress(buf)
        err = float((y.double() - x.double()).abs().max()) / (args.eb * (float(x.max()) - float(x.min())))
        ob = torch.empty(fz.compress_bound(x.shape), dtype=torch.uint8, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            fz.compress(x, args.eb, out=ob, **kw)
        e1.record()
        torch.cuda.synchronize(dev)
        yb = torch.empty_like(x)
        fz.decompress(buf, out=yb)
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record()
        for _ in range(3):
            fz.decompress(buf, out=yb)
        e3.record()
        torch.cuda.synchronize(dev)
        out[f"cr_{name}"] = round(4 * N / buf.numel(), 4)
        out[f"compress_gbs_{name}"] = round(4 * N * 3 / (e0.elapsed_time(e1) * 1e-3) / 1e9, 2)
        out[f"decompress_gbs_{name}"] = round(4 * N * 3 / (e2.elapsed_time(e3) * 1e-3) / 1e9, 2)
        out[f"max_err_over_eb_{name}"] = round(err, 6)
    out["mlp_vs_exhaustive"] = round(out["cr_mlp"] / out["cr_exhaustive"], 4)
    out["mlp_vs_plain"] = round(out["cr_mlp"] / out["cr_plain"], 4)
    return out


def _launches(L, ctx):
    import paper_2509_20563_gb300 as fz
    p = fz.Profile()
    L.fz_ctx_get_profile(ctx.handle, C.byref(p))
    return p.launches


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="fz", choices=["fz", "reference"])
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--eb", type=float, default=1e-4)
    ap.add_argument("--e2e-steps", type=int, default=16, help="end-to-end steps, shared by the host threads")
    ap.add_argument("--cpu-slab", type=int, default=160, help="z-slab of the field the CPU oracle times")
    ap.add_argument("--ref-slab", type=int, default=16, help="z-slab per step for --impl reference")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-field batched workload")
    ap.add_argument("--no-learned", action="store_true", help="skip the selector training and CR comparison")
    ap.add_argument("--no-configs", action="store_true", help="skip the other plain-pipeline workloads")
    ap.add_argument("--no-rd", action="store_true", help="skip the rate-distortion / Eq. 1 report")
    ap.add_argument("--no-hist", action="store_true", help="skip the histogram-stage comparison")
    ap.add_argument("--no-speed", action="store_true", help="skip the bit-shuffle (FZMod-Speed) pipeline")
    ap.add_argument("--no-quality", action="store_true",
                    help="skip the full-field interpolation (FZMod-Quality) pipeline")
    ap.add_argument("--config-reps", type=int, default=10, help="timed calls per extra workload and bound")
    ap.add_argument("--traffic", type=float, default=None, help="ncu dram bytes per launch of the dominant kernel")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        if args.impl == "reference":
            if rank != 0:
                return
        else:
            torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_fz(args, rank, world, local_rank)
    if world > 1 and args.impl != "reference":
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
