"""The multi-process benchmark path (replicas: every rank compresses its
own field, no collective on the data path) reduces its timings correctly:
world_size 2 over gloo on the CPU."""
import os
import socket
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                     # rank 1 is the slowest
        dist.barrier()
        mx = bench.max_over_ranks(ms, world, "cpu")
        gbs = bench.aggregate_gbs(4, world, 1 << 30, mx)
        q.put((rank, mx, gbs))
    finally:
        dist.destroy_process_group()


def test_two_rank_reduction_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]
    want = 4 * 2 * (1 << 30) / 15e-3 / 1e9
    assert all(abs(o[2] - want) < 1e-9 * want for o in out)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.aggregate_gbs(2, 1, 10 ** 9, 1000.0) == 2.0
