"""The multi-GPU form is replicas (signals are independent; no data-path
collective): each rank transforms its own seeded signals and the job's rate
is all signals over the slowest rank's time.  The host side of that path is
checked here with two gloo ranks on the CPU: disjoint signal seeds, the
max-over-ranks reduction, and the whole-job value."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import torch
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        seed0 = bench.rank_seed0(rank)
        my_ms = 10.0 * (rank + 1)  # rank 1 is the slower one
        m = bench.max_over_ranks(torch, dist, ws, my_ms)
        seeds = torch.arange(seed0, seed0 + 152, dtype=torch.int64)
        gathered = [torch.zeros_like(seeds) for _ in range(ws)]
        dist.all_gather(gathered, seeds)
        q.put((rank, m, bench.job_value(ws, 152, 200, m), [g.tolist() for g in gathered]))
    finally:
        dist.destroy_process_group()


def test_two_replicas_on_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, value, gathered in res:
        assert m == 20.0  # the slowest rank's time, on every rank
        assert abs(value - 2 * 152 * 200 / 0.020) < 1e-6
        assert not set(gathered[0]) & set(gathered[1])  # disjoint signals
