"""bench.py's multi-GPU logic with two gloo ranks on the CPU: each rank renders its own views (weak
scaling, no data-path collective), the job's time is the slowest rank's, and the reported rate counts
every rank's rays."""

import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        w = bench.make_workload(512)
        views = bench.rank_views(w, rank)
        eyes = [list(map(float, c["c2w"][[3, 7, 11]])) for c in views]
        gathered = [None] * world
        dist.all_gather_object(gathered, eyes)
        local_ms = 10.0 * (rank + 1)
        job_ms = bench.reduce_max(local_ms, world)
        rate = bench.job_rate(1_000_000, world, job_ms)
        q.put((rank, gathered, job_ms, rate, len(views)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, job_ms, rate, n_views in out:
        assert job_ms == 20.0                       # slowest rank
        assert rate == pytest.approx(1_000_000 * 2 / 0.020 / 1e6)
        assert n_views == 8
        assert gathered[0] != gathered[1]           # different views per rank
