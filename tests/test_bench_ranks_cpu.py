"""The multi-rank path of bench.py on CPU: two `gloo` ranks (the GPU run uses one process per GPU
over NCCL, replicas of the same step).  The job's step time is the slowest rank's, every rank
agrees on it, and the barrier that brackets the timed region lets no rank through early."""
import os
import socket
import sys
import time

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = bench.rank_env()
        # rank 1 arrives late: nobody leaves the barrier before it arrives
        if rank == 1:
            time.sleep(0.5)
        t0 = time.time()
        bench.ranks_barrier()
        waited = time.time() - t0
        t = bench.max_over_ranks(10.0 + 5.0 * rank)
        out.put((rank, w, r, lr, waited, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_step():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    world, port = 2, _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r, w, rr, lr, waited, t) in enumerate(res):
        assert (r, w, rr, lr) == (rank, world, rank, rank)
        assert t == 15.0
    assert res[0][4] >= 0.3   # rank 0 waited for rank 1 at the barrier


def test_single_process_needs_no_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.rank_env() == (1, 0, 0)
    assert bench.max_over_ranks(3.5) == 3.5
    bench.ranks_barrier()
