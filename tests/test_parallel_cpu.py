"""Multi-rank host logic on CPU (gloo, world size 2): sharding of the
simulation batch, all-gather of per-simulation results and the max-over-ranks
timing reduction used by the benchmark."""
import os
import socket

import numpy as np
import pytest

from paper_1701_03549_gb300 import parallel

RESULT_DTYPE = np.dtype([(f, "<u4") for f in
                         ("burnt", "inter", "target", "steps", "status",
                          "trials")])


@pytest.mark.parametrize("n,world", [(0, 1), (1, 2), (4096, 2), (4097, 3),
                                     (10, 8), (7, 7)])
def test_shards_cover_the_batch_once(n, world):
    seen = []
    sizes = []
    for r in range(world):
        lo, hi = parallel.shard_range(n, r, world)
        seen.extend(range(lo, hi))
        sizes.append(hi - lo)
    assert seen == list(range(n))
    assert max(sizes) - min(sizes) <= 1


def test_rank_seed_ranges_are_disjoint():
    a = parallel.rank_seed_offset(0, 1000)
    b = parallel.rank_seed_offset(1, 1000)
    assert b - a == 1000


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 11
        lo, hi = parallel.shard_range(n, rank, world)
        mine = np.zeros(hi - lo, RESULT_DTYPE)
        mine["burnt"] = np.arange(lo, hi) * 3
        mine["steps"] = rank + 1
        allr = parallel.gather_results(mine, world)
        t = parallel.max_over_ranks(0.5 + rank, world)
        c = parallel.sum_over_ranks(10 ** 12 + rank, world)
        q.put((rank, allr["burnt"].tolist(), allr["steps"].tolist(), (t, c)))
    finally:
        dist.destroy_process_group()


def test_gather_max_and_sum_over_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q))
             for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, burnt, steps, t in out:
        assert burnt == [3 * i for i in range(11)]
        assert steps == [1] * 6 + [2] * 5
        assert t == (1.5, 2 * 10 ** 12 + 1)


def _shard_worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        def fake(lo, hi):        # a deterministic stand-in for one GPU's shard
            r = np.zeros(hi - lo, RESULT_DTYPE)
            r["burnt"] = (np.arange(lo, hi) * 7919) % 1000
            r["trials"] = np.arange(lo, hi)
            return r
        got = parallel.sharded_results(23, fake, rank, world)
        q.put((rank, got["burnt"].tolist(), got["trials"].tolist()))
    finally:
        dist.destroy_process_group()


def test_sharded_results_equal_the_unsharded_batch():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 3, port, q))
             for r in range(3)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, burnt, trials in out:
        assert burnt == [(i * 7919) % 1000 for i in range(23)]
        assert trials == list(range(23))


def _dying_worker(rank, world, port, q):
    import datetime

    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(3)              # dies between generations, before the gather
    import time
    t0 = time.time()
    try:
        parallel.sharded_results(8, lambda lo, hi: np.zeros(hi - lo,
                                                             RESULT_DTYPE),
                                 rank, world)
        q.put((rank, "no error", time.time() - t0))
    except Exception as e:   # the collective fails instead of hanging
        q.put((rank, type(e).__name__, time.time() - t0))
    q.close()
    q.join_thread()          # flush the message before the hard exit
    os._exit(0)


def test_a_dead_rank_is_an_error_not_a_hang():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dying_worker, args=(r, 2, port, q))
             for r in range(2)]
    for p in procs:
        p.start()
    rank, what, dt = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert rank == 0 and what != "no error", (what, dt)
    assert dt < 60
    assert procs[1].exitcode == 3
