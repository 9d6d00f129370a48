"""Multi-rank bench logic on CPU (gloo, world size 2): replicas with a barrier and the
max over ranks of the per-step time; rank 0 alone prints."""
import os
import time

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    calls = []

    def step():
        calls.append(1)
        time.sleep(0.01 * (rank + 1))       # rank 1 is the slow replica

    t0 = [0.0]
    ms = bench.timed_replicas(torch, step, 3, 2, dist, "cpu",
                              lambda: t0.__setitem__(0, time.perf_counter()),
                              lambda: (time.perf_counter() - t0[0]) * 1e3)
    q.put((rank, ms, len(calls)))
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, n0), (r1, ms1, n1) = out
    assert n0 == n1 == 5                        # 2 warm-up + 3 timed steps on every rank
    assert ms0 == ms1                           # both report the max over ranks
    assert ms0 >= 20.0                          # the slow replica's ~20 ms per step


def test_single_rank_is_unchanged():
    assert bench.max_over_ranks(torch, 12.5, None, "cpu") == 12.5
