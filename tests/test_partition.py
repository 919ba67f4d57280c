"""Multi-GPU stream partitioning, exercised with world_size 2 on CPU (gloo):
each rank computes its own share; the all-gathered shares cover every stream
exactly once and the per-rank token counts stay within one stream length."""
import os

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import synthetic as S
from paper_2602_19626_gb300.partition import partition_streams


def test_partition_cover_and_balance():
    lens = S.stream_lengths(2, 256, 512, 16384)
    for world in (1, 2, 3, 8):
        parts = partition_streams(lens, world)
        flat = sorted(j for p in parts for j in p)
        assert flat == list(range(len(lens)))
        loads = [int(sum(lens[j] for j in p)) for p in parts]
        assert max(loads) - min(loads) <= int(max(lens))


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lens = S.stream_lengths(2, 256, 512, 16384)
    mine = partition_streams(lens, world)[rank]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    if rank == 0:
        out.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_partition_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    lens = S.stream_lengths(2, 256, 512, 16384)
    assert sorted(gathered[0] + gathered[1]) == list(range(256))
    assert not set(gathered[0]) & set(gathered[1])
    loads = [sum(int(lens[j]) for j in g) for g in gathered]
    assert abs(loads[0] - loads[1]) <= int(lens.max())
