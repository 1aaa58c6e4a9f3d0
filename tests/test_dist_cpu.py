"""Host-side multi-process logic with 2 gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest

from paper_2009_08500_gb300 import dist


def test_shard_covers_every_item_once():
    for n in (0, 1, 7, 4096, 4097):
        for world in (1, 2, 3, 8):
            parts = [dist.shard(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as tdist
    dist.init("gloo")
    r, w, lr = dist.env()
    lo, hi = dist.shard(10, r, w)
    dist.barrier()
    q.put((r, w, lo, hi, dist.max_over_ranks(1.5 + r), dist.sum_over_ranks(hi - lo)))
    tdist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 2, 0, 5, 2.5, 10.0), (1, 2, 5, 10, 2.5, 10.0)]
