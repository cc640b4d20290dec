"""Multi-rank path on CPU: two gloo ranks place the serving requests independently and
agree, every request is served exactly once, the work is balanced, and the
max-over-ranks time reduction the benchmark uses returns the slowest rank."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2002_09217_gb300 import inputs, placement


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    reqs = inputs.serving_requests(n=64)
    mine = placement.my_share(reqs, rank, world)
    ids = torch.zeros(64, dtype=torch.int64)
    for r in mine:
        ids[r.rid] = 1
    dist.all_reduce(ids)                       # each request counted by exactly one rank
    work = torch.tensor([sum(placement.cost(r) for r in mine)], dtype=torch.float64)
    works = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(works, work)
    t = torch.tensor([1.0 + rank], dtype=torch.float64)   # per-rank elapsed time
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    out[rank] = (ids.tolist(), [float(w) for w in works], float(t))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_share_the_requests():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        ids, works, tmax = out[rank]
        assert ids == [1] * 64
        assert tmax == 2.0
        assert max(works) <= 1.25 * min(works)
    # the assignment is a pure function of the request list
    reqs = inputs.serving_requests(n=64)
    assert placement.assign(reqs, 2) == placement.assign(list(reqs), 2)
