"""The multi-process host logic on CPU: two gloo ranks shard a request stream with no overlap
and agree on the slowest rank's time and the total of processed models."""
import os

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    from paper_2506_11657_gb300 import dist as D
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, lr = D.rank_info()
        mine = D.shard(range(11), r, ws)
        t = D.max_over_ranks(1.0 + r)
        n = D.sum_over_ranks(len(mine))
        q.put((r, mine, t, n))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29600 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert out[0][1] == [0, 2, 4, 6, 8, 10] and out[1][1] == [1, 3, 5, 7, 9]
    assert all(o[2] == 2.0 for o in out)       # slowest rank's time
    assert all(o[3] == 11 for o in out)        # every request served exactly once


def test_shard_single_process():
    from paper_2506_11657_gb300 import dist as D
    assert D.shard([5, 6, 7], 0, 1) == [5, 6, 7]
    with pytest.raises(ValueError):
        D.shard([1], 2, 2)
    assert D.max_over_ranks(3.5) == 3.5
