"""Host logic of runs on several GPUs, exercised as world-size-2 gloo process groups on
the CPU: the deal of batched matrices to ranks, max/sum over ranks, and a replica step
whose timing is the maximum over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2102_08505_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, lr, w = shard.rank_info()
        work = [((7 * i) % 13) + 1.0 for i in range(37)]
        parts = shard.deal(work, w)
        mine = parts[r]
        # each rank "processes" its share; the job's time is the slowest rank's
        t = sum(work[i] for i in mine)
        tmax = shard.max_over_ranks(t)
        total = shard.sum_over_ranks(len(mine))
        shard.barrier()
        q.put((r, lr, w, parts, t, tmax, total))
    finally:
        dist.destroy_process_group()


def test_deal_is_a_balanced_partition():
    work = [5, 1, 1, 1, 1, 1, 4, 3, 2, 2]
    parts = shard.deal(work, 3)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(work)))
    loads = [sum(work[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(work)
    assert parts == shard.deal(work, 3)  # deterministic
    assert shard.deal([], 2) == [[], []]
    assert shard.deal(work, 1) == [list(range(len(work)))]
    with pytest.raises(ValueError):
        shard.deal(work, 0)


def test_gloo_world2_deal_and_max_over_ranks():
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
    res.sort()
    (r0, l0, w0, parts0, t0, m0, n0), (r1, l1, w1, parts1, t1, m1, n1) = res
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert parts0 == parts1 and sorted(parts0[0] + parts0[1]) == list(range(37))
    assert m0 == m1 == max(t0, t1)
    assert n0 == n1 == 37
