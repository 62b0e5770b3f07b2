"""Multi-process (world size 2, gloo on CPU) checks of the rank bookkeeping used by bench.py for
independent problems: disjoint, complete shards and max-time / sum-work reductions."""
import os
import socket

import pytest

from paper_2412_12360_b300 import ranks


def test_shard_partitions_items():
    for n in (0, 1, 5, 16, 17):
        for w in (1, 2, 3, 4, 8):
            got = sorted(i for r in range(w) for i in ranks.shard(n, w, r))
            assert got == list(range(n))
            sizes = [len(ranks.shard(n, w, r)) for r in range(w)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        ranks.shard(4, 2, 2)


def test_throughput_uses_slowest_rank():
    assert ranks.throughput([10, 10], [1.0, 2.0]) == 10.0


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
    mine = ranks.shard(16, world, rank)
    t, u = ranks.reduce_time_and_work(1.0 + rank, float(len(mine)))
    q.put((rank, mine, t, u))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(out[0][1] + out[1][1]) == list(range(16))
    for _, _, t, u in out:
        assert t == 2.0 and u == 16.0
