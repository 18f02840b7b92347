"""The N > 1 host path on the CPU: two gloo ranks (no GPU)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1707_02347_gb300 import replicas  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mx = replicas.max_over_ranks(1.5 + rank)          # per-rank "time"
        g = torch.full((3,), float(rank + 1))
        replicas.sum_over_ranks(g)
        mine = list(replicas.shard(24, rank, world))
        q.put((rank, mx, g.tolist(), mine))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out.sort()
    assert [o[1] for o in out] == [2.5, 2.5]               # max over ranks
    assert out[0][2] == out[1][2] == [3.0, 3.0, 3.0]       # sum over ranks
    assert sorted(out[0][3] + out[1][3]) == list(range(24))  # shards cover every shot once
    assert replicas.job_throughput(10.0, world, 2.5) == 8.0


def test_shard_sizes():
    for n in (0, 1, 5, 24, 25):
        for world in (1, 2, 3, 8):
            parts = [replicas.shard(n, r, world) for r in range(world)]
            assert sum(len(p) for p in parts) == n
            assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1
            flat = [i for p in parts for i in p]
            assert flat == list(range(n))
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)
