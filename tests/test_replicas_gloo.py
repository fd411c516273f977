"""Replica logic of multi-GPU runs, on CPU with two gloo ranks: shares of the
pairs cover every pair exactly once, seeds differ per rank, and the timing
reduction takes the slowest rank."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_2409_15615_gb300 import replicas

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = replicas.shard(257, rank, world)
    t = replicas.max_over_ranks(1.0 + rank * 2.5)
    dist.barrier()
    q.put((rank, lo, hi, replicas.pair_seed(1000, rank), t))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    covered = []
    for rank, lo, hi, seed, t in out:
        covered.extend(range(lo, hi))
        assert t == 3.5  # max over ranks of 1.0 and 3.5
    assert covered == list(range(257))
    assert len({o[3] for o in out}) == world


def test_shard_and_throughput():
    from paper_2409_15615_gb300 import replicas

    for n in (0, 1, 7, 256):
        for w in (1, 2, 3, 8):
            parts = [replicas.shard(n, r, w) for r in range(w)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(w - 1))
            assert max(h - l for l, h in parts) - min(h - l for l, h in parts) <= 1
    assert replicas.whole_job_throughput(10, 4, 2.0) == 20.0
    assert replicas.max_over_ranks(2.0) == 2.0
