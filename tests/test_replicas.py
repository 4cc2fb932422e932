"""Host logic of the multi-GPU path (replicas), with two gloo ranks on CPU."""
import os
import socket

import pytest

from paper_1709_10314_gb300.replicas import job_throughput, max_over_ranks, rank_seed


def test_rank_keys_disjoint():
    per = 64
    ranges = [set(range(rank_seed(1, r, per), rank_seed(1, r, per) + per)) for r in range(8)]
    for i in range(8):
        for j in range(i + 1, 8):
            assert not ranges[i] & ranges[j]
    assert rank_seed(2**64 - 1, 1, 1) == 0  # 64-bit wrap like the Philox key


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    vals = max_over_ranks([1.0 + rank, 10.0 - rank])
    dist.barrier()
    q.put((rank, vals, rank_seed(5, rank, 64)))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for rank, vals, key in res:
        assert vals == [2.0, 10.0]           # max over both ranks
        assert key == 5 + 64 * rank          # disjoint key ranges
    assert job_throughput(100, 2, 0.5) == pytest.approx(400.0)
