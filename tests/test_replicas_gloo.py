"""Multi-rank logic of the replica runs, on CPU with the gloo backend."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2609_26108_b300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [2.0, 3.0][rank]
    value, slowest = replicas.job_throughput(local, 192)
    out[rank] = (value, slowest)
    dist.barrier()
    dist.destroy_process_group()


def test_job_throughput_takes_slowest_rank_and_all_units():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        value, slowest = out[r]
        assert slowest == 3.0
        assert value == pytest.approx(2 * 192 / 3.0)


def test_single_process_and_shards():
    value, slowest = replicas.job_throughput(2.0, 100)
    assert value == 50.0 and slowest == 2.0
    items = list(range(64))
    parts = [replicas.shard(items, r, 3) for r in range(3)]
    assert sum(parts, []) == items
    assert max(map(len, parts)) - min(map(len, parts)) <= 1
