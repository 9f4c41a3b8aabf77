"""Replica aggregation across two gloo ranks on CPU (the multi-GPU path is replicas only)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2506_21908_gb300.replicas import aggregate, throughput
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units = 1000.0 * (rank + 1)
    secs = 2.0 + rank
    total, tmax = aggregate(units, secs)
    out[rank] = (total, tmax, throughput(units, secs))
    dist.destroy_process_group()


def test_two_rank_replica_aggregation():
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
        total, tmax, thr = out[r]
        assert total == pytest.approx(3000.0)
        assert tmax == pytest.approx(3.0)
        assert thr == pytest.approx(1000.0)


def test_single_process_is_identity():
    from paper_2506_21908_gb300.replicas import aggregate
    assert aggregate(5.0, 2.0) == (5.0, 2.0)
