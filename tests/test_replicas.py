"""Multi-rank path on the CPU: world_size-2 gloo ranks aggregate replica throughput
(units summed over ranks, time = the slowest rank)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    from paper_2409_02964_gb300.replicas import job_throughput
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    secs = [2.0, 3.0][rank]
    units = [100.0, 200.0][rank]
    value, tmax, total = job_throughput(secs, units)
    out[rank] = (value, tmax, total)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_throughput():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        value, tmax, total = out[r]
        assert tmax == 3.0 and total == 300.0
        assert value == pytest.approx(100.0)


def test_single_process_is_its_own_job():
    from paper_2409_02964_gb300.replicas import job_throughput
    assert job_throughput(2.0, 50.0) == (25.0, 2.0, 50.0)
