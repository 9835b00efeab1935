"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): every
rank gets its own gather, the job time is the maximum over ranks, and the
whole-job throughput counts every rank's pairs."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = 10.0 + 5.0 * rank           # rank 1 is slower
    total = bench.job_time_ms(local, world, device="cpu")
    value = bench.job_value(4, world, total)
    out[rank] = (total, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_time_and_job_value():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    for r in range(world):
        total, value = out[r]
        assert total == 15.0
        assert abs(value - world * 4 / 0.015) < 1e-9


def test_ranks_get_independent_gathers(monkeypatch):
    import bench
    monkeypatch.setattr(bench, "N", 64)
    geo0, f0 = bench.make_workload(0)
    geo1, f1 = bench.make_workload(1)
    assert geo0 == geo1
    assert not np.allclose(f0, f1)
