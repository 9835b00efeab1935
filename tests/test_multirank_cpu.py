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


def test_shard_bounds_cover_every_gather_once():
    from paper_1604_07651_gb300.shard import shard_bounds
    rng = np.random.default_rng(5)
    for n in (0, 1, 2, 3, 7, 256):
        for world in (1, 2, 3, 4, 8):
            for weights in (n, list(rng.integers(30000, 1440000, n))):
                b = shard_bounds(weights, world)
                assert len(b) == world and b[0][0] == 0 and b[-1][1] == n
                assert all(b[r][1] == b[r + 1][0] for r in range(world - 1))   # contiguous, in order
                assert all(lo <= hi for lo, hi in b)
    # equal costs: shard sizes differ by at most one
    for n, world in ((7, 2), (256, 3), (5, 8)):
        sizes = [hi - lo for lo, hi in shard_bounds(n, world)]
        assert max(sizes) - min(sizes) <= 1
    # uneven costs: each shard within one item's cost of the equal split
    w = list(rng.integers(30000, 1440000, 256))
    for world in (2, 4, 8):
        costs = [sum(w[lo:hi]) for lo, hi in shard_bounds(w, world)]
        assert max(costs) - sum(w) / world <= max(w)


def _shard_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1604_07651_gb300.shard import gather_in_order, shard_bounds
    n = 11
    weights = [(i * 7919) % 13 + 1 for i in range(n)]
    lo, hi = shard_bounds(weights, world)[rank]
    # stand-in for this rank's transforms: one host array per gather of its shard
    local = [np.full(3, float(i)) + rank * 0.0 for i in range(lo, hi)]
    allres = gather_in_order(local, world)
    out[rank] = (lo, hi, [float(a[0]) for a in allres])
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_a_batch_and_reassemble_in_order():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_shard_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    (lo0, hi0, r0), (lo1, hi1, r1) = out[0], out[1]
    assert lo0 == 0 and hi0 == lo1 and hi1 == 11 and hi0 > 0 and lo1 < 11
    assert r0 == r1 == [float(i) for i in range(11)]
