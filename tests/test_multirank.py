"""The multi-rank host logic of bench.py on CPU: two gloo ranks, each with its
own scan (weak scaling), time taken as the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    ms = 100.0 + 50.0 * rank            # rank 1 is the slow one
    m = bench.max_over_ranks(ms, world, device="cpu")
    G, _, gd, _ = bench.workload("c1", rank)
    out[rank] = (m, bench.weak_value(1000, 10, world, m), float(G["mu"].sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_independent_scans():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")      # no fork of a process that already runs threads
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    (m0, v0, s0), (m1, v1, s1) = out[0], out[1]
    assert m0 == m1 == 150.0
    assert v0 == v1 == pytest.approx(1000 * 10 * 2 / 0.150)
    assert s0 != s1          # each rank projects its own seeded scan
