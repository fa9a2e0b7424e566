"""The multi-rank host logic of bench.py on CPU (gloo, world size 2).

The path has no exchange step: N ranks are N independent replicas that render
the same frame, and the job's time is the slowest rank's.  These tests run the
same helpers bench.py uses, with real gloo ranks and no GPU."""
import importlib.util
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port):
    import sys
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        # slowest rank decides the job time; every rank sees the same value
        local_ms = 10.0 + 5.0 * rank
        slowest = b.max_over_ranks(local_ms, "cpu", world)
        assert slowest == 10.0 + 5.0 * (world - 1), slowest
        v = b.job_throughput(world, 4, b.OUT_W * b.OUT_H / 1e6, slowest)
        assert abs(v - world * 4 * 1920 * 1080 / 1e6 / (slowest / 1e3)) < 1e-9 * v
        # replicas: every rank generates the identical seeded frame input
        if ROOT not in sys.path:
            sys.path.insert(0, ROOT)
        import scenes
        sc = scenes.random_scene(n=257, seed=3, sh_degree=3)
        digest = torch.tensor([float(np.float64(sc["means"]).sum()), float(np.float64(sc["sh"]).sum())],
                              dtype=torch.float64)
        got = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(got, digest)
        assert all(torch.equal(g, got[0]) for g in got)
        # the reference arm runs on rank 0 only: other ranks return 0 without work
        if rank != 0:
            class A:
                steps, warmup = 1, 0
            assert b.run_reference(A()) == 0
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_timing_world2():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    if not torch.distributed.is_available() or not torch.distributed.is_gloo_available():
        pytest.skip("gloo not available")
    mp.spawn(_rank_main, args=(2, _free_port()), nprocs=2, join=True)


def test_job_throughput_single():
    b = _bench()
    assert b.job_throughput(1, 10, 2.0, 1000.0) == pytest.approx(20.0)
    assert b.max_over_ranks(3.5, "cpu", 1) == 3.5
