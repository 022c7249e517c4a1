"""The N > 1 path of bench.py on CPU (gloo, world size 2): independent seeded models per rank (weak
scaling, no data exchange), max-over-ranks timing and whole-job throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_local = 100.0 + 50.0 * rank  # rank 1 is slower
        t_max = bench.max_over_ranks(t_local)
        value = bench.job_throughput(3, world, t_max)
        from paper_2306_17537_gb300 import inputs

        wl = inputs.config2(bench.rank_seed(7, rank), scale=16)
        out[rank] = (t_max, value, float(wl.sigma6.sum()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_max_time_and_solve_different_models():
    world, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    (t0, v0, s0), (t1, v1, s1) = out[0], out[1]
    assert t0 == t1 == 150.0
    assert v0 == v1 == pytest.approx(3 * 2 / 0.150)
    assert s0 != s1  # each rank has its own tool position / model


def test_single_process_helpers_without_a_process_group():
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_throughput(4, 1, 2000.0) == pytest.approx(2.0)
    assert bench.rank_seed(3, 0) == 3 and bench.rank_seed(3, 5) == 8
