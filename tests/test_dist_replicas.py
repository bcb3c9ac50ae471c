"""The N > 1 path of the benchmark is replicas only: every rank advances its own
grid, the job time is the maximum over ranks (taken after a barrier) and the value
is the cell updates of all ranks over that time.  Checked here on CPU with two
gloo ranks (no GPU: the host logic only)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.dist_env()
        bench.barrier(torch)
        # each replica reports its own time; the job takes the slowest
        job_ms = bench.max_over_ranks(torch, 100.0 + 25.0 * rank)
        value = bench.job_mlups(1000, 10, w, job_ms)
        out[rank] = (r, w, lr, job_ms, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank_and_sum_the_work():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        rr, w, lr, job_ms, value = res[r]
        assert (rr, w, lr) == (r, world, r)
        assert job_ms == 125.0  # the slowest rank, on every rank
        assert value == pytest.approx(1000 * 10 * world / 0.125 / 1e6)


def test_single_process_values_without_a_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(torch, 3.5) == 3.5
    assert bench.job_mlups(16_777_216, 1000, 1, 337.0) == pytest.approx(16_777_216 * 1000 / 0.337 / 1e6)
