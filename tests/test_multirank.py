"""The N > 1 host path of bench.py on CPU: two gloo ranks, each with its own
(independent) work, a barrier, and the job's rate from the slowest rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_ms = [100.0, 250.0][rank]  # rank 1 is the slow one
    dist.barrier()
    rate, max_ms = bench.whole_job_rate(50, local_ms, world, dist)
    out[rank] = (rate, max_ms)
    dist.destroy_process_group()


def test_two_rank_rate_uses_the_slowest_rank():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        rate, max_ms = res[r]
        assert max_ms == 250.0
        assert rate == pytest.approx(2 * 50 / 0.25)


def test_single_rank_rate():
    import bench

    rate, max_ms = bench.whole_job_rate(10, 20.0, 1)
    assert max_ms == 20.0 and rate == pytest.approx(500.0)
