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


def test_reference_arm_under_torchrun_two_ranks():
    """`bench.py --impl reference` launched as the driver launches it for
    N = 2 (torchrun, one process per rank, rendezvous on 127.0.0.1): rank 0
    times the oracle on whole frames of the workload and prints one JSON line
    with the reference arm's keys and the same config as the GPU arm's; the
    other rank exits 0 without work or output."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    import bench
    from paper_2412_09723_gb300 import scenes

    cam = scenes.CAM_VGA
    assert d["config"] == bench._config(cam, d["config"]["duplicates_K"])
    assert d["config"]["duplicates_K"] > 0
