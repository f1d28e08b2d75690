"""The multi-rank timing of the benchmark (independent replicas, one per
GPU): the job time is the slowest rank's and the throughput counts the units
of every rank.  Run as two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        # rank 0 took 100 ms for its 10 units, rank 1 took 250 ms for its 10
        total, value = bench.job_throughput(100.0 if rank == 0 else 250.0, 10, 2, device="cpu")
        out.put((rank, total, value))
    finally:
        dist.destroy_process_group()


def test_job_throughput_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, total, value in res:
        assert total == 250.0                     # the slowest rank bounds the job
        assert value == pytest.approx(20 / 0.25)  # 2 ranks x 10 units in 0.25 s


def test_job_throughput_single_rank():
    import bench
    total, value = bench.job_throughput(400.0, 8, 1)
    assert total == 400.0 and value == pytest.approx(20.0)


def test_reference_arm_line_on_a_small_grid():
    """The reference arm (the CPU oracle) prints the base contract's line:
    the metric, solves/s from operator applications with the sample stated,
    zero copies in its e2e, and impl = reference."""
    import argparse

    import bench
    args = argparse.Namespace(n=128, rtol=1e-8, steps=2, warmup=1, gpus=1)
    out = bench.run_reference(args)
    assert out["impl"] == "reference" and out["metric"] == bench.METRIC
    assert out["unit"] == "solves/s" and out["higher_is_better"] is True
    assert out["value"] > 0 and out["steps"] == 2 and out["warmup"] == 1
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == out["value"]
    assert "operator applications" in cb["sample"]
    assert out["e2e"] == {"value": out["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
