"""Host logic of the multi-process benchmark, on CPU with the gloo backend.

With N > 1 every rank runs its own replica of the workload (the solves are
independent; there is no data-path collective).  The timing is the maximum
over ranks and the job throughput counts all replicas; the reference arm
prints from rank 0 only.
"""
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


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench._max_over_ranks(100.0 + 50.0 * rank, torch.device("cpu"))
    value = bench._job_mlups(world, 512 ** 3, 200, 3, ms)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, value))


def test_max_over_ranks_and_job_throughput_with_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want_ms = 150.0
    for rank, ms, value in out:
        assert ms == want_ms
        assert value == pytest.approx(2 * 512 ** 3 * 200 * 3 / (want_ms / 1e3) / 1e6)


def test_reference_arm_prints_only_on_rank0(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        workload = "stack32"
        steps = 1
        warmup = 0
        gpus = 2
        ref_planes = 4
        ref_seconds = 0.1

    bench.run_reference(Args())
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank0(capsys, monkeypatch):
    import json

    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")

    class Args:
        workload = "stack32"
        steps = 1
        warmup = 0
        gpus = 1
        ref_planes = 4
        ref_seconds = 0.2

    bench.run_reference(Args())
    d = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "MLUP/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
