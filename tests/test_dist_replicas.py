"""The N > 1 path of bench.py on CPU: world-size-2 gloo ranks, each timing an
independent replica; the reported time is the maximum over ranks after a
barrier (replicas only: one problem has no exchange step on this build)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench._dist()
    assert (ws, r, local) == (world, rank, rank)
    bench._barrier(ws)
    t = bench._reduce_max(1.5 + rank, ws)      # rank-local "replica time"
    out[rank] = t
    dist.destroy_process_group()


def test_replica_max_over_ranks_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 2.5


def _ref_worker(rank, world, port, out):
    import argparse
    import contextlib
    import io
    import json
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.cpu_baseline_sample = lambda *a, **k: (2.0 + rank, 0.01)   # stands in for the oracle's dense solve
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(argparse.Namespace(warmup=3, steps=2, gpus=world))
    lines = [json.loads(s) for s in buf.getvalue().splitlines() if s.strip()]
    out[rank] = lines
    dist.destroy_process_group()


def test_reference_arm_prints_on_rank_0_only_gloo():
    """--impl reference under torchrun: rank 0 times the oracle and prints one
    JSON line; the other ranks exit without work."""
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_ref_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[1] == []
    (line,) = out[0]
    assert line["impl"] == "reference" and line["value"] == 2.0 and line["n_gpus"] == world
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": 2.0, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["higher_is_better"] is False and line["unit"] == "s"
