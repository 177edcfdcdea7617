"""The multi-GPU path is replicas only (sources are independent): two gloo
ranks on the CPU exercise its host logic -- the barrier, the slowest rank's
time as the job's time, the whole-job value, rank 0 alone printing, and the
reference arm doing no work on other ranks."""
from __future__ import annotations

import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        reps = bench.Replicas(dist, torch.device("cpu"))
        reps.barrier()
        # each rank's own step time; the job takes the slowest
        ms = reps.max_over_ranks(100.0 + 50.0 * rank)
        value = bench.whole_job_gteps(world, 4096, 1000, ms * 1e-3)
        buf = io.StringIO()
        with redirect_stdout(buf):
            bench.emit({"value": value}, rank)
            # the reference arm: ranks other than 0 return before any work
            if rank != 0:
                bench.run_reference(None, None, None, None, "unused")
        reps.barrier()
        q.put((rank, ms, value, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        rank, ms, value, printed = q.get(timeout=120)
        out[rank] = (ms, value, printed)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks agree on the slowest time and on the whole-job value
    assert out[0][0] == out[1][0] == 150.0
    assert out[0][1] == out[1][1] == pytest.approx(2 * 4096 * 1000 / 0.150 / 1e9)
    # rank 0 alone printed, and printed one JSON line
    assert out[1][2] == ""
    assert out[0][2].count("\n") == 1 and '"value"' in out[0][2]

