"""The N > 1 path of bench.py on the CPU: two gloo ranks.

Ranks render independent head poses (replicas, no data-path collective); the
only exchange is the max over ranks of the timed duration, and the whole-job
value counts every rank's pixels over that slowest time.  The reference arm
runs on rank 0 only."""
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


def _worker(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    bench.init_dist(world)
    try:
        # the slowest rank sets the job time on every rank
        local_ms = 10.0 * (rank + 1)
        mx = bench.max_over_ranks(local_ms)
        value = bench.whole_job_rate(1000.0 * 5, mx, world)
        # each rank draws its own head poses (weak scaling over independent eyes)
        _, heads, _ = bench.make_workload("tiny", 2, rank)
        pose = [float(x) for x in heads[0][0].pose[9:12]]
        # the reference arm: rank 0 alone runs and prints; the others exit 0 without work
        buf = io.StringIO()
        rc = None
        if rank != 0:
            class Args:
                workload, poses, warmup, steps, gpus = "tiny", 1, 0, 1, world
            with redirect_stdout(buf):
                rc = bench.run_reference(Args())
        out.put((rank, mx, value, pose, rc, buf.getvalue()))
    finally:
        bench.finish_dist(world)


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        rank, mx, value, pose, rc, printed = q.get(timeout=240)
        res[rank] = (mx, value, pose, rc, printed)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][0] == res[1][0] == 20.0
    assert abs(res[0][1] - 2 * 5000 / 0.020 / 1e6) < 1e-9 and res[0][1] == res[1][1]
    assert res[0][2] != res[1][2]  # independent head poses per rank
    assert res[1][3] == 0 and res[1][4] == ""  # reference arm: rank 1 does nothing


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert not dist.is_initialized()
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.whole_job_rate(4.608e6, 0.5, 1) == pytest.approx(9216.0)
