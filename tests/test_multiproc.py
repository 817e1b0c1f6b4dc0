"""The N-GPU form of the benchmark on CPU: replicas in a world of two gloo
ranks (rendezvous on 127.0.0.1).  Bodies are independent, so the replicas
exchange nothing but the step time; each rank draws its own population; the
reference arm runs on rank 0 alone."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    from paper_2509_04666_gb300 import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # step time of the slowest replica, seen by every rank
        mx = bench.max_over_ranks(100.0 + 25.0 * rank, dist, "cpu")
        args = type("A", (), {"n_bodies": 64, "n_frames": 3288, "ref_sample": 4, "warmup": 0,
                              "steps": 1, "gpus": world})()
        w = bench.make_workload(args, rank)
        buf = io.StringIO()
        with redirect_stdout(buf):
            rc = bench.run_reference(args) if rank == 1 else 0
        q.put((rank, mx, float(w.states[0, 0]), w.seed, rc, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_replicas_agree_on_the_slowest_step():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, mx, x0, seed, rc, printed = q.get(timeout=300)
        out[rank] = (mx, x0, seed, rc, printed)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 125.0            # max over ranks on both
    assert out[0][2] != out[1][2] and out[0][1] != out[1][1]   # own population per rank
    assert out[1][3] == 0 and out[1][4] == ""          # reference arm: rank 1 does nothing


def test_job_rate_counts_every_replica():
    import bench
    assert bench.job_rate(1, 757000 * 365.0, 2000.0) == pytest.approx(1.381525e8)
    assert bench.job_rate(4, 1000.0, 500.0) == 4 * bench.job_rate(1, 1000.0, 500.0)
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
