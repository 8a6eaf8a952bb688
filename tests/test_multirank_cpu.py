"""The N > 1 path of bench.py on the host: two gloo ranks (world size 2).
Replicas only (independent ciphertexts per rank, no collective on the data
path): the only exchanges are the barrier and the max-over-ranks of the timed
region, and the job's throughput counts every rank's units over that time.
Under torchrun the reference arm runs on rank 0 alone."""
import contextlib
import io
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist)  # rank 1 is the slowest
    dist.barrier()
    value = bench.job_throughput(world, 8, 50, ms)
    args = type("A", (), {"warmup": 1, "steps": 1})()
    out = io.StringIO()
    rc = None
    if rank == 1:  # a non-zero rank of the reference arm exits at once, silently
        with contextlib.redirect_stdout(out):
            rc = bench.run_reference(args, rank, world)
    q.put((rank, ms, value, rc, out.getvalue()))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_aggregate_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, v0, _, _), (r1, ms1, v1, rc1, out1) = res
    assert ms0 == ms1 == 15.0                      # both ranks see the slowest rank's time
    assert v0 == v1 == 2 * 8 * 50 / 0.015          # whole-job units over that time
    assert rc1 == 0 and out1 == ""                 # reference arm: rank 1 does no work


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(12.5, None) == 12.5
    assert bench.job_throughput(1, 8, 10, 1000.0) == 80.0
