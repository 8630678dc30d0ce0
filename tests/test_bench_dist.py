"""The bench's multi-rank path on CPU (gloo, world size 2): every rank solves its own replica, the job's
time is the slowest rank's, the whole-job rate counts the units of all ranks, and under torchrun the
reference arm prints from rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_s = 1.0 + 2.0 * rank          # rank 0: 1 s, rank 1: 3 s
        slowest = bench.max_over_ranks(local_s, world)
        rate = bench.whole_job_rate(4, world, slowest)
        # the reference arm: only rank 0 runs and prints
        buf = io.StringIO()
        args = type("A", (), {})()
        if rank != 0:
            with redirect_stdout(buf):
                bench.run_reference(args)  # returns before touching args on ranks > 0
        q.put((rank, slowest, rate, buf.getvalue()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, slowest, rate, printed in out:
        assert slowest == 3.0                # max over ranks
        assert rate == pytest.approx(2 * 4 / 3.0)
    assert out[1][3] == ""                   # rank 1 of the reference arm prints nothing


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.whole_job_rate(3, 1, 1.5) == 2.0
