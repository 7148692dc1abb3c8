"""The multi-GPU path is replicas only (each rank solves its own copy; no data exchange): its host logic
runs here with two gloo ranks on the CPU.  The job time is the slowest rank's on every rank, the whole-job
value counts the solves of all ranks, and the reference arm (the oracle) runs on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = [2.0, 3.0][rank]
    t_max = bench.slowest_rank_seconds(elapsed, world)
    # the reference arm on a rank other than 0 returns at once and prints nothing
    out = io.StringIO()
    if rank != 0:
        with redirect_stdout(out):
            bench.run_reference(None, rank, world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t_max, world * 5 / t_max, out.getvalue()))


def test_two_replicas_take_the_slowest_rank():
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
    assert [r[1] for r in res] == [3.0, 3.0]                   # max over ranks, on every rank
    assert res[0][2] == pytest.approx(2 * 5 / 3.0)              # all ranks' solves / slowest time
    assert res[1][3] == ""                                       # rank 1: no reference-arm output


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank_seconds(1.5, 1) == 1.5
