"""Host logic of bench.py's N > 1 path on CPU (gloo, world size 2): the
whole-job figures are the maximum elapsed time and the summed work over
ranks, and the reference arm runs on rank 0 only."""
import contextlib
import io
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed, count = bench.aggregate_over_ranks(dist, 1.5 + rank, 1000 * (rank + 1), "cpu")
    out.put((rank, elapsed, count))
    # reference arm: rank 1 returns at once, printing nothing
    if rank == 1:
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            bench.run_reference(None)
        out.put(("ref", buf.getvalue()))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = [q.get() for _ in range(3)]
    ranks = sorted(g for g in got if g[0] != "ref")
    assert ranks == [(0, 2.5, 3000.0), (1, 2.5, 3000.0)]
    assert [g for g in got if g[0] == "ref"] == [("ref", "")]


def test_aggregate_without_process_group_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(None, 2.0, 7) == (2.0, 7.0)
