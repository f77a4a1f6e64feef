"""Host logic of bench.py's N > 1 path on CPU (gloo, world size 2): the
whole-job figures are the maximum elapsed time and the summed work over
ranks, the reference arm runs on rank 0 only, and every rank installs rank
0's learned law (one law or time pieces) before the sharded solve."""
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


class _FakePlan:
    """Records the law a rank installs (the plan's tilt calls, no GPU)."""

    def __init__(self, n, pieces, h):
        self.n = n
        self._pieces = pieces
        self._h = h
        self.installed = None

    def tilt_pieces(self):
        return self._pieces

    def export_h(self):
        return self._h

    def set_tilt(self, h, alpha, clocks=True):
        self.installed = ("one", 1, [float(x) for x in h])

    def set_tilt_pieces(self, h, alpha):
        self.installed = ("pieces", int(h.shape[0]), [float(x) for x in h.ravel()])


def _share_worker(rank, world, port, pieces, out):
    sys.path.insert(0, ROOT)
    import numpy as np
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    n = 5
    # each rank learned its own law; rank 1's differs in pieces and values
    k = pieces if rank == 0 else 1
    h = (np.arange(k * n, dtype=np.float32) + 1.0 + 100.0 * rank)
    plan = _FakePlan(n, k, h if k == 1 else h.reshape(k, n))
    bench.share_law(plan, dist, rank, "cpu")
    out.put((rank, plan.installed))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("pieces", [1, 4])
def test_every_rank_installs_rank_0s_law(pieces):
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_share_worker, args=(r, 2, port, pieces, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(q.get() for _ in range(2))
    want = ("one" if pieces == 1 else "pieces", pieces,
            [float(x) for x in range(1, pieces * 5 + 1)])
    assert got[0] == want and got[1] == want, got
