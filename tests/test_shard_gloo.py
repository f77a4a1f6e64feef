"""Host logic of a sharded solve on CPU ranks (gloo, world size 2).

Every rank takes mlmc_shard_range of each level's new walk indices, walks
them (here with the oracle's Algorithm 2 on the same counter-based streams)
and the exchange of paper_1904_12754_gb300.shard sums the per-level row
sums, totals and the deadline vote over the ranks through the ctypes
callback the library calls.  The merged sums must equal those of one rank
walking every index: the same walks (bit-equal trajectories by
construction of the generator), sums within rounding.  The GPU side of the
same path (the library's controller with two ranks) is in
tests/test_gpu_shard.py.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    import mlmc_inputs as I
    a = I.random_sparse(41, 4, seed=12, signed=True, diag=True)
    return a, 0.7, np.random.default_rng(9).standard_normal(a.n)


def _worker(rank, world, port, q, extras, vote):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch
    from oracle import walker as W
    from paper_1904_12754_gb300 import mlmc as M
    from paper_1904_12754_gb300.shard import DistExchange
    a, t, v = _problem()
    wk = W.Walker(a, t, v, seed=321, precision=W.FP64)
    n = a.n
    # two levels (l0 = 2 and the coupled level 3), two rounds of walks each
    levels = [(2, False), (3, True)]
    part = [np.zeros(n) for _ in levels]
    tot = [np.zeros(8) for _ in levels]
    done = [0, 0]
    ex = DistExchange(group=None, device="cpu", count=len(levels) * (n + 8) + 1)
    results = []
    for extra in extras:
        for k, (lvl, coarse) in enumerate(levels):
            lo, hi = M.shard_range(extra, rank, world)
            if hi > lo:
                s, y2, jumps, lim = wk.mlmcl(lvl, coarse, done[k] + lo, hi - lo)
                part[k] += s
                tot[k] += np.array([y2, jumps, (hi - lo) * n, lim, 0, 0, 0, 0])
            done[k] += extra
        # the library's exchange layout: nl x n sums | nl x 8 totals | vote
        buf = np.concatenate(part + tot + [np.array([1.0 if (vote and rank == 1) else 0.0])])
        ex.buf[:buf.size] = torch.from_numpy(buf)
        rc = ex.callback(buf.size, None)
        results.append((rc, ex.buf[:buf.size].numpy().copy()))
    q.put((rank, results))
    dist.barrier()
    dist.destroy_process_group()


def _run(extras, vote=False):
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q, extras, vote)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    return dict(q.get() for _ in range(2))


@pytest.mark.parametrize("extras", [[64, 37], [3, 1]])
def test_two_ranks_merge_to_the_one_rank_sums(extras):
    sys.path.insert(0, ROOT)
    from oracle import walker as W
    got = _run(extras)
    a, t, v = _problem()
    n = a.n
    wk = W.Walker(a, t, v, seed=321, precision=W.FP64)
    done = 0
    for r, extra in enumerate(extras):
        done += extra
        want = []
        for lvl, coarse in [(2, False), (3, True)]:
            s, y2, jumps, lim = wk.mlmcl(lvl, coarse, 0, done)
            want.append((s, y2, jumps))
        for rank in (0, 1):
            rc, buf = got[rank][r]
            assert rc == 0
            for k, (s, y2, jumps) in enumerate(want):
                gs = buf[k * n:(k + 1) * n]
                gt = buf[2 * n + 8 * k: 2 * n + 8 * (k + 1)]
                assert np.allclose(gs, s, rtol=1e-12, atol=1e-12 * np.abs(s).max())
                assert gt[1] == jumps and gt[2] == done * n
                assert abs(gt[0] - y2) <= 1e-12 * y2
            assert buf[-1] == 0.0
        # both ranks hold the same merged numbers, bit for bit
        assert np.array_equal(got[0][r][1], got[1][r][1])


def test_a_rank_past_its_deadline_stops_both():
    got = _run([8], vote=True)
    assert got[0][0][1][-1] == 1.0 and got[1][0][1][-1] == 1.0


def test_shard_ranges_partition_the_walks():
    sys.path.insert(0, ROOT)
    from paper_1904_12754_gb300 import mlmc as M
    for extra in (0, 1, 5, 64, 1001):
        for world in (1, 2, 3, 8):
            got = [M.shard_range(extra, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == extra
            assert all(got[r][1] == got[r + 1][0] for r in range(world - 1))
            sizes = [hi - lo for lo, hi in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(M.MlmcError):
        M.shard_range(10, 2, 2)
