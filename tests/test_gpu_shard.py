"""GPU: the library's sharded controller (mlmc_plan_set_shard) with two
ranks, each a host thread driving its own plan on this GPU.

The ranks' kernels never wait on one another: each rank synchronises its
own stream before the exchange, and the exchange is a host-side all-reduce
(a barrier over the threads, summing host buffers), called by the library
through the ctypes callback.  Checked:
  - a fixed sample (pilot only): the two-rank estimate equals the one-rank
    estimate of the same walks to rounding, and both ranks return the same x;
  - the full controller to a tolerance (FP64 and FP32, plain and with tilted
    clocks): both ranks converge to the same estimate, within the tolerance
    of the FP64 judge;
  - a failing exchange ends the solve with MLMC_ERR_EXCHANGE on the rank
    whose callback failed (a host-side failure; nothing faults on the GPU).
"""
import threading

import numpy as np
import pytest

import mlmc_inputs as I
from oracle import reference as R

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


class ThreadAllReduce:
    """Sum of the ranks' host buffers, for ranks that are threads."""

    def __init__(self, world, size, fail_rank=None):
        self.bufs = [np.zeros(size) for _ in range(world)]
        self.total = np.zeros(size)
        self.barrier = threading.Barrier(world, timeout=120)
        self.fail_rank = fail_rank
        self.calls = 0

    def callback(self, rank):
        from paper_1904_12754_gb300 import mlmc as M

        def _cb(count, _ctx):
            if rank == self.fail_rank:
                self.barrier.abort()
                return 1
            try:
                self.barrier.wait()
                if rank == 0:
                    self.total[:count] = sum(b[:count] for b in self.bufs)
                    self.calls += 1
                self.barrier.wait()
                self.bufs[rank][:count] = self.total[:count]
                self.barrier.wait()
                return 0
            except threading.BrokenBarrierError:
                return 1
        return M.EXCHANGE_FN(_cb)


def _solve(a, t, v, world, seed, rel_tol, h=None, fail_rank=None, **sched):
    from paper_1904_12754_gb300 import mlmc as M
    s = M.schedule_default(**sched)
    torch = torch_cuda()
    plans = [M.Plan.from_csr(a, t, s, rel_tol=rel_tol, stream=torch.cuda.Stream().cuda_stream)
             for _ in range(world)]
    if h is not None:
        for p in plans:
            p.set_tilt(h, 0.1, clocks=True)
    ex = None
    if world > 1:
        ex = ThreadAllReduce(world, plans[0].shard_buffer_doubles(), fail_rank)
        for r, p in enumerate(plans):
            p.set_shard(r, world, ex.callback(r), ex.bufs[r])
    xs = [np.zeros(a.n) for _ in range(world)]
    status = [None] * world
    stats = [None] * world

    def run(r):
        try:
            status[r] = plans[r].expmv(v, xs[r], seed, allow_not_converged=True)
            stats[r] = plans[r].stats()
        except M.MlmcError as e:
            status[r] = e.status

    threads = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=300)
        assert not th.is_alive()
    for p in plans:
        p.close()
    return xs, status, stats, ex


@pytest.mark.parametrize("prec", [0, 1])
def test_fixed_sample_two_ranks_equal_one(prec):
    a = I.random_sparse(500, 5, seed=4, signed=True, diag=True)
    t, v = 0.5, np.random.default_rng(1).standard_normal(500)
    kw = dict(precision=prec, num_levels=3, max_levels=3, pilot_walks=257, max_walks_per_row=257)
    x1, st1, s1, _ = _solve(a, t, v, 1, 77, 1e-6, **kw)
    x2, st2, s2, ex = _solve(a, t, v, 2, 77, 1e-6, **kw)
    assert ex.calls >= 1
    assert np.array_equal(x2[0], x2[1])               # the ranks agree bit for bit
    # FP64: the same walks summed in another order; FP32: the per-lane FP32
    # Kahan sums also group the walks differently (each rank's items), a few
    # FP32 ulps of a row's sum
    rtol = 1e-12 if prec == 0 else 1e-6
    assert np.allclose(x2[0], x1[0], rtol=rtol, atol=rtol * np.abs(x1[0]).max())
    lv1, lv2 = s1[0][0], s2[0][0]
    assert [l["walks_per_row"] for l in lv1] == [l["walks_per_row"] for l in lv2] == [257] * 3
    assert [l["jumps"] for l in lv1] == [l["jumps"] for l in lv2]


@pytest.mark.parametrize("prec", [0, 1])
def test_controller_two_ranks_reach_the_tolerance(prec):
    w = I.workload_c1()
    tol = 1e-2
    ref = R.expmv(w.a.scipy(), w.t, w.v)
    xs, st, stats, ex = _solve(w.a, w.t, w.v, 2, 5, tol, precision=prec, num_levels=3,
                               max_levels=8, pilot_walks=64)
    assert st == [0, 0]
    assert np.array_equal(xs[0], xs[1])
    err = np.linalg.norm(xs[0] - ref) / np.linalg.norm(ref)
    assert err <= 2 * tol
    assert stats[0][1] <= tol and stats[0][1] == stats[1][1]


def test_two_ranks_with_tilted_clocks_on_a_scale_free_graph():
    b = I.ba_graph(3001, 4, seed=5)
    t = 1.0 / I.lambda_max(b)
    v = np.ones(b.n)
    x = R.expmv(b.scipy(), t, v)
    h = np.sqrt(x * v).astype(np.float32)
    xs, st, stats, ex = _solve(b, t, v, 2, 9, 1e-3, h=h, precision=1, num_levels=3, max_levels=6)
    assert st == [0, 0]
    assert np.array_equal(xs[0], xs[1])
    assert np.linalg.norm(xs[0] - x) / np.linalg.norm(x) <= 2e-3


def test_a_failing_exchange_is_reported():
    from paper_1904_12754_gb300 import mlmc as M
    a = I.random_sparse(200, 4, seed=3, signed=True, diag=True)
    v = np.ones(200)
    xs, st, stats, ex = _solve(a, 0.4, v, 2, 1, 1e-3, fail_rank=1, precision=1, num_levels=2,
                               max_levels=2)
    assert st[1] == M.MLMC_ERR_EXCHANGE
    assert st[0] == M.MLMC_ERR_EXCHANGE     # its peer's barrier broke: its exchange failed too
