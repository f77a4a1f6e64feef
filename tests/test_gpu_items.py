"""GPU parity on the work decomposition that the full-size launches use.

The walk kernel hands out work items of one row's chunk of walks
(32 x walks-per-lane walks) and splits a request into launches of a bounded
number of replicas per row.  The full-size benchmark runs several items per
row (automatic chunks of 4096 walks, items with r_lo > 0) and several
launches per request; these tests make both happen at oracle-checkable sizes
and compare every walk bit for bit with the oracle (Algorithm 2 with the
readings R1-R5):

- item split: reps = 2*4096 + 37 walks per row, with the automatic chunk
  (three items per row, the last ragged) and with walks_per_lane forced to
  1 and 2 (chunks of 32 and 64 walks: hundreds of items per row);
- FP32 shared first-uniform blocks (four walks per Philox block, reading R4)
  that straddle item boundaries: rep_begin = 1, 2, 3 (mod 4), so the first
  block of every item starts mid-block;
- launch split: launch_reps forced to 37 and 100, so one request becomes
  hundreds of launches whose replica ranges start at arbitrary offsets;
- the same splits in forward mode (Eq. 5), where launch_reps bounds the walks
  of one launch;
- the proposal (importance-sampling) tables under the same splits.
"""
import numpy as np
import pytest

import mlmc_inputs as I
from oracle import walker as W

from gpu_helpers import (compare_fwd_walks, compare_walks, gpu_trace, make_plan, oracle_walks,
                         torch_cuda)

pytestmark = pytest.mark.gpu

REPS = 2 * 4096 + 37


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _problems():
    out = {}
    # BA graph: most rows have t L_ii < 1 (screened short walks), the hubs
    # have t L_ii > 1 (one-wave long walks).
    b = I.ba_graph(240, 4, seed=11)
    out["ba_240"] = (b, 1.0 / I.lambda_max(b), np.ones(b.n))
    # signed rows with diagonals, t L_ii spread around 1
    a = I.random_sparse(97, 6, seed=23, signed=True, diag=True)
    out["signed_97"] = (a, 0.6, np.random.default_rng(4).standard_normal(a.n))
    return out


PROBLEMS = _problems()


def _check(name, prec, level, coarse, rep_begin, reps, seed, **sched):
    a, t, v = PROBLEMS[name]
    fp64 = prec == 0
    with make_plan(a, t, prec, **sched) as plan:
        got = gpu_trace(plan, level, coarse, rep_begin, reps, v, seed=seed)
    rows = np.repeat(np.arange(a.n), reps)
    rr = np.tile(np.arange(rep_begin, rep_begin + reps), a.n)
    orc, wk = oracle_walks(a, t, v, seed, fp64, rows, rr, level, coarse)
    compare_walks(got, orc, v, wk.tables.dl, level, fp64,
                  f"{name}/prec{prec}/l{level}/{sched}/rb{rep_begin}")
    assert orc["jumps"].sum() > 0
    # both kinds of walk happen: ones that never leave the row and ones that jump
    assert np.any(orc["jumps"] == 0) and np.any(orc["jumps"] > 0)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("rep_begin", [1, 2, 3])
@pytest.mark.parametrize("walks_per_lane", [0, 1, 2])
def test_items_split_rows_bit_exact(prec, rep_begin, walks_per_lane):
    # walks_per_lane 0: automatic 4096-walk items, 3 per row (4096, 4096, 37);
    # 1 and 2: 258 and 129 items per row.  rep_begin = 1..3 (mod 4) puts
    # every item's first FP32 shared block mid-block.
    _check("ba_240", prec, 3, True, rep_begin, REPS, 4321, walks_per_lane=walks_per_lane)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("level,coarse", [(2, False), (5, True)])
def test_items_split_signed_rows_bit_exact(prec, level, coarse):
    _check("signed_97", prec, level, coarse, 6, REPS, 99, walks_per_lane=1)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("launch_reps", [37, 100])
def test_launch_split_bit_exact(prec, launch_reps):
    # one request of 8229 replicas per row as 223 (or 83) launches whose
    # replica ranges start at offsets that are not multiples of 4 or 32
    _check("ba_240", prec, 4, True, 3, REPS, 777, launch_reps=launch_reps)


def test_launch_and_item_split_together_fp32_l0():
    _check("ba_240", 1, 2, False, 1, REPS, 31337, launch_reps=1000, walks_per_lane=2)


def test_launch_split_row_sums_equal_one_launch():
    # mlmcl per-row sums and totals do not depend on how the request is split
    # (same walks, FP32 values; the sums differ only by the rounding of a
    # different grouping: each lane's FP32 Kahan sum over its walks of an item
    # is exact to a few FP32 ulps of the item's sum, so 1e-6 of the largest
    # row sum bounds the difference)
    torch = torch_cuda()
    a, t, v = PROBLEMS["ba_240"]
    res = []
    for sched in ({}, {"launch_reps": 37, "walks_per_lane": 1}):
        with make_plan(a, t, 1, **sched) as plan:
            dv = torch.from_numpy(v).cuda()
            s = torch.zeros(a.n, dtype=torch.float64, device="cuda")
            tot = torch.zeros(8, dtype=torch.float64, device="cuda")
            plan.mlmcl(3, True, 2, REPS, dv, 5, s, tot)
            torch.cuda.synchronize()
            res.append((s.cpu().numpy(), tot.cpu().numpy()))
    (s0, t0), (s1, t1) = res
    assert np.all(t0[1:5] == t1[1:5])
    assert np.abs(s0 - s1).max() <= 1e-6 * np.abs(s0).max()
    assert abs(t0[0] - t1[0]) <= 1e-6 * t0[0]


@pytest.mark.parametrize("prec", [0, 1])
def test_proposal_items_and_launches_split_bit_exact(prec):
    a, t, v = PROBLEMS["ba_240"]
    h = (0.1 + np.random.default_rng(5).gamma(2.0, 1.0, a.n)).astype(np.float32)
    reps = 4096 + 45
    with make_plan(a, t, prec, walks_per_lane=1, launch_reps=300) as plan:
        plan.set_proposal(h, 0.1)
        got = gpu_trace(plan, 3, True, 2, reps, v, seed=808)
    tb = W.build_tables(a, t, h, 0.1)
    wk = W.Walker(a, t, v, seed=808, precision=W.FP64 if prec == 0 else W.FP32, tables=tb)
    orc = wk.walks(np.repeat(np.arange(a.n), reps), np.tile(np.arange(2, 2 + reps), a.n), 3, True)
    compare_walks(got, orc, v, tb.dl, 3, prec == 0, "proposal split")


def _fwd_trace(plan, level, coarse, g0, walks, v, seed):
    from paper_1904_12754_gb300 import mlmc as M
    torch = torch_cuda()
    dv = torch.from_numpy(np.ascontiguousarray(v, np.float64)).cuda()
    rec = torch.zeros(walks * M.WALK_RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    plan.trace(level, coarse, g0, walks, dv, seed, rec)
    torch.cuda.synchronize()
    return rec.cpu().numpy().view(M.WALK_RECORD_DTYPE)


@pytest.mark.parametrize("prec", [0, 1])
def test_forward_launch_and_item_split_bit_exact(prec):
    # forward mode: launch_reps bounds the walks of one launch (here 333, so
    # 151 launches starting at arbitrary walk indices) and walks_per_lane = 1
    # gives 32-walk items; every walk against the oracle's forward walker
    from paper_1904_12754_gb300 import mlmc as M
    a, t, v = PROBLEMS["signed_97"]
    walks, g0 = 50_000, 7
    with make_plan(a, t, prec, mode=M.FORWARD, launch_reps=333, walks_per_lane=1) as plan:
        got = _fwd_trace(plan, 3, True, g0, walks, v, 4242)
    fw = W.ForwardWalker(a, t, v, seed=4242, precision=W.FP64 if prec == 0 else W.FP32)
    compare_fwd_walks(got, fw.walks_fwd(g0, walks, 3, True), fw, 3, prec == 0, "forward split")
