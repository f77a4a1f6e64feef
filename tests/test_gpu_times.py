"""GPU parity of the intermediate-time samples (mlmc_trace_times,
mlmc_expmv_times; Sec. 5, Fig. 7, Algorithm 3's grid-time weights) against
the CPU oracle: every walk's index trajectory bit for bit and its samples at
t k / T within 1e-12 (FP64) / 1e-5 (FP32) relative, over several items per
row and rows that are screened and not; the controller's x(t_k) against the
FP64 judge exp(t_k A) v at every time."""
import numpy as np
import pytest

import mlmc_inputs as I
from oracle import reference as R
from oracle import walker as W

from gpu_helpers import compare_walks, make_plan, small_problems, torch_cuda

pytestmark = pytest.mark.gpu

PROBLEMS = small_problems()


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _trace_times(plan, level, coarse, rep_begin, reps, v, seed, n_times):
    from paper_1904_12754_gb300 import mlmc as M
    torch = torch_cuda()
    dv = torch.from_numpy(np.ascontiguousarray(v, np.float64)).cuda()
    rec = torch.zeros(plan.n * reps * M.WALK_RECORD_DTYPE.itemsize, dtype=torch.uint8,
                      device="cuda")
    yt = torch.zeros(plan.n * reps * (n_times - 1), dtype=torch.float64, device="cuda")
    plan.trace_times(level, coarse, rep_begin, reps, dv, seed, n_times, rec, yt)
    torch.cuda.synchronize()
    return rec.cpu().numpy().view(M.WALK_RECORD_DTYPE), yt.cpu().numpy().reshape(-1, n_times - 1)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["signed_301", "ba_3001", "laplace2d_32"])
@pytest.mark.parametrize("level,coarse,n_times", [(3, False, 8), (4, True, 4), (6, True, 8)])
def test_time_samples_match_oracle(name, prec, level, coarse, n_times):
    a, t, v = PROBLEMS[name]
    if prec == 0 and n_times > 8:
        pytest.skip("FP64 walks take at most 8 times")
    reps = 77
    with make_plan(a, t, prec) as plan:
        got, gyt = _trace_times(plan, level, coarse, 2, reps, v, 99, n_times)
    wk = W.Walker(a, t, v, seed=99, precision=W.FP64 if prec == 0 else W.FP32)
    orc, oyt = wk.walks_times(np.repeat(np.arange(a.n), reps),
                              np.tile(np.arange(2, 2 + reps), a.n), level, coarse, n_times)
    compare_walks(got, orc, v, wk.tables.dl, level, prec == 0, f"times {name}/{prec}/l{level}")
    scale = np.abs(oyt).max() + 1e-300
    rel = 1e-12 if prec == 0 else 1e-5
    bad = np.abs(gyt - oyt) > rel * np.abs(oyt) + (64 if prec else 1e3) * np.finfo(
        np.float32 if prec else np.float64).eps * scale
    assert not bad.any(), (np.argwhere(bad)[:5], gyt[bad][:5], oyt[bad][:5])
    assert np.any(oyt != 0)


def test_time_samples_with_split_items_and_a_tilt():
    a, t, v = PROBLEMS["ba_3001"]
    h = np.exp(0.5 * np.random.default_rng(2).standard_normal(a.n)).astype(np.float32)
    reps = 1100
    rows = np.arange(0, a.n, 17)
    with make_plan(a, t, 1, walks_per_lane=1, launch_reps=500) as plan:
        plan.set_tilt(h, 0.1, clocks=True)
        got, gyt = _trace_times(plan, 5, True, 3, reps, v, 5, 16)
    tb = W.build_tables(a, t, h, 0.1, clocks=True)
    wk = W.Walker(a, t, v, seed=5, precision=W.FP32, tables=tb)
    orc, oyt = wk.walks_times(np.repeat(rows, reps), np.tile(np.arange(3, 3 + reps), rows.size),
                              5, True, 16)
    sel = (rows[:, None] * reps + np.arange(reps)[None, :]).ravel()
    compare_walks(got[sel], orc, v, tb.dl, 5, False, "times tilt")
    scale = np.abs(oyt).max()
    assert np.all(np.abs(gyt[sel] - oyt) <= 1e-5 * np.abs(oyt) + 64 * 1.2e-7 * scale)


def test_walk_limit_keeps_the_passed_times():
    a = I.laplacian_2d(6, 1.0)
    t, v = 2.0, np.random.default_rng(2).random(a.n)
    with make_plan(a, t, 0, max_jumps=3) as plan:
        got, gyt = _trace_times(plan, 4, False, 0, 8, v, 3, 8)
    wk = W.Walker(a, t, v, seed=3, max_jumps=3)
    orc, oyt = wk.walks_times(np.repeat(np.arange(a.n), 8), np.tile(np.arange(8), a.n), 4, False, 8)
    assert np.array_equal(got["status"], orc["status"]) and np.any(orc["status"] == 1)
    assert np.allclose(gyt, oyt, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("prec", [0, 1])
def test_solution_at_intermediate_times(prec):
    # heat equation of the paper's Sec. 5 (2D Laplacian, C1): x(t k/4) at
    # every k against the FP64 judge
    w = I.workload_c1()
    from paper_1904_12754_gb300 import mlmc as M
    sched = M.schedule_default(precision=prec, num_levels=3, max_levels=8, l0=2,
                               time_budget_s=60.0)
    n_times = 4
    xt = np.zeros((n_times, w.a.n))
    with M.Plan.from_csr(w.a, w.t, sched, rel_tol=1e-2, stream=torch_cuda().cuda.current_stream().cuda_stream) as plan:
        plan.expmv_times(w.v, xt, n_times, seed=7)
        _, est = plan.stats()
        x = np.zeros(w.a.n)
        plan.expmv(w.v, x, seed=7)
    # the same walks give the final time as mlmc_expmv's x, up to the order of
    # the sums (the controller's decisions can differ in a sample count)
    assert np.linalg.norm(xt[-1] - x) / np.linalg.norm(x) <= 2e-2
    for k in range(1, n_times + 1):
        ref = R.expmv(w.a.scipy(), w.t * k / n_times, w.v)
        err = np.linalg.norm(xt[k - 1] - ref) / np.linalg.norm(ref)
        assert err <= 2e-2, (k, err)
