"""Checkpoint and resume of a solve (mlmc_plan_save_state / _load_state /
mlmc_expmv_resume).  Walks are addressed by (replica, row, level), so a
resumed solve that continues from M_l draws exactly the walks an
uninterrupted one would: a state saved after walks 0..63 and resumed to 128
walks per row equals a fresh solve of walks 0..127."""
import numpy as np
import pytest

import mlmc_inputs as I
from oracle import reference as R

from gpu_helpers import small_problems, stream_handle

pytestmark = pytest.mark.gpu

PROBLEMS = small_problems()


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _plan(a, t, prec, pilot, cap, levels=3, l0=2, tol=1e-9, budget=600.0):
    from paper_1904_12754_gb300 import mlmc as M
    sched = M.schedule_default(precision=prec, num_levels=levels, max_levels=levels,
                               pilot_walks=pilot, max_walks_per_row=cap, time_budget_s=budget)
    sched.l0 = l0
    return M.Plan.from_csr(a, t, sched, rel_tol=tol, stream=stream_handle())


@pytest.mark.parametrize("prec", [0, 1])
def test_resume_continues_the_walk_indices(prec):
    a, t, v = PROBLEMS["signed_301"]
    with _plan(a, t, prec, 64, 64) as first:
        x0 = np.zeros(a.n)
        first.expmv(v, x0, seed=5, allow_not_converged=True)
        state = first.save_state()
    with _plan(a, t, prec, 64, 128) as more:
        more.load_state(state)
        assert more.save_state() == state            # load then save round-trips
        x1 = np.zeros(a.n)
        more.expmv_resume(x1, allow_not_converged=True)
        lv, _ = more.stats()
        assert [l["walks_per_row"] for l in lv] == [128] * 3
    with _plan(a, t, prec, 128, 128) as fresh:
        x2 = np.zeros(a.n)
        fresh.expmv(v, x2, seed=5, allow_not_converged=True)
    tol = 1e-12 if prec == 0 else 1e-6
    assert np.abs(x1 - x2).max() <= tol * np.abs(x2).max()
    assert np.abs(x0 - x2).max() > 1e3 * tol * np.abs(x2).max()   # the top-up changed x


def test_interrupted_solve_resumes_to_tolerance():
    from paper_1904_12754_gb300 import mlmc as M
    a = I.laplacian_2d(24)
    t = 0.3
    v = np.random.default_rng(2).random(a.n)
    ref = R.expmv(a.scipy(), t, v)
    tol = 2e-3
    sched = M.schedule_default(precision=M.FP64, num_levels=3, max_levels=8, pilot_walks=64,
                               max_walks_per_row=256)
    sched.l0 = 2
    with M.Plan.from_csr(a, t, sched, rel_tol=tol, stream=stream_handle()) as capped:
        x = np.zeros(a.n)
        rc = capped.expmv(v, x, seed=9, allow_not_converged=True)
        assert rc == M.MLMC_ERR_NOT_CONVERGED     # the sample cap stops it
        state = capped.save_state()
    sched.max_walks_per_row = 1 << 30
    results = []
    for _ in range(2):
        with M.Plan.from_csr(a, t, sched, rel_tol=tol, stream=stream_handle()) as plan:
            plan.load_state(state)
            y = np.zeros(a.n)
            plan.expmv_resume(y)
            _, est = plan.stats()
            assert est <= tol
            results.append(y)
    err = np.linalg.norm(results[0] - ref) / np.linalg.norm(ref)
    assert err <= 2.5 * tol
    # two plans resuming from the same state draw the same walks
    assert np.abs(results[0] - results[1]).max() <= 1e-12 * np.abs(results[0]).max()


def test_state_is_rejected_by_a_different_plan():
    a, t, v = PROBLEMS["signed_301"]
    with _plan(a, t, 1, 64, 64) as p:
        with pytest.raises(RuntimeError):
            p.save_state()                        # nothing solved yet
        x = np.zeros(a.n)
        p.expmv(v, x, seed=1, allow_not_converged=True)
        state = p.save_state()
        x_sum = p.expmv_sum(v, seed=2, allow_not_converged=True)
        with pytest.raises(RuntimeError):
            p.expmv_resume(x)                     # the last solve was not an mlmc_expmv
        assert np.isfinite(x_sum)
    with _plan(a, t, 1, 64, 64, l0=3) as other_l0:
        with pytest.raises(RuntimeError):
            other_l0.load_state(state)
    with _plan(a, t, 0, 64, 64) as other_precision:
        with pytest.raises(RuntimeError):
            other_precision.load_state(state)
    with _plan(a, t, 1, 64, 64) as same:
        with pytest.raises(RuntimeError):
            same.load_state(state[:-8])           # truncated
        same.load_state(state)
