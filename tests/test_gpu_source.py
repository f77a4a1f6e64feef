"""GPU parity of the source term (Algorithm 3): with mlmc_plan_set_source the
walks add Simpson sums of F along their paths.  The GPU evaluates each holding
segment's geometric sum in closed form; the oracle accumulates grid point by
grid point as the paper's listing does.  Trajectories must match bit for bit,
samples within 1e-12 (FP64) / 1e-5 (FP32) of their scale, the pilot sample
within rounding, and the controller's solution of du/dt = Au + F within the
tolerance of the exact exp(tA)v + int_0^t exp(sA)F ds."""
import numpy as np
import pytest

import mlmc_inputs as I
from oracle import reference as R
from oracle import walker as W

from gpu_helpers import EPS32, EPS64, gpu_trace, make_plan, small_problems, stream_handle

pytestmark = pytest.mark.gpu

PROBLEMS = small_problems()


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _f_for(a, seed):
    return np.random.default_rng(seed).standard_normal(a.n)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["signed_301", "ba_3001", "hub_777", "laplace2d_32"])
@pytest.mark.parametrize("level,coarse", [(1, False), (3, True), (6, True)])
def test_source_trajectories_match_oracle(name, prec, level, coarse):
    a, t, v = PROBLEMS[name]
    f = _f_for(a, 3)
    reps = 45
    with make_plan(a, t, prec, l0=1) as plan:
        plan.set_source(f)
        got = gpu_trace(plan, level, coarse, 2, reps, v, seed=321)
    fp64 = prec == 0
    wk = W.Walker(a, t, v, seed=321, precision=W.FP64 if fp64 else W.FP32, f=f)
    rows = np.repeat(np.arange(a.n), reps)
    orc = wk.walks(rows, np.tile(np.arange(2, 2 + reps), a.n), level, coarse)
    for fld in ("end", "jumps", "hash", "status", "sign"):
        assert np.array_equal(got[fld], orc[fld]), fld
    want = orc["y"] + orc["src"]
    n_grid = 2.0 ** level
    scale = np.abs(v[orc["end"]]) * np.exp(np.abs(orc["log_c"]) + np.abs(orc["log_f"]))
    terms = (orc["jumps"] + 3.0) * np.abs(wk.tables.dl).max() / n_grid
    if fp64:
        tol = 1e-12 * np.abs(want) + 64 * EPS64 * scale * terms + 1e-11 * orc["src_abs"]
    else:
        tol = 1e-5 * np.abs(want) + 64 * EPS32 * scale * (terms + 1.0) + 2e-5 * orc["src_abs"]
    bad = np.flatnonzero(np.abs(got["y"] - want) > tol)
    assert bad.size == 0, (bad[:5], got["y"][bad[:5]], want[bad[:5]])
    assert np.abs(orc["src"]).max() > 0


@pytest.mark.parametrize("prec", [0, 1])
def test_source_pilot_sample_matches_oracle(prec):
    from paper_1904_12754_gb300 import mlmc as M
    a, t, v = PROBLEMS["signed_301"]
    f = _f_for(a, 4)
    levels, pilot = 3, 64
    sched = M.schedule_default(precision=prec, num_levels=levels, max_levels=levels,
                               pilot_walks=pilot, max_walks_per_row=pilot)
    sched.l0 = 2
    with M.Plan.from_csr(a, t, sched, rel_tol=1e-6, stream=stream_handle()) as plan:
        plan.set_source(f)
        x = np.zeros(a.n)
        plan.expmv(v, x, seed=17, allow_not_converged=True)
    wk = W.Walker(a, t, v, seed=17, precision=W.FP64 if prec == 0 else W.FP32, f=f)
    want = np.zeros(a.n)
    for l in range(2, 2 + levels):
        s, _, _, lim = wk.mlmcl(l, l > 2, 0, pilot)
        assert lim == 0
        want += s / pilot
    tol = 1e-11 if prec == 0 else 2e-5
    assert np.abs(x - want).max() <= tol * np.abs(want).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_inhomogeneous_solution_reaches_tolerance(prec):
    from paper_1904_12754_gb300 import mlmc as M
    a = I.random_sparse(400, 4, seed=31, signed=True, diag=True)
    t = 0.5
    rng = np.random.default_rng(6)
    v, f = rng.standard_normal(a.n), rng.standard_normal(a.n)
    exact = R.expmv(a.scipy(), t, v) + R.expmv_source_exact(a.scipy(), t, f)
    tol = 1e-2
    sched = M.schedule_default(precision=prec, num_levels=3, max_levels=10, time_budget_s=60.0)
    with M.Plan.from_csr(a, t, sched, rel_tol=tol, stream=stream_handle()) as plan:
        assert plan.info()["l0"] >= 1
        plan.set_source(f)
        x = np.zeros(a.n)
        plan.expmv(v, x, seed=11)
        _, est = plan.stats()
        # v = 0: the integral alone
        y = np.zeros(a.n)
        plan.expmv(np.zeros(a.n), y, seed=12)
    err = np.linalg.norm(x - exact) / np.linalg.norm(exact)
    assert est <= tol and err <= 2.5 * tol, (est, err)
    integ = R.expmv_source_exact(a.scipy(), t, f)
    assert np.linalg.norm(y - integ) / np.linalg.norm(integ) <= 2.5 * tol


def test_source_rejections():
    from paper_1904_12754_gb300 import mlmc as M
    a, t, v = PROBLEMS["signed_301"]
    f = _f_for(a, 1)
    with make_plan(a, t, 1, l0=0) as plan:
        with pytest.raises(RuntimeError):
            plan.set_source(f)                       # Simpson needs l0 >= 1
    with make_plan(a, t, 1, l0=1) as plan:
        plan.set_source(f)
        with pytest.raises(RuntimeError):
            plan.set_proposal(np.ones(a.n, np.float32), 0.1)
        torch = __import__("torch")
        dv = torch.from_numpy(v).cuda()
        sums = torch.zeros(a.n, dtype=torch.float64, device="cuda")
        tot = torch.zeros(5, dtype=torch.float64, device="cuda")
        with pytest.raises(RuntimeError):
            plan.mlmcl(1, True, 0, 4, dv, 1, sums, tot)  # coarse level 1: no even coarse grid
        with pytest.raises(RuntimeError):
            M.Batch([plan], M.schedule_default(precision=1), rel_tol=1e-2, stream=stream_handle())
        plan.set_source(None)
        plan.set_proposal(np.ones(a.n, np.float32), 0.1)  # allowed again
        torch.cuda.synchronize()
    with make_plan(a, t, 1, l0=1, mode=M.FORWARD) as plan:
        with pytest.raises(RuntimeError):
            plan.set_source(f)
