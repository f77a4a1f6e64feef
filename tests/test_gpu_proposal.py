"""GPU parity of the importance-sampling proposal (the learned-proposal path)
against the CPU oracle: proposal tables bit for bit (log k/q to float
rounding), trajectories bit for bit with values that include the
likelihood-ratio factor, and unbiasedness against the exact moments."""
import numpy as np
import pytest

import mlmc_inputs as I
from oracle import reference as R
from oracle import walker as W

from gpu_helpers import compare_walks, gpu_trace, make_plan, small_problems, torch_cuda

pytestmark = pytest.mark.gpu

PROBLEMS = small_problems()


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _h_for(a, seed):
    # any positive h: a seeded function of the row (not a GPU value)
    rng = np.random.default_rng(seed)
    return (0.1 + rng.gamma(2.0, 1.0, a.n)).astype(np.float32)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_proposal_tables_match_oracle(name):
    a, t, v = PROBLEMS[name]
    h = _h_for(a, 3)
    with make_plan(a, t, 0) as plan:
        plan.set_proposal(h, 0.15)
        got = plan.export_proposal()
    tb = W.build_tables(a, t, h, 0.15)
    mask = np.zeros(max(a.nnz, 1), bool)
    for i in range(a.n):
        mask[a.row_ptr[i]:a.row_ptr[i] + tb.deg[i]] = True
    for k in ("thr", "keep_col", "keep_neg", "alias_col", "alias_neg"):
        assert np.array_equal(got[k][mask], getattr(tb, k)[mask]), k
    for k in ("lr_keep", "lr_alias"):
        g, o = got[k][mask].astype(np.float64), getattr(tb, k)[mask].astype(np.float64)
        assert np.all(np.abs(g - o) <= 2 * np.spacing(np.abs(o).astype(np.float32)) + 1e-12), k


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["signed_301", "ba_3001", "hub_777"])
@pytest.mark.parametrize("level,coarse", [(2, False), (4, True)])
def test_proposal_trajectories_match_oracle(name, prec, level, coarse):
    a, t, v = PROBLEMS[name]
    h = _h_for(a, 7)
    reps = 77  # > 32: lanes run several walks each (walk-state reset on refill)
    with make_plan(a, t, prec) as plan:
        plan.set_proposal(h, 0.1)
        got = gpu_trace(plan, level, coarse, 3, reps, v, seed=55)
    tb = W.build_tables(a, t, h, 0.1)
    wk = W.Walker(a, t, v, seed=55, precision=W.FP64 if prec == 0 else W.FP32, tables=tb)
    orc = wk.walks(np.repeat(np.arange(a.n), reps), np.tile(np.arange(3, 3 + reps), a.n), level,
                   coarse)
    compare_walks(got, orc, v, tb.dl, level, prec == 0, f"{name}/{prec}/l{level}")
    assert orc["jumps"].sum() > 0


@pytest.mark.parametrize("prec", [0, 1])
def test_proposal_estimator_is_unbiased(prec):
    torch = torch_cuda()
    a = I.random_sparse(7, 3, seed=31, signed=True, diag=True)
    t = 0.8
    v = np.random.default_rng(2).random(7) - 0.4
    h = _h_for(a, 11)
    m1, m2 = R.level_moments(a.dense(), t, v, 1, False)
    reps = 1 << 18
    with make_plan(a, t, prec) as plan:
        plan.set_proposal(h, 0.2)
        dv = torch.from_numpy(v).cuda()
        s = torch.zeros(a.n, dtype=torch.float64, device="cuda")
        tot = torch.zeros(8, dtype=torch.float64, device="cuda")
        plan.mlmcl(1, False, 0, reps, dv, 99, s, tot)
        torch.cuda.synchronize()
        s, y2 = s.cpu().numpy(), float(tot[0])
    # standard error from the proposal's own second moment (a bound on it)
    var = np.maximum(m2, y2 / reps)
    z = (s / reps - m1) / np.sqrt(var / reps)
    assert np.abs(z).max() <= 4.0


def test_proposal_rejects_bad_h():
    from paper_1904_12754_gb300 import mlmc as M
    a, t, v = PROBLEMS["signed_301"]
    h = _h_for(a, 1)
    h[5] = 0.0
    with make_plan(a, t, 0) as plan:
        with pytest.raises(M.MlmcError):
            plan.set_proposal(h, 0.1)
        with pytest.raises(M.MlmcError):
            plan.set_proposal(_h_for(a, 1), 0.0)
