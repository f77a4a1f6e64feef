"""GPU parity of the forward mode (the full-vector representation, Eq. 5)
against the CPU oracle: the device transpose and the tables of A^T bit for
bit, each walk's start, end, jump count, sign and hash bit for bit with its
value within 1e-12 (FP64) / 1e-5 (FP32) relative, the pilot-only estimate
against the oracle's replay, and the controller's result on nonsymmetric
matrices against the FP64 judge."""
import numpy as np
import pytest

import mlmc_inputs as I
from oracle import reference as R
from oracle import walker as W

from gpu_helpers import (EPS32, EPS64, compare_fwd_walks as _compare, make_plan, small_problems,
                         stream_handle, torch_cuda)

pytestmark = pytest.mark.gpu

PROBLEMS = small_problems()


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _fwd_plan(a, t, precision, **kw):
    from paper_1904_12754_gb300 import mlmc as M
    return make_plan(a, t, precision, mode=M.FORWARD, **kw)


def _fwd_trace(plan, level, coarse, g0, walks, v, seed):
    from paper_1904_12754_gb300 import mlmc as M
    torch = torch_cuda()
    dv = torch.from_numpy(np.ascontiguousarray(v, np.float64)).cuda()
    rec = torch.zeros(walks * M.WALK_RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    plan.trace(level, coarse, g0, walks, dv, seed, rec)
    torch.cuda.synchronize()
    return rec.cpu().numpy().view(M.WALK_RECORD_DTYPE)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_transposed_tables_bit_exact(name):
    a, t, v = PROBLEMS[name]
    b = W.transpose(a)
    with _fwd_plan(a, t, 0) as plan:
        got = plan.export_tables()
    tb = W.build_tables(b, t)
    assert np.array_equal(got["deg"], tb.deg)
    for k, ref in (("l_ii", tb.L), ("dl", tb.dl), ("inv_rate", tb.inv_rate)):
        assert np.array_equal(got[k].view(np.uint64), ref.view(np.uint64)), k
    assert np.array_equal(got["dl32"].view(np.uint32), tb.dl32.view(np.uint32))
    mask = np.zeros(max(b.row_ptr[-1], 1), bool)
    for i in range(b.n):
        mask[b.row_ptr[i]:b.row_ptr[i] + tb.deg[i]] = True
    for k in ("thr", "keep_col", "keep_neg", "alias_col", "alias_neg"):
        assert np.array_equal(got[k][mask], getattr(tb, k)[mask]), k


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("level,coarse", [(2, False), (5, True)])
def test_forward_trajectories_bit_exact(name, prec, level, coarse):
    a, t, v = PROBLEMS[name]
    v = v.copy()
    v[::7] = 0.0          # zero entries are never starts
    walks, g0 = 5003, 11  # several work items and a ragged tail
    with _fwd_plan(a, t, prec) as plan:
        got = _fwd_trace(plan, level, coarse, g0, walks, v, seed=4321)
    fw = W.ForwardWalker(a, t, v, seed=4321, precision=W.FP64 if prec == 0 else W.FP32)
    orc = fw.walks_fwd(g0, walks, level, coarse)
    _compare(got, orc, fw, level, prec == 0, f"{name}/{prec}/l{level}")
    assert np.all(v[got["pad"]] != 0.0)
    assert orc["jumps"].sum() > 0


def test_forward_high_walk_indices():
    # walk index bits 32-63 sit in counter word 1
    a, t, v = PROBLEMS["signed_301"]
    g0 = (1 << 33) + 5
    with _fwd_plan(a, t, 1) as plan:
        got = _fwd_trace(plan, 3, True, g0, 700, v, seed=99)
    fw = W.ForwardWalker(a, t, v, seed=99, precision=W.FP32)
    _compare(got, fw.walks_fwd(g0, 700, 3, True), fw, 3, False, "high g")


@pytest.mark.parametrize("prec", [0, 1])
def test_forward_proposal_trajectories(prec):
    a, t, v = PROBLEMS["hub_777"]
    h = (0.1 + np.random.default_rng(5).gamma(2.0, 1.0, a.n)).astype(np.float32)
    with _fwd_plan(a, t, prec) as plan:
        plan.set_proposal(h, 0.1)
        got = _fwd_trace(plan, 4, True, 0, 3001, v, seed=8)
    fw = W.ForwardWalker(a, t, v, seed=8, precision=W.FP64 if prec == 0 else W.FP32, h=h,
                         alpha=0.1)
    _compare(got, fw.walks_fwd(0, 3001, 4, True), fw, 4, prec == 0, "forward IS")


@pytest.mark.parametrize("prec", [0, 1])
def test_forward_pilot_sample_matches_oracle(prec):
    from paper_1904_12754_gb300 import mlmc as M
    a, t, v = PROBLEMS["signed_301"]
    levels, pilot = 3, 40
    sched = M.schedule_default(precision=prec, num_levels=levels, max_levels=levels,
                               pilot_walks=pilot, max_walks_per_row=pilot, mode=M.FORWARD)
    with M.Plan.from_csr(a, t, sched, rel_tol=1e-6, stream=stream_handle()) as plan:
        x = np.zeros(a.n)
        plan.expmv(v, x, seed=61, allow_not_converged=True)
        l0 = plan.info()["l0"]
        stats, _ = plan.stats()
    m = pilot * a.n
    assert [s["walks_per_row"] for s in stats] == [m] * levels
    fw = W.ForwardWalker(a, t, v, seed=61, precision=W.FP64 if prec == 0 else W.FP32)
    want = np.zeros(a.n)
    for l in range(l0, l0 + levels):
        sx, _, _, lim = fw.mlmcl_fwd(l, l > l0, 0, m)
        assert lim == 0
        want += sx / m
    tol = 1e-11 if prec == 0 else 2e-5
    assert np.abs(x - want).max() <= tol * np.abs(want).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_forward_expmv_reaches_tolerance_on_convection_diffusion(prec):
    from paper_1904_12754_gb300 import mlmc as M
    a = I.convdiff_3d(10)
    t = 0.5
    v = np.random.default_rng(9).random(a.n)
    ref = R.expmv(a.scipy(), t, v)
    tol = 1e-2
    sched = M.schedule_default(precision=prec, num_levels=3, max_levels=10, mode=M.FORWARD,
                               time_budget_s=60.0)
    with M.Plan.from_csr(a, t, sched, rel_tol=tol, stream=stream_handle()) as plan:
        x = np.zeros(a.n)
        plan.expmv(v, x, seed=5)
        _, est = plan.stats()
        tc = plan.expmv_sum(v, seed=6)
        _, est_sum = plan.stats()
    err = np.linalg.norm(x - ref) / np.linalg.norm(ref)
    assert est <= tol and err <= 2.5 * tol, (est, err)
    assert est_sum <= tol and abs(tc - ref.sum()) <= 2.5 * tol * abs(ref.sum())


def test_forward_plans_rejected_where_rows_are_needed():
    from paper_1904_12754_gb300 import mlmc as M
    a, t, v = PROBLEMS["signed_301"]
    torch = torch_cuda()
    with _fwd_plan(a, t, 1) as plan:
        with pytest.raises(RuntimeError):
            plan.expmv_entry(3, v, seed=1)
        sched = M.schedule_default(precision=1)
        with pytest.raises(RuntimeError):
            M.Batch([plan], sched, rel_tol=1e-2, stream=stream_handle())
        rec = torch.zeros(a.n * 4 * M.WALK_RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        dv = torch.from_numpy(v).cuda()
        with pytest.raises(RuntimeError):
            plan.trace_noalloc(2, False, 0, 4, dv, 1, rec)
        torch.cuda.synchronize()


def test_forward_zero_rhs_gives_zero():
    from paper_1904_12754_gb300 import mlmc as M
    a, t, _ = PROBLEMS["signed_301"]
    with _fwd_plan(a, t, 1) as plan:
        x = np.full(a.n, 7.0)
        plan.expmv(np.zeros(a.n), x, seed=1)
    assert np.all(x == 0.0)
